// pa_schedule.cu -- chunk schedules of the host-buffer path (host logic only).
//
// pa_beamform_host moves frames through three stages per chunk: the upload
// of the chunk's RF, its launch sequence (clear, fused kernel, post-filter,
// log) and the download of its images.  Uploads run one at a time, launch
// sequences run one at a time (each waits for the previous chunk's), and so
// do downloads; a chunk's upload also waits until the download that last used
// its buffer set is done.  The fused kernel is persistent: a launch of f
// frames runs ceil(f * items / resident) waves of thread blocks, so chunk
// sizes that fill the last wave waste nothing there (as far as the items
// cost the same: cheap items at the end of the work list fill a partial last
// wave, which wave_share expresses).  The model below gives
// the makespan of a schedule; the search picks the best schedule of a
// parametrised family (short head, evenly sized middle chunks, a tail whose
// chunks shrink so that each download hides behind the next, smaller,
// launch sequence).

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "pa_internal.cuh"
#include "pa_schedule.h"

namespace {
pa_status sfail(pa_status s, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  pa::set_error_message(buf);
  return s;
}
}  // namespace

namespace pa {

double pipe_makespan(const pa_pipe_model& m, const int32_t* ch, int n) {
  const int sets = std::max(1, std::min(m.n_sets, 8));
  double buf[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  double up_free = 0.0, k_free = 0.0, down_free = 0.0, end = 0.0;
  const double items = std::max(1, m.items_per_frame);
  const double res = std::max(1, m.resident);
  const double q = std::min(1.0, std::max(0.0, m.wave_share));
  for (int c = 0; c < n; ++c) {
    const double f = ch[c];
    const int b = c % sets;
    const double us = std::max(up_free, buf[b]);
    const double ue = us + f * m.upload_us;
    up_free = ue;
    const double ks = std::max(ue, k_free);
    const double w = f * items / res;  // waves of the fused kernel
    const double ke =
        ks + f * m.kernel_us * ((1.0 - q) + q * std::ceil(w - 1e-9) / w) + m.launch_us;
    k_free = ke;
    const double ds = std::max(ke, down_free);
    const double de = ds + f * m.download_us;
    down_free = de;
    buf[b] = de;
    end = std::max(end, de);
  }
  return end;
}

// Search over head a, middle chunk size mid, first tail chunk t1 and tail
// ratio rho (and the single chunk).  Middle sizes that would need more than
// 256 middle chunks are skipped, except chunks of cap frames, so the cost
// stays bounded for long calls.
std::vector<int32_t> pipe_search(const pa_pipe_model& m, int n, int cap) {
  std::vector<int32_t> best, ch;
  if (n <= 0) return best;
  cap = std::max(1, std::min(cap, n));
  double best_t = 0.0;
  if (n <= cap) {  // one chunk
    best.assign(1, n);
    best_t = pipe_makespan(m, best.data(), 1);
  }
  const double rhos[4] = {0.3, 0.45, 0.6, 0.75};
  std::vector<int32_t> tail;
  for (int a = 1; a <= std::min(cap, 8); ++a) {
    for (int t1 = 0; t1 <= std::min(cap, 16); ++t1) {
      for (int ri = 0; ri < (t1 > 1 ? 4 : 1); ++ri) {
        tail.clear();
        for (int t = t1; t >= 1;) {
          tail.push_back(t);
          int nt = (int)std::floor(t * rhos[ri]);
          t = std::min(nt, t - 1);
        }
        int rest = n - a;
        for (int t : tail) rest -= t;
        if (rest < 0) continue;
        for (int mid = 1; mid <= cap; ++mid) {
          if (rest == 0 && mid > 1) break;
          if (rest / mid > 256 && mid != cap) continue;  // long calls: full chunks only
          ch.clear();
          ch.push_back(a);
          if (rest % mid) ch.push_back(rest % mid);
          for (int q = 0; q < rest / mid; ++q) ch.push_back(mid);
          ch.insert(ch.end(), tail.begin(), tail.end());
          const double t = pipe_makespan(m, ch.data(), (int)ch.size());
          if (best.empty() || t < best_t - 1e-9) {
            best = ch;
            best_t = t;
          }
        }
      }
    }
  }
  return best;
}

}  // namespace pa

extern "C" {

pa_status pa_pipe_time(const pa_pipe_model* m, const int32_t* chunks, int32_t n_chunks,
                       double* us) {
  if (!m || !us || (n_chunks > 0 && !chunks)) return sfail(PA_EINVAL, "null argument");
  if (n_chunks < 0) return sfail(PA_EINVAL, "n_chunks < 0");
  if (m->items_per_frame < 1 || m->resident < 1 || m->n_sets < 1 || m->n_sets > 8)
    return sfail(PA_EINVAL, "model needs items_per_frame, resident >= 1, n_sets 1..8");
  for (int c = 0; c < n_chunks; ++c)
    if (chunks[c] < 1) return sfail(PA_EINVAL, "chunk %d has %d frames", c, chunks[c]);
  *us = pa::pipe_makespan(*m, chunks, n_chunks);
  return PA_OK;
}

pa_status pa_pipe_schedule(const pa_pipe_model* m, int32_t n_frames, int32_t max_chunk,
                           int32_t* chunks, int32_t max_chunks, int32_t* n_chunks) {
  if (!m || !chunks || !n_chunks) return sfail(PA_EINVAL, "null argument");
  if (n_frames < 1 || max_chunk < 1) return sfail(PA_EINVAL, "n_frames, max_chunk >= 1");
  if (m->items_per_frame < 1 || m->resident < 1 || m->n_sets < 1 || m->n_sets > 8)
    return sfail(PA_EINVAL, "model needs items_per_frame, resident >= 1, n_sets 1..8");
  const std::vector<int32_t> s = pa::pipe_search(*m, n_frames, max_chunk);
  if ((int)s.size() > max_chunks)
    return sfail(PA_EINVAL, "schedule has %d chunks, room for %d", (int)s.size(),
                           max_chunks);
  std::copy(s.begin(), s.end(), chunks);
  *n_chunks = (int32_t)s.size();
  return PA_OK;
}

}  // extern "C"
