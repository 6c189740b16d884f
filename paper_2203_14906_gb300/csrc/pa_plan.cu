// pa_plan.cu -- host side of the C ABI: descriptor validation, tile
// configuration, the plan-time delay / apodisation table kernel (Section 5:
// delays are computed once and kept resident in device memory), per-tile RF
// windows, post-filter masks, and the launch sequence of pa_beamform.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "pa_internal.cuh"
#include "pa_schedule.h"

using namespace pa;

// ------------------------------------------------------------------ errors
namespace {
thread_local std::string g_err;

pa_status fail(pa_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define PA_CUDA(call)                                                         \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess)                                                    \
      return fail(PA_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

int popcount3(uint32_t m) { return (int)((m & 1u) + ((m >> 1) & 1u) + ((m >> 2) & 1u)); }

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};
}  // namespace

// ------------------------------------------------------------------- plan
// Buffer sets (and streams) of the host-buffer path.
constexpr int kHostSets = 3;

struct pa_plan_s {
  pa_plan_desc d{};
  int device = 0, num_sms = 0;
  int K = 1;
  bool apod = false, comp = false;
  bool full = false;  // per-pixel delay table (PA_TABLE_FULL) instead of the lattice
  // tiling
  int m = 1, R = 1, slots = 1, warps = 1, ngroups = 1, threads = 32;
  int tile_x = 0, tile_z = 32, nxt = 0, nzt = 0, n_tiles = 0, nx_pad = 0, nz_pad = 0;
  int u0 = 0, u1 = 0, nv = 0, dmin = 0, ndrows = 0, window = 0;
  size_t full_entries = 0;  // entries of the full table (n_tiles * (steps + 3) * 32 * slots * kC)
  size_t smem = 0;
  int blocks_per_sm = 0;
  bool use_tma = false;
  int lo_align = 4;   // window starts are multiples of this many samples
  int nc = 32;        // channel steps per staged chunk (multiple of kC)
  int tmem_cols = 0;  // TMEM columns per fused-kernel block (compensated sums)
  int expect_extra = 0;   // > 0 only under PA_INJECT_TMA_SHORTFALL (tests the bounded wait)
  long long timeouts_seen = 0;  // timed-out waits already reported by pa_beamform_host
  int wr = 0;         // raw samples per channel delivered by one TMA box
  int rp = 0;         // raw-buffer row pitch in samples (128-byte aligned rows)
  int pairs_off = 0;  // shared-memory offset of the interpolation slots
  // post
  int M = 1, log2M = 0, post_wpb = 1, n_out = 0, n_tw = 0;
  int out_id[3] = {-1, -1, -1};  // output slot (0..n_out) of DAS, DMAS, HO
  uint32_t warnings = 0;
  float dyn_range = 60.f;
  // device memory
  int2* table = nullptr;     // lattice table
  int2* ftab = nullptr;      // full table (see k_table_full)
  float* wtab = nullptr;
  int* lo = nullptr;
  int2* urange = nullptr;
  int2* vchunks = nullptr;
  int4* items = nullptr;   // work-item table (tile, group, tx, tz)
  int2* slot_rg = nullptr; // warp slot -> (column residue, column group)
  float2* tw = nullptr;
  float* mask = nullptr;
  // [err, counter, maxslots..., timeouts]; [0] serves pa_beamform, all three
  // the buffer sets of pa_beamform_host
  int* scratch[kHostSets] = {nullptr, nullptr, nullptr};
  size_t scratch_ints = 0;
  // host-buffer path
  void* h_rf = nullptr;
  float* h_out = nullptr;
  size_t h_rf_bytes = 0, h_out_bytes = 0;
  cudaStream_t hs[kHostSets] = {nullptr, nullptr, nullptr};
  cudaEvent_t h_ev = nullptr;
  cudaEvent_t h_done[kHostSets] = {nullptr, nullptr, nullptr};
  // chunk schedules of the host path, per (frames, stages): every candidate
  // timed once, the three fastest once more, then the fastest kept
  struct HostTune {
    int nf = 0;
    uint32_t stages = 0;
    std::vector<std::vector<int32_t>> cand;
    std::vector<double> best_ms;  // < 0: not measured yet
    std::vector<int> order;       // candidates in the order they are timed
    size_t pos = 0;
    int attempts = 0;             // uncounted (cold) calls of order[pos]
    bool second_round = false;
    int chosen = -1;              // index into cand once tuned
    std::vector<int32_t> fixed;   // set by pa_plan_set_host_schedule
    const std::vector<int32_t>& current() const {
      return !fixed.empty() ? fixed : cand[chosen >= 0 ? chosen : order[pos]];
    }
  };
  std::vector<HostTune> tunes;
  long long graph_builds = 0;  // executable graphs instantiated so far
  // whole host-path calls as graphs (pinned host buffers): every chunk's
  // upload, launch sequence and download, per (frames, stages, schedule);
  // they name the staging buffers, so growing those drops them
  struct HostGraph {
    int nf = 0;
    uint32_t stages = 0;
    std::vector<int32_t> sched;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphNode_t> up, down;  // per chunk
    std::vector<void*> up_dev, down_dev;
    std::vector<size_t> up_off, down_off, up_bytes, down_bytes;
    const void* rf_host = nullptr;
    float* out_host = nullptr;
  };
  std::vector<HostGraph> host_graphs;
  // CUDA graphs of the launch sequence, one per (frames, stages)
  struct GraphEntry {
    int nf = 0;
    uint32_t stages = 0;
    cudaGraph_t graph = nullptr;  // kept alive: exec-node updates name its nodes
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t n_memset = nullptr;  // clearing kernel
    cudaGraphNode_t n_bf = nullptr, n_post = nullptr, n_log = nullptr;
    // timing graphs (built while pa_plan_profile is on): an event-record
    // node before and after each kernel, given fresh events every launch
    uint32_t prof = 0;  // kernel kinds timed (bit per kind)
    cudaGraphNode_t n_ev[3][2] = {};
  };
  std::vector<GraphEntry> graphs;
  bool use_graph = true;
  int lane_rows_log2 = 5;  // depth rows per lane group of the fused kernel (log2)
  int table_zb = 0;        // lattice table layout: 0 row-major, else log2 depth-block height
  // kernel timing (pa_plan_profile): bit k set = kernel kind k is timed
  uint32_t prof = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_free;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
  // facts
  int64_t active_pairs = 0, executed_pairs = 0;
  size_t device_bytes = 0;
  size_t elt = 4;
};

namespace {

// ---------------------------------------------------------- plan kernels
// Layout of the full table, in the order the fused kernel reads it: per
// tile, channel step u' = u - u0 (steps + 3 of them: the last three are
// padding, so the kernel loads two steps ahead with no bound check), half h
// = c / 2 of a thread's kC = 4 pixels, thread t = (rg * slots + sl) * LR + zl
// of the tile (row group rg of the tile's 32 rows, warp slot sl, row zl
// within the group) and pixel c % 2:
//   (((tile * (steps + 3) + u') * 2 + h) * (32 slots) + t) * 2 + c % 2
// with LR depth rows per lane group and RG = 32 / LR.  A thread loads a step
// as two 16-byte entries pairs; the 32 lanes of a warp read each of them as
// 512 contiguous bytes.
struct FullGeom {
  int nxt, n_tiles, tile_x, tile_z, m, slots, steps, lr_log2, nx, nz, n_elem, u0, nv;
};

static_assert(kC == 4, "the full table splits a thread's step into two entry pairs");

__host__ __device__ __forceinline__ size_t full_index(const FullGeom& f, int tile, int up, int c,
                                                     int sl, int zt) {
  const int lr = 1 << f.lr_log2;
  const int rg = zt >> f.lr_log2, zl = zt & (lr - 1);
  const size_t threads = (size_t)32 * f.slots;
  const size_t t = ((size_t)rg * f.slots + sl) * lr + zl;
  return ((((size_t)tile * (f.steps + 3) + up) * 2 + (c >> 1)) * threads + t) * 2 + (c & 1);
}

// Entries of one tile in the full table.
__host__ __device__ __forceinline__ size_t full_per_tile(const FullGeom& f) {
  return (size_t)(f.steps + 3) * 32 * f.slots * kC;
}

// (step, pixel, slot, row in the tile) of entry e of a tile.
__device__ __forceinline__ void full_decode(const FullGeom& f, size_t e, int* up, int* c, int* sl,
                                            int* zt) {
  const int lr = 1 << f.lr_log2;
  const size_t threads = (size_t)32 * f.slots;
  const int c_lo = (int)(e & 1);
  size_t q = e >> 1;
  const size_t t = q % threads;
  q /= threads;
  *c = (int)(q & 1) * 2 + c_lo;
  *up = (int)(q >> 1);
  const int zl = (int)(t % lr);
  const size_t t2 = t / lr;
  *sl = (int)(t2 % f.slots);
  const int rg = (int)(t2 / f.slots);
  *zt = rg * lr + zl;
}

// Pixel column of pixel c of warp slot sl in tile column tx.
__host__ __device__ __forceinline__ int full_column(const FullGeom& f, int tx, int sl, int c) {
  return tx * f.tile_x + (sl / f.m) * f.m * kC + (sl % f.m) + f.m * c;
}

struct TableGeom {
  int ndrows, nzp, dmin, ns, nearest, zb;
  double x_const;  // x0 + (N-1)/2 pitch: dx of lattice offset d is x_const + (d + 1/2) dx
  double dx, z0, dz, fs, c, t0, fnum;
  // full table: element i = v + u0 of N at x_i = (i - (N-1)/2) pitch
  double x0, pitch;
  int n_elem, u0, nv;
};

// The one-way time of flight in samples from a pixel at lateral offset dxv
// from the element and depth zp, tau = fs (r / c - t0), as the integer sample
// n0 = floor(tau) and the fraction a = tau - n0 (nearest-sample delays,
// Eq. 1: n0 = round(tau), a = 0).
__device__ void delay_sample(const TableGeom& g, double dxv, double zp, int* n0_out,
                             double* a_out) {
  const double tau = g.fs * (sqrt(dxv * dxv + zp * zp) / g.c - g.t0);
  double fl = g.nearest ? floor(tau + 0.5) : floor(tau);
  double a = g.nearest ? 0.0 : tau - fl;
  const double lim = 1048576.0;
  if (fl < -lim) { fl = -lim; a = 0.0; }
  if (fl > lim) { fl = lim; a = 0.0; }
  int n0 = (int)fl;
  // A delay whose taps leave the record contributes nothing (s = 0).  Staged
  // samples outside [0, Ns) are zero, so pointing such delays at a slot whose
  // two taps both lie outside the record gives s = 0 with no test per pair:
  // n0 = -1 (taps -1, 0) moves to -2, n0 = Ns-1 (taps Ns-1, Ns) moves to Ns.
  // (With a = 0 the nearest sample reads only the first tap: slots n0 = -1 and
  // n0 = Ns-1 already give 0 and r[Ns-1], so no remapping is needed.)
  if (!g.nearest && n0 == -1) n0 = -2;
  if (!g.nearest && n0 == g.ns - 1) n0 = g.ns;
  *n0_out = n0;
  *a_out = a;
}

// Hann dynamic-aperture weight of an element at lateral offset dxv from a
// pixel at depth zp (0 outside the aperture |dxv| <= zp / (2F)).
__device__ float apod_weight(const TableGeom& g, double dxv, double zp) {
  float w = 0.f;
  const double half = zp / (2.0 * g.fnum);
  if (half > 0.0 && fabs(dxv) <= half) {
    const double cw = cos(3.14159265358979323846 * dxv / (2.0 * half));
    w = (float)(cw * cw);
  }
  return w;
}

// Lateral offset x_j - x_i of pixel column j and virtual channel v (element
// i = v + u0), both positions computed as the grid and the array define them.
__device__ double full_dx(const TableGeom& g, int j, int v) {
  const double xp = g.x0 + ((double)j + 0.5) * g.dx;
  const double xi = ((double)(v + g.u0) - 0.5 * (double)(g.n_elem - 1)) * g.pitch;
  return xp - xi;
}

__device__ double pixel_z(const TableGeom& g, int z) { return g.z0 + ((double)z + 0.5) * g.dz; }

// Lattice table: every lattice offset d = j - m i and depth row, entry
// {n0 * 8 (the byte stride of an interpolation slot), FP32 bits of a}.
__global__ void k_table(TableGeom g, int2* table, float* wtab) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = blockIdx.y;
  if (z >= g.nzp || row >= g.ndrows) return;
  const double dxv = g.x_const + ((double)(g.dmin + row) + 0.5) * g.dx;
  const double zp = pixel_z(g, z);
  int n0;
  double a;
  delay_sample(g, dxv, zp, &n0, &a);
  const size_t ti = table_index(row, z, g.ndrows, g.nzp, g.zb);
  table[ti] = make_int2(n0 * 8, __float_as_int((float)a));
  if (wtab) wtab[ti] = apod_weight(g, dxv, zp);
}

// Full table: the entry of every (pixel, channel step) pair the fused kernel
// evaluates (pixel c of slot sl pairs with channel u + c at step u), in the
// layout of full_index: {(n0 - lo) * 8, FP32 bits of a}, the sample relative
// to the RF window its tile stages for that channel (lo, from
// k_windows_full) as a byte offset into the window's interpolation slots.
// The padding steps hold zeros.
__global__ void k_table_full(TableGeom g, FullGeom f, const int* lo, int2* table, float* wtab) {
  const int tile = blockIdx.y;
  const size_t per_tile = full_per_tile(f);
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= per_tile) return;
  int up, c, sl, zt;
  full_decode(f, e, &up, &c, &sl, &zt);
  const size_t ti = (size_t)tile * per_tile + e;
  if (up >= f.steps) {
    table[ti] = make_int2(0, 0);
    if (wtab) wtab[ti] = 0.f;
    return;
  }
  const int tx = tile % f.nxt, tz = tile / f.nxt;
  const int j = full_column(f, tx, sl, c);
  const int v = up + c;
  const double dxv = full_dx(g, j, v);
  const double zp = pixel_z(g, tz * f.tile_z + zt);
  int n0;
  double a;
  delay_sample(g, dxv, zp, &n0, &a);
  table[ti] = make_int2((n0 - lo[(size_t)tile * g.nv + v]) * 8, __float_as_int((float)a));
  if (wtab) wtab[ti] = apod_weight(g, dxv, zp);
}

// Pairs with a non-zero apodisation weight in the full table (real pixels
// and elements only).
__global__ void k_count_active_full(FullGeom f, const float* wtab, unsigned long long* count) {
  const int tile = blockIdx.y;
  const size_t per_tile = full_per_tile(f);
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long cnt = 0;
  if (e < per_tile) {
    int up, c, sl, zt;
    full_decode(f, e, &up, &c, &sl, &zt);
    const int j = full_column(f, tile % f.nxt, sl, c);
    const int z = (tile / f.nxt) * f.tile_z + zt;
    const int i = up + c + f.u0;
    if (up < f.steps && j < f.nx && z < f.nz && i >= 0 && i < f.n_elem &&
        wtab[(size_t)tile * per_tile + e] > 0.f)
      cnt = 1;
  }
  for (int s = 16; s >= 1; s >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, s);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(count, cnt);
}

struct TileGeom {
  int nxt, nzt, tile_x, tile_z, m, dmin, nzp, nv, u0, ndrows, zb;
  int full;  // 1: full table (laid out as full_index says)
};

// Lattice-table row of pixel column j and virtual channel v (offset
// d = j - m i, i = v + u0).
__device__ __forceinline__ int tile_row(const TileGeom& g, int j, int v) {
  return j - g.m * (v + g.u0) - g.dmin;
}

// First staged sample (rounded down to a multiple of 4) and window width of
// every (tile, virtual channel).  The delay grows with depth for z > 0, so the
// minimum over the tile is on its first row and the maximum on its last.
__global__ void k_windows(TileGeom g, int lo_align, const int2* table, int* lo, int* wmax,
                          int* err) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int tile = blockIdx.y;
  if (v >= g.nv) return;
  const int tx = tile % g.nxt, tz = tile / g.nxt;
  const int zf = tz * g.tile_z, zl = zf + g.tile_z - 1;
  int mn = 0x7fffffff, mx = -0x7fffffff;
  for (int jj = 0; jj < g.tile_x; ++jj) {
    const int row = tile_row(g, tx * g.tile_x + jj, v);
    if (row < 0 || row >= g.ndrows) {
      atomicOr(err, 4);
      continue;
    }
    mn = min(mn, table[table_index(row, zf, g.ndrows, g.nzp, g.zb)].x >> 3);
    mx = max(mx, table[table_index(row, zl, g.ndrows, g.nzp, g.zb)].x >> 3);
  }
  const int lo_al = mn & ~(lo_align - 1);  // lo_align is a power of two
  lo[(size_t)tile * g.nv + v] = lo_al;
  atomicMax(wmax, mx - lo_al + 1);
}

// The same windows for the full table, from the delays themselves (the
// packed table is written relative to them afterwards).
__global__ void k_windows_full(TableGeom tg, TileGeom g, int lo_align, int* lo, int* wmax) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int tile = blockIdx.y;
  if (v >= g.nv) return;
  const int tx = tile % g.nxt, tz = tile / g.nxt;
  const int zf = tz * g.tile_z, zl = zf + g.tile_z - 1;
  int mn = 0x7fffffff, mx = -0x7fffffff;
  for (int jj = 0; jj < g.tile_x; ++jj) {
    const double dxv = full_dx(tg, tx * g.tile_x + jj, v);
    int n0;
    double a;
    delay_sample(tg, dxv, pixel_z(tg, zf), &n0, &a);
    mn = min(mn, n0);
    delay_sample(tg, dxv, pixel_z(tg, zl), &n0, &a);
    mx = max(mx, n0);
  }
  const int lo_al = mn & ~(lo_align - 1);
  lo[(size_t)tile * g.nv + v] = lo_al;
  atomicMax(wmax, mx - lo_al + 1);
}

// Channel-step range of every warp slot.  Without apodisation every step is
// evaluated; with it, only steps whose lattice offset has a non-zero weight on
// the warp's deepest row (the widest aperture of its rows).
__global__ void k_uranges(TileGeom g, FullGeom f, int slots, int u1, int kc, const float* wtab,
                          int2* urange) {
  const int sl = blockIdx.x * blockDim.x + threadIdx.x;
  const int tile = blockIdx.y;
  if (sl >= slots) return;
  int2 r = make_int2(g.u0, u1);
  if (wtab) {
    const int tx = tile % g.nxt, tz = tile / g.nxt;
    const int r_m = sl % g.m, grp = sl / g.m;
    const int jt = tx * g.tile_x + grp * g.m * kc + r_m;
    const int zl = tz * g.tile_z + g.tile_z - 1;
    int ua = u1, ub = g.u0;
    for (int u = g.u0; u < u1; ++u) {
      // lattice: the kC pixels of the slot share one entry at step u; full:
      // pixel c (column jt + m c) pairs with channel u + c, each its own entry
      bool on = false;
      if (g.full) {
        for (int c = 0; c < kc; ++c)
          on |= wtab[full_index(f, tile, u - g.u0, c, sl, g.tile_z - 1)] > 0.f;
      } else {
        const int row = tile_row(g, jt, u - g.u0);
        if (row >= 0 && row < g.ndrows) on = wtab[table_index(row, zl, g.ndrows, g.nzp, g.zb)] > 0.f;
      }
      if (on) {
        ua = min(ua, u);
        ub = max(ub, u + 1);
      }
    }
    if (ua >= ub) {
      r = make_int2(g.u0, g.u0);
    } else {
      ua = g.u0 + ((ua - g.u0) / kc) * kc;
      ub = g.u0 + ((ub - g.u0 + kc - 1) / kc) * kc;
      r = make_int2(ua, ub);
    }
  }
  urange[(size_t)tile * slots + sl] = r;
}

// Clears the work counter and image maxima before a launch sequence.
__global__ void k_zero_ints(int* p, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = 0;
}

// Pairs with a non-zero apodisation weight (for the active-pair rate).
__global__ void k_count_active(TileGeom g, int nx, int nz, int n, const float* wtab,
                               unsigned long long* count) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  unsigned long long c = 0;
  if (z < nz) {
    for (int i = 0; i < n; ++i) {
      const int row = tile_row(g, j, i - g.u0);
      if (wtab[table_index(row, z, g.ndrows, g.nzp, g.zb)] > 0.f) ++c;
    }
  }
  for (int s = 16; s >= 1; s >>= 1) c += __shfl_xor_sync(0xffffffffu, c, s);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// -------------------------------------------------------- host helpers
double band_weight(double f, double lo, double hi, double roll) {
  if (f >= lo && f <= hi) return 1.0;
  const double u = (f < lo) ? (lo - f) : (f - hi);
  if (u < roll) return 0.5 * (1.0 + std::cos(M_PI * u / roll));
  return 0.0;
}

// Real post-filter mask of one output: raised-cosine band (order-dependent
// default band, or the descriptor's) times the analytic-signal weights.
// Returns true when the band lies wholly above the axial Nyquist rate, in
// which case only DC is removed.
bool build_mask(const pa_plan_desc& d, bool even_order, int M, float* out) {
  const double dz = (d.z1_m - d.z0_m) / d.nz;
  const double f_nyq = d.c_m_s / (2.0 * dz);
  const double f0 = d.f0_hz;
  const double roll = 0.25 * f0;
  const bool off = d.band_hi_hz < 0.0;
  double lo, hi;
  if (d.band_lo_hz > 0.0 && d.band_hi_hz > 0.0) {
    lo = d.band_lo_hz;
    hi = d.band_hi_hz;
  } else if (even_order) {
    lo = 1.5 * f0;
    hi = 2.5 * f0;
  } else {
    lo = 0.5 * f0;
    hi = 1.5 * f0;
  }
  const bool dc_only = !off && lo >= f_nyq;
  hi = std::min(hi, f_nyq);
  for (int b = 0; b < M; ++b) {
    double an = (b == 0 || 2 * b == M) ? 1.0 : (2 * b < M ? 2.0 : 0.0);
    double bp;
    if (an == 0.0) bp = 0.0;
    else if (off) bp = 1.0;
    else if (dc_only) bp = (b == 0) ? 0.0 : 1.0;
    else bp = band_weight(d.c_m_s * b / (M * dz), lo, hi, roll);
    out[b] = (float)(bp * an);
  }
  return dc_only;
}

// pitch / lateral pixel pitch when it is an integer m in 1..32 (the lattice
// table applies), else 0.
int lattice_m(const pa_plan_desc& d) {
  const double dx = (d.x1_m - d.x0_m) / d.nx;
  const double mr = d.pitch_m / dx;
  const double mi = std::round(mr);
  if (mi < 1 || mi > 32 || std::fabs(mr - mi) > 1e-6 * mi) return 0;
  return (int)mi;
}

pa_status validate(const pa_plan_desc* d) {
  if (!d) return fail(PA_EINVAL, "null descriptor");
  if (d->n_elem < 1) return fail(PA_EINVAL, "n_elem must be >= 1 (got %d)", d->n_elem);
  if (d->n_samples < 2) return fail(PA_EINVAL, "n_samples must be >= 2 (got %d)", d->n_samples);
  if (d->nx < 1 || d->nz < 1) return fail(PA_EINVAL, "empty image grid %dx%d", d->nx, d->nz);
  if (d->order_k < 1 || d->order_k > kMaxOrder)
    return fail(PA_EINVAL, "order_k must be in 1..%d (got %d)", kMaxOrder, d->order_k);
  if (d->n_elem < d->order_k)
    return fail(PA_EINVAL, "order_k=%d needs at least as many elements (n_elem=%d)", d->order_k,
                d->n_elem);
  if (!(d->pitch_m > 0) || !(d->c_m_s > 0) || !(d->fs_hz > 0))
    return fail(PA_EINVAL, "pitch, c and fs must be positive");
  if (!(d->x1_m > d->x0_m) || !(d->z1_m > d->z0_m))
    return fail(PA_EINVAL, "grid extents must be increasing");
  if (d->z0_m < 0) return fail(PA_EINVAL, "z0 must be >= 0 (pixels in front of the array)");
  if ((d->outputs & 7u) == 0 || (d->outputs & ~7u))
    return fail(PA_EINVAL, "outputs mask 0x%x invalid", d->outputs);
  if (d->rf_dtype != PA_RF_F32 && d->rf_dtype != PA_RF_BF16 && d->rf_dtype != PA_RF_F16)
    return fail(PA_EINVAL, "rf_dtype %d invalid", (int)d->rf_dtype);
  if (d->f_number < 0) return fail(PA_EINVAL, "f_number must be >= 0");
  if (d->interp != PA_INTERP_LINEAR && d->interp != PA_INTERP_NEAREST)
    return fail(PA_EINVAL, "interp %d invalid", (int)d->interp);
  if (d->f_number > 0 || d->band_hi_hz >= 0) {
    if (!(d->f0_hz > 0) && !(d->band_lo_hz > 0 && d->band_hi_hz > 0) && d->band_hi_hz >= 0)
      return fail(PA_EINVAL, "f0_hz must be positive for the default band");
  }
  if (d->max_batch > 65535) return fail(PA_EINVAL, "max_batch must be <= 65535");
  if (d->delay_table != PA_TABLE_AUTO && d->delay_table != PA_TABLE_LATTICE &&
      d->delay_table != PA_TABLE_FULL)
    return fail(PA_EINVAL, "delay_table %d invalid", (int)d->delay_table);
  if (d->delay_table == PA_TABLE_LATTICE && lattice_m(*d) == 0)
    return fail(PA_EINVAL,
                "pitch / lateral pixel pitch = %.9g is not an integer in 1..32: the lattice "
                "delay table needs (x1-x0)/nx = pitch/m (PA_TABLE_AUTO or PA_TABLE_FULL take "
                "any grid)",
                d->pitch_m * d->nx / (d->x1_m - d->x0_m));
  return PA_OK;
}

// Tiling from the descriptor alone (no device work).
void configure(pa_plan_s* P) {
  const pa_plan_desc& d = P->d;
  P->K = d.order_k;
  P->apod = d.f_number > 0;
  P->comp = d.compensated != 0;
  const double dx = (d.x1_m - d.x0_m) / d.nx;
  const int lm = lattice_m(d);
  P->full = d.delay_table == PA_TABLE_FULL || (d.delay_table == PA_TABLE_AUTO && lm == 0);
  // 32-column tiles halve the staged samples per pair; small images keep
  // 16-column tiles so that there are enough tiles to fill the GPU, unless a
  // full launch (max_batch frames) holds at least 1024 32 x 32 tiles.
  const int64_t wide_tiles =
      (int64_t)((d.nx + 31) / 32) * ((d.nz + 31) / 32) * std::max(1, d.max_batch);
  const bool big = (int64_t)d.nx * d.nz >= 512 * 512 || wide_tiles >= 1024;
  if (P->full) {
    // No table entry is shared, so the column stride m of a thread's pixels
    // is free: 4 (as the lattice has at cfg2) keeps a warp's slots on
    // neighbouring columns, whose delays for one channel differ least, so
    // its shared-memory gathers stay narrow.  The RF window of a tile spans
    // the delays over its lateral extent: tiles stay within ~3.2 mm.
    int cols = big ? 32 : 16;
    while (cols > 8 && cols * dx > 3.2e-3) cols /= 2;
    P->m = cols >= 16 ? 4 : 2;
    P->R = cols / (P->m * kC);
  } else {
    P->m = lm;
    P->R = std::max(1, (big ? 8 : 4) / P->m);
  }
  P->slots = P->m * P->R;
  int B = 1;
  for (int b = 1; b <= 8; ++b)
    if (P->slots % b == 0) B = b;
  if (B == 1) {  // prime m > 8: pair up column groups so a block has two warps
    P->R *= 2;
    P->slots *= 2;
    B = 2;
  }
  P->warps = B;
  P->ngroups = P->slots / B;
  // Lane groups of 8 rows x 4 neighbouring slots (a half-warp's shared
  // gather spans ~18 slots instead of ~32) for orders <= 4 without
  // apodisation, where the block's warps split that way.  Apodised plans
  // keep 32 rows x 1 slot, because a warp iterates over the union of its
  // slots' channel ranges; orders >= 5 are arithmetic-bound and lose to the
  // split table loads of 8-row groups.  Measured on GB300 (fused kernel per
  // launch, 32 -> 8 rows): cfg2 FP32 k = 1, 2 0.594 -> 0.488 ms, k = 3
  // 0.651 -> 0.641 ms, k = 4 0.701 -> 0.692 ms, k = 5 0.831 -> 0.837 ms,
  // k = 7 1.280 -> 1.339 ms; cfg5 (apodised) 2.91 -> 3.06 ms; 16-row groups
  // were never the fastest, and 4-row groups (8 slots per warp) were slower
  // still (k = 2 0.488 -> 0.615 ms, k = 3 0.619 -> 0.671 ms).
  // PA_LANE_ROWS=32|16|8 picks one, for comparisons.
  P->lane_rows_log2 = (B % 4 == 0 && !P->apod && P->K <= 4) ? 3 : 5;
  // Compensated sums keep their Kahan totals in TMEM; its accesses are
  // warp-wide, so every lane of a warp must run the same channel steps:
  // apodised plans (per-slot channel ranges) then keep one slot per warp.
  P->tmem_cols = P->comp ? tmem_columns(B, P->K <= 2 ? 3 : P->K + 2) : 0;
  if (const char* e = getenv("PA_LANE_ROWS")) {
    const int want = atoi(e) == 8 ? 3 : (atoi(e) == 16 ? 4 : 5);
    if (B % (1 << (5 - want)) == 0 && !(P->tmem_cols && P->apod)) P->lane_rows_log2 = want;
  }
  // Lattice table layout: depth blocks of 8 rows (a warp's four lattice
  // rows at one step in one contiguous 256-byte run: half the L1 wavefronts
  // of four 64-byte pieces) where that measured faster, row-major elsewhere.
  // Measured on GB300 (fused kernel per launch, one run, against row-major):
  // cfg2 k = 1, 2 0.488 -> 0.458 ms (bound by the L1 data pipe), BF16 +
  // Kahan k = 3 0.662 -> 0.653 ms, cfg3 BF16 + Kahan 1.261 -> 1.236 ms; but
  // plain FP32 k = 3 0.617 -> 0.628 ms, and blocks of 32 rows were slower
  // than row-major for every plan tried (k = 5 0.819 -> 0.838 ms, the cfg5
  // batch 2.675 -> 2.790 ms) although a warp's loads have the same shape.
  // (8-row lane groups imply no apodisation; the fused kernel computes the
  // blocked address only in the instantiations for k <= 2 or compensated
  // sums without apodisation.)
  P->table_zb = (P->lane_rows_log2 == 3 && !P->apod && (P->K <= 2 || P->comp)) ? 3 : 0;
  P->threads = 32 * B;
  P->tile_x = P->m * kC * P->R;
  P->tile_z = 32;
  P->nxt = (d.nx + P->tile_x - 1) / P->tile_x;
  P->nzt = (d.nz + P->tile_z - 1) / P->tile_z;
  P->n_tiles = P->nxt * P->nzt;
  P->nx_pad = P->nxt * P->tile_x;
  P->nz_pad = P->nzt * P->tile_z;
  P->u0 = -(kC - 1);
  const int steps = ((d.n_elem + kC - 1 + kC - 1) / kC) * kC;  // round N + kC - 1 up
  P->u1 = P->u0 + steps;
  const int i_max = P->u1 - 1 + kC - 1;
  P->nv = i_max - P->u0 + 1;
  if (P->full) {  // one entry per evaluated (pixel, channel step) pair
    P->dmin = 0;
    P->ndrows = 0;
    P->full_entries = (size_t)P->n_tiles * (steps + 3) * 32 * P->slots * kC;
  } else {
    P->dmin = -P->m * i_max;
    const int dmax = P->nx_pad - 1 + P->m * (kC - 1);
    P->ndrows = dmax - P->dmin + 1;
  }
  P->M = 1;
  P->log2M = 0;
  while (P->M < d.nz) {
    P->M <<= 1;
    ++P->log2M;
  }
  // warps per post block: most resident warps per SM for the shared memory
  // they need (post_buffers padded M-point buffers per team of
  // post_team_warps warps, plus the twiddles and mask), in whole teams
  {
    const int tw_warps = post_team_warps(P->M);
    const size_t per_team = (size_t)post_buffers(P->M) * post_padded_len(P->M) * sizeof(float2);
    const size_t tw = (size_t)P->M * (sizeof(float2) + sizeof(float));  // twiddles + mask
    const size_t sm_bytes = 227 * 1024;
    int best = tw_warps;
    size_t best_warps = 0;
    for (int w = tw_warps; w <= 8; w += tw_warps) {
      const size_t blk = (w / tw_warps) * per_team + tw + 1024;
      const size_t warps = (sm_bytes / blk) * w;
      if (blk <= 200 * 1024 && warps > best_warps) {
        best_warps = warps;
        best = w;
      }
    }
    P->post_wpb = best;
  }
  P->n_out = popcount3(d.outputs);
  int s = 0;
  for (int o = 0; o < 3; ++o) P->out_id[o] = (d.outputs >> o & 1u) ? s++ : -1;
  P->dyn_range = d.dyn_range_db > 0 ? (float)d.dyn_range_db : 60.f;
  P->elt = d.rf_dtype == PA_RF_F32 ? 4 : 2;
  // TMA boxes start on 16-byte boundaries: window starts are multiples of
  // 16 / elt samples, and rows must be 16-byte strided.
  P->lo_align = (int)(16 / P->elt);
  // Measured on GB300: TMA staging wins for 16-bit RF (half-size raw buffer),
  // vectorised loads win for FP32 RF (the FP32 raw buffer costs a resident
  // block per SM).  PA_STAGING=tma|loads overrides the choice.
  P->use_tma = (d.n_samples % P->lo_align) == 0 && P->elt == 2;
  // Failure injection for tests, compiled into the checked build only: every
  // chunk expects 16 bytes more than its boxes deliver, so each block's
  // bounded wait runs out (about a second), sets error flag 8, counts a
  // timeout and ends.  Every box of the chunk has landed by then (only the
  // expected count is short), so no copy is left in flight.
#ifdef PA_CHECK_BOUNDS
  P->expect_extra = getenv("PA_INJECT_TMA_SHORTFALL") ? 16 : 0;
#endif
  const char* staging = getenv("PA_STAGING");
  if (staging && strcmp(staging, "loads") == 0) P->use_tma = false;
  if (staging && strcmp(staging, "tma") == 0) P->use_tma = (d.n_samples % P->lo_align) == 0;
  if (P->d.max_batch <= 0) P->d.max_batch = 1;
}

// Resident fused-kernel blocks per SM.  For plans that keep their Kahan
// totals in TMEM the count comes from the kernel's registers, shared memory
// and threads (the occupancy calculator reports one block per SM for a
// kernel that allocates tensor memory) and is capped so that the resident
// blocks' TMEM columns fit the SM's 512.
cudaError_t fused_blocks_per_sm(const pa_plan_s* P, size_t smem, int* n) {
  cudaError_t e = bf_occupancy(P->K, P->apod, P->comp, P->full, P->threads, smem, n);
  if (e != cudaSuccess || !P->tmem_cols) return e;
  cudaFuncAttributes a;
  e = cudaFuncGetAttributes(&a, bf_func(P->K, P->apod, P->comp, P->full));
  if (e != cudaSuccess) return e;
  int dev = 0, regs_sm = 0, smem_sm = 0, thr_sm = 0, blk_sm = 0, rsv = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  const int warps = (P->threads + 31) / 32;
  const int regs_warp = ((a.numRegs * 32 + 255) / 256) * 256;  // 256-register units per warp
  int b = std::min(regs_sm / std::max(1, regs_warp * warps), thr_sm / (32 * warps));
  b = std::min(b, (int)((size_t)smem_sm / (smem + a.sharedSizeBytes + (size_t)rsv)));
  b = std::min(b, blk_sm);
  *n = std::max(0, std::min(b, kTmemColsPerSm / P->tmem_cols));
  return cudaSuccess;
}

// Bytes of the delay table and its apodisation weights.
size_t delay_table_bytes(const pa_plan_s* P) {
  if (P->full) return P->full_entries * (sizeof(int2) + (P->apod ? sizeof(float) : 0));
  return (size_t)P->ndrows * P->nz_pad * (sizeof(int2) + (P->apod ? sizeof(float) : 0));
}

pa_status check_table_size(const pa_plan_s* P) {
  if (P->full && delay_table_bytes(P) > PA_FULL_TABLE_MAX_BYTES)
    return fail(PA_EUNSUPPORTED,
                "the full delay table of %zu entries (%zu bytes) exceeds "
                "PA_FULL_TABLE_MAX_BYTES",
                P->full_entries, delay_table_bytes(P));
  return PA_OK;
}

size_t table_bytes(const pa_plan_s* P) {
  size_t b = delay_table_bytes(P);
  b += (size_t)P->n_tiles * P->ngroups * sizeof(int4) + (size_t)P->slots * sizeof(int2);
  b += (size_t)P->n_tiles * P->nv * sizeof(int);
  b += (size_t)P->n_tiles * P->slots * sizeof(int2);
  b += (size_t)P->n_tiles * P->ngroups * sizeof(int2);
  b += (size_t)2 * P->M * sizeof(float2) + (size_t)3 * P->M * sizeof(float);
  return b;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

template <typename T>
pa_status dalloc(pa_plan_s* P, T** ptr, size_t n) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)ptr, n * sizeof(T));
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? PA_ENOMEM : PA_ECUDA, "cudaMalloc(%zu): %s",
                n * sizeof(T), cudaGetErrorString(e));
  }
  P->device_bytes += n * sizeof(T);
  return PA_OK;
}

void free_plan(pa_plan_s* P) {
  if (!P) return;
  DeviceGuard g(P->device);
  for (int s = 0; s < kHostSets; ++s)
    if (P->hs[s]) cudaStreamSynchronize(P->hs[s]);
  cudaFree(P->table);
  cudaFree(P->ftab);
  cudaFree(P->wtab);
  cudaFree(P->lo);
  cudaFree(P->urange);
  cudaFree(P->vchunks);
  cudaFree(P->items);
  cudaFree(P->slot_rg);
  cudaFree(P->tw);
  cudaFree(P->mask);
  for (int s = 0; s < kHostSets; ++s) cudaFree(P->scratch[s]);
  cudaFree(P->h_rf);
  cudaFree(P->h_out);
  for (int s = 0; s < kHostSets; ++s)
    if (P->hs[s]) cudaStreamDestroy(P->hs[s]);
  if (P->h_ev) cudaEventDestroy(P->h_ev);
  for (int s = 0; s < kHostSets; ++s)
    if (P->h_done[s]) cudaEventDestroy(P->h_done[s]);
  for (auto& g : P->graphs) {
    cudaGraphExecDestroy(g.exec);
    cudaGraphDestroy(g.graph);
  }
  for (auto& g : P->host_graphs) {
    cudaGraphExecDestroy(g.exec);
    cudaGraphDestroy(g.graph);
  }
  for (auto& e : P->ev_free) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  for (auto& e : P->ev_used) {
    cudaEventSynchronize(e.second.second);
    cudaEventDestroy(e.second.first);
    cudaEventDestroy(e.second.second);
  }
  delete P;
}

pa_status build_plan(pa_plan_s* P, cudaStream_t st) {
  const pa_plan_desc& d = P->d;
  PA_CUDA(cudaGetDevice(&P->device));
  PA_CUDA(cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device));

  pa_status s;
  const size_t tab_n = (size_t)P->ndrows * P->nz_pad;
  if ((s = check_table_size(P)) != PA_OK) return s;
  if (P->full) {
    if ((s = dalloc(P, &P->ftab, P->full_entries)) != PA_OK) return s;
  } else if ((s = dalloc(P, &P->table, tab_n)) != PA_OK) {
    return s;
  }
  if (P->apod && (s = dalloc(P, &P->wtab, P->full ? P->full_entries : tab_n)) != PA_OK) return s;
  if ((s = dalloc(P, &P->items, (size_t)P->n_tiles * P->ngroups)) != PA_OK) return s;
  if ((s = dalloc(P, &P->slot_rg, (size_t)P->slots)) != PA_OK) return s;
  if ((s = dalloc(P, &P->lo, (size_t)P->n_tiles * P->nv)) != PA_OK) return s;
  if ((s = dalloc(P, &P->urange, (size_t)P->n_tiles * P->slots)) != PA_OK) return s;
  if ((s = dalloc(P, &P->vchunks, (size_t)P->n_tiles * P->ngroups)) != PA_OK) return s;
  if ((s = dalloc(P, &P->tw, (size_t)2 * P->M)) != PA_OK) return s;  // >= n_tw
  if ((s = dalloc(P, &P->mask, (size_t)3 * P->M)) != PA_OK) return s;
  // [0] error flags, [1] work counter, [2, 2 + 3 max_batch) image maxima,
  // [last] running count of timed-out waits
  P->scratch_ints = 3 + (size_t)P->d.max_batch * 3;
  if ((s = dalloc(P, &P->scratch[0], P->scratch_ints)) != PA_OK) return s;
  PA_CUDA(cudaMemsetAsync(P->scratch[0], 0, P->scratch_ints * sizeof(int), st));

  if ((size_t)36 * P->M > (size_t)200 * 1024)
    return fail(PA_EUNSUPPORTED, "nz = %d needs a %d-point envelope FFT; at most 4096 is supported",
                d.nz, P->M);

  // delay / apodisation table
  TableGeom tg;
  tg.ndrows = P->ndrows;
  tg.nzp = P->nz_pad;
  tg.zb = P->table_zb;
  tg.dmin = P->dmin;
  tg.ns = d.n_samples;
  tg.nearest = d.interp == PA_INTERP_NEAREST;
  tg.dx = (d.x1_m - d.x0_m) / d.nx;
  tg.x_const = d.x0_m + 0.5 * (d.n_elem - 1) * d.pitch_m;
  tg.z0 = d.z0_m;
  tg.dz = (d.z1_m - d.z0_m) / d.nz;
  tg.fs = d.fs_hz;
  tg.c = d.c_m_s;
  tg.t0 = d.t0_s;
  tg.fnum = d.f_number;
  tg.x0 = d.x0_m;
  tg.pitch = d.pitch_m;
  tg.n_elem = d.n_elem;
  tg.u0 = P->u0;
  tg.nv = P->nv;

  // per-tile windows and warp ranges
  TileGeom g;
  g.nxt = P->nxt;
  g.nzt = P->nzt;
  g.tile_x = P->tile_x;
  g.tile_z = P->tile_z;
  g.m = P->m;
  g.dmin = P->dmin;
  g.nzp = P->nz_pad;
  g.nv = P->nv;
  g.u0 = P->u0;
  g.ndrows = P->ndrows;
  g.zb = P->table_zb;
  g.full = P->full ? 1 : 0;
  FullGeom fg{P->nxt, P->n_tiles, P->tile_x, P->tile_z, P->m, P->slots, P->u1 - P->u0,
              P->lane_rows_log2, d.nx, d.nz, d.n_elem, P->u0, P->nv};
  int* wmax = P->scratch[0] + 2;  // borrowed before first use as image maxima
  if (P->full) {
    // windows first: the packed entries are written relative to them
    dim3 gw((P->nv + 127) / 128, P->n_tiles);
    k_windows_full<<<gw, 128, 0, st>>>(tg, g, P->lo_align, P->lo, wmax);
    PA_CUDA(cudaGetLastError());
    const size_t per_tile = P->full_entries / P->n_tiles;
    dim3 gt((unsigned)((per_tile + 255) / 256), P->n_tiles);
    k_table_full<<<gt, 256, 0, st>>>(tg, fg, P->lo, P->ftab, P->wtab);
    PA_CUDA(cudaGetLastError());
  } else {
    dim3 gt((P->nz_pad + 127) / 128, P->ndrows);
    k_table<<<gt, 128, 0, st>>>(tg, P->table, P->wtab);
    PA_CUDA(cudaGetLastError());
    dim3 gw((P->nv + 127) / 128, P->n_tiles);
    k_windows<<<gw, 128, 0, st>>>(g, P->lo_align, P->table, P->lo, wmax, P->scratch[0]);
    PA_CUDA(cudaGetLastError());
  }
  {
    dim3 grid((P->slots + 31) / 32, P->n_tiles);
    k_uranges<<<grid, 32, 0, st>>>(g, fg, P->slots, P->u1, kC, P->wtab, P->urange);
    PA_CUDA(cudaGetLastError());
  }
  unsigned long long* cnt = nullptr;
  if (P->apod) {
    PA_CUDA(cudaMalloc(&cnt, sizeof(unsigned long long)));
    PA_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
    if (P->full) {
      const size_t per_tile = P->full_entries / P->n_tiles;
      dim3 grid((unsigned)((per_tile + 255) / 256), P->n_tiles);
      k_count_active_full<<<grid, 256, 0, st>>>(fg, P->wtab, cnt);
    } else {
      dim3 grid((d.nz + 127) / 128, d.nx);
      k_count_active<<<grid, 128, 0, st>>>(g, d.nx, d.nz, d.n_elem, P->wtab, cnt);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      cudaFree(cnt);
      return fail(PA_ECUDA, "k_count_active: %s", cudaGetErrorString(e));
    }
  }

  int head[3] = {0, 0, 0};
  std::vector<int2> ur((size_t)P->n_tiles * P->slots);
  PA_CUDA(cudaMemcpyAsync(head, P->scratch[0], sizeof head, cudaMemcpyDeviceToHost, st));
  PA_CUDA(cudaMemcpyAsync(ur.data(), P->urange, ur.size() * sizeof(int2), cudaMemcpyDeviceToHost,
                          st));
  unsigned long long active = 0;
  if (cnt) PA_CUDA(cudaMemcpyAsync(&active, cnt, sizeof active, cudaMemcpyDeviceToHost, st));
  cudaError_t se = cudaStreamSynchronize(st);
  if (cnt) cudaFree(cnt);
  if (se != cudaSuccess) return fail(PA_ECUDA, "plan build: %s", cudaGetErrorString(se));
  if (head[0] != 0) return fail(PA_ECUDA, "plan build: table row outside range (flag %d)", head[0]);
  const int width = head[2];
  P->window = ((std::max(width, 1) + 3) / 4) * 4;

  PA_CUDA(cudaMemsetAsync(P->scratch[0], 0, P->scratch_ints * sizeof(int), st));

  // TMA box geometry of one staged channel
  P->wr = ((P->window + 1 + P->lo_align - 1) / P->lo_align) * P->lo_align;
  if (P->wr > 256) P->use_tma = false;  // TMA boxes span at most 256 elements
  if (P->use_tma && !tensor_map_encoder()) P->use_tma = false;
  P->rp = (int)((((size_t)P->wr * P->elt + 127) & ~size_t(127)) / P->elt);
  // Chunk length: every chunk costs a staging pass and two block barriers,
  // so the channel steps are cut into as few, evenly sized chunks as keep
  // the fused kernel's occupancy at what 32-step chunks give (measured at
  // N = 128: 5 chunks of 28 steps 0.696 ms, 4 of 36 0.692 ms, 3 of 44
  // 0.678 ms).  Limits: the slot buffer (at most 200 KiB), one issuing lane
  // per staged channel under TMA (ncs <= 32 warps), and the multiply-shift
  // division of the staging loops (exact while ncs * (W/4)^2 < 2^20).
  // PA_CHUNK_STEPS caps the chunk length (for measurements).
  {
    const int steps = P->u1 - P->u0;
    auto smem_for = [&](int c) {
      const int ncs = c + kC - 1;
      const size_t raw = P->use_tma ? (size_t)ncs * P->rp * P->elt : 0;
      return (size_t)kRawOff + ((raw + 127) & ~size_t(127)) + (size_t)ncs * P->window * 8;
    };
    auto fits = [&](int c) {
      const int ncs = c + kC - 1;
      const long long w4 = P->window / 4;
      return smem_for(c) <= 200 * 1024 && ncs <= 32 * P->warps &&
             (long long)ncs * w4 * w4 < (1ll << 20);
    };
    auto occupancy = [&](int c) {
      int b = 0;
      if (fused_blocks_per_sm(P, smem_for(c), &b) != cudaSuccess) b = 0;
      return b;
    };
    auto even = [&](int nch) { return ((steps + nch - 1) / nch + kC - 1) / kC * kC; };
    int cap = kNCMax;
    if (const char* e = getenv("PA_CHUNK_STEPS")) cap = std::max(kC, std::min(kNCMax, atoi(e)));
    int ref = std::min(32, cap);
    while (ref > kC && !fits(ref)) ref -= kC;
    const int occ_ref = occupancy(ref);
    int nc = ref;
    for (int nch = (steps + cap - 1) / cap; nch <= (steps + ref - 1) / ref; ++nch) {
      const int c = std::min(even(nch), cap);
      if (c > ref && fits(c) && occupancy(c) >= occ_ref) {
        nc = c;
        break;
      }
    }
    if (nc == ref) nc = std::min(ref, even((steps + ref - 1) / ref));
    P->nc = nc;
  }
  cudaGetLastError();

  // tile chunk ranges and executed pairs
  std::vector<int2> vk((size_t)P->n_tiles * P->ngroups);
  int64_t exec = 0;
  for (int t = 0; t < P->n_tiles; ++t) {
    for (int gr = 0; gr < P->ngroups; ++gr) {
      int ua = P->u1, ub = P->u0;
      for (int w = 0; w < P->warps; ++w) {
        const int2 r = ur[(size_t)t * P->slots + gr * P->warps + w];
        if (r.y > r.x) {
          ua = std::min(ua, r.x);
          ub = std::max(ub, r.y);
          exec += (int64_t)(r.y - r.x) * 32 * kC;
        }
      }
      int2 c = make_int2(0, 0);
      if (ub > ua) c = make_int2((ua - P->u0) / P->nc, (ub - P->u0 + P->nc - 1) / P->nc);
      vk[(size_t)t * P->ngroups + gr] = c;
    }
  }
  P->executed_pairs = exec;
  P->active_pairs = P->apod ? (int64_t)active : (int64_t)d.nx * d.nz * d.n_elem;
  PA_CUDA(cudaMemcpyAsync(P->vchunks, vk.data(), vk.size() * sizeof(int2), cudaMemcpyHostToDevice,
                          st));
  // work items (tile, residue group) deepest tiles first; the frame is the
  // fastest index of a work item, so frames of one tile run back to back
  std::vector<int4> it((size_t)P->n_tiles * P->ngroups);
  for (int t = 0; t < P->n_tiles; ++t) {
    const int tz = P->nzt - 1 - t / P->nxt, tx = t % P->nxt;
    for (int gr = 0; gr < P->ngroups; ++gr)
      it[(size_t)t * P->ngroups + gr] = make_int4(tz * P->nxt + tx, gr, tx, tz);
  }
  std::vector<int2> srg(P->slots);
  for (int sl = 0; sl < P->slots; ++sl) srg[sl] = make_int2(sl % P->m, sl / P->m);
  PA_CUDA(cudaMemcpyAsync(P->items, it.data(), it.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
  PA_CUDA(cudaMemcpyAsync(P->slot_rg, srg.data(), srg.size() * sizeof(int2), cudaMemcpyHostToDevice,
                          st));

  // shared memory and occupancy of the fused kernel
  const int ncs = P->nc + kC - 1;
  const size_t raw_bytes = P->use_tma ? (size_t)ncs * P->rp * P->elt : 0;
  P->pairs_off = kRawOff + (int)((raw_bytes + 127) & ~size_t(127));
  P->smem = (size_t)P->pairs_off + (size_t)ncs * P->window * sizeof(float2);
  const long long w4 = P->window / 4;
  if ((long long)ncs * w4 * w4 >= (1ll << 20))
    return fail(PA_EUNSUPPORTED, "RF window of %d samples per channel is too wide; use a finer "
                "depth grid", P->window);
  if (P->smem > 200 * 1024)
    return fail(PA_EUNSUPPORTED,
                "RF window of %d samples per channel needs %zu B of shared memory; use a finer "
                "depth grid",
                P->window, P->smem);
  // (resident blocks never ask for more TMEM than an SM has, so no block's
  // allocation waits on another block of the same launch)
  PA_CUDA(fused_blocks_per_sm(P, P->smem, &P->blocks_per_sm));
  if (P->blocks_per_sm < 1)
    return fail(PA_EUNSUPPORTED, "fused kernel does not fit an SM (%d threads, %zu B smem)",
                P->threads, P->smem);

  // post-filter tables (host FP64 -> FP32)
  // per-pass twiddle blocks of the Stockham FFT, in the order the passes run
  std::vector<float2> tw;
  {
    int ns = 1, rem = P->log2M;
    if (post_inplace_func(P->M) && post_first_radix(P->M) == 16) {
      ns = 16;  // first pass of radix 16 (sub-transform length 1: no twiddles)
      rem -= 4;
    }
    while (rem > 0) {
      const int lr = rem >= 3 ? 3 : rem;
      const int R = 1 << lr;
      if (ns > 1)
        for (int k = 0; k < ns; ++k)
          for (int r = 1; r < R; ++r) {
            const double ang = -2.0 * M_PI * (double)r * k / (double)(ns * R);
            tw.push_back(make_float2((float)std::cos(ang), (float)std::sin(ang)));
          }
      ns *= R;
      rem -= lr;
    }
    if (tw.empty()) tw.push_back(make_float2(1.f, 0.f));
  }
  P->n_tw = (int)tw.size();
  std::vector<float> mk((size_t)3 * P->M, 0.f);
  const bool even_of[3] = {false, true, (P->K % 2) == 0};
  for (int o = 0; o < 3; ++o) {
    if (P->out_id[o] < 0) continue;
    if (build_mask(d, even_of[o], P->M, mk.data() + (size_t)P->out_id[o] * P->M))
      P->warnings |= 1u << P->out_id[o];
  }
  PA_CUDA(cudaMemcpyAsync(P->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
  PA_CUDA(cudaMemcpyAsync(P->mask, mk.data(), mk.size() * sizeof(float), cudaMemcpyHostToDevice,
                          st));
  // post kernel: (3 post_wpb post_padded_len(M) + M) * 8 bytes, at most 200 KiB
  PA_CUDA(post_configure((size_t)200 * 1024));
  PA_CUDA(cudaStreamSynchronize(st));
  return PA_OK;
}

int stage_index(uint32_t stages, uint32_t stage) { return popcount3(stages & (stage - 1u)); }

// A timing event pair from the plan's free list (created when it is empty).
bool take_events(pa_plan_s* P, std::pair<cudaEvent_t, cudaEvent_t>* ev) {
  if (!P->ev_free.empty()) {
    *ev = P->ev_free.back();
    P->ev_free.pop_back();
    return true;
  }
  *ev = {nullptr, nullptr};
  if (cudaEventCreate(&ev->first) != cudaSuccess) {
    ev->first = nullptr;
    return false;
  }
  if (cudaEventCreate(&ev->second) != cudaSuccess) {
    cudaEventDestroy(ev->first);
    *ev = {nullptr, nullptr};
    return false;
  }
  return true;
}

// Event pair around one kernel launch when timing is enabled.
struct ProfScope {
  pa_plan_s* P;
  int kind;
  cudaStream_t st;
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  ProfScope(pa_plan_s* p, int k, cudaStream_t s) : P(p), kind(k), st(s) {
    if (!(P->prof >> kind & 1u)) return;
    if (!take_events(P, &ev)) return;
    cudaEventRecord(ev.first, st);
  }
  ~ProfScope() {
    if (!ev.first) return;
    cudaEventRecord(ev.second, st);
    P->ev_used.push_back({kind, ev});
  }
};

// Parameters of the launches of one chunk of nf <= max_batch frames.
struct ChunkLaunch {
  BfParams b;
  PostParams q;
  LogParams l;
  LaunchSpec sb, sq, sl;
  bool post = false, log = false;
  int* zero = nullptr;  // counter + image maxima, cleared before the kernels
  size_t zero_ints = 0;
};

bool encode_rf_map(pa_plan_s* P, const void* rf, int nf, CUtensorMap* map) {
  const pa_plan_desc& d = P->d;
  const cuuint64_t dims[3] = {(cuuint64_t)d.n_samples, (cuuint64_t)d.n_elem, (cuuint64_t)nf};
  const cuuint64_t strides[2] = {(cuuint64_t)d.n_samples * P->elt,
                                 (cuuint64_t)d.n_samples * d.n_elem * P->elt};
  const cuuint32_t box[3] = {(cuuint32_t)P->wr, 1, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapDataType dt =
      P->elt == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
  return tensor_map_encoder()(map, dt, 3, const_cast<void*>(rf), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

pa_status prepare_chunk(pa_plan_s* P, const void* rf, int nf, float* out, uint32_t stages,
                        int* scratch, ChunkLaunch* c) {
  const pa_plan_desc& d = P->d;
  const int n_st = popcount3(stages);
  const int planes = n_st * P->n_out;
  const uint32_t raw_stage =
      (stages & PA_STAGE_RAW) ? PA_STAGE_RAW : ((stages & PA_STAGE_ENV) ? PA_STAGE_ENV : PA_STAGE_LOG);
  const uint32_t env_stage = (stages & PA_STAGE_ENV) ? PA_STAGE_ENV : PA_STAGE_LOG;
  const int s_raw = stage_index(stages, raw_stage);
  const int s_env = stage_index(stages, env_stage);
  c->zero = scratch + 1;
  c->zero_ints = 1 + (size_t)nf * P->n_out;

  BfParams& b = c->b;
  memset(&b.tmap, 0, sizeof b.tmap);
  b.use_tma = P->use_tma ? 1 : 0;
  b.wr = P->wr;
  b.rp = P->rp;
  b.nc = P->nc;
  b.ncs = P->nc + kC - 1;
  b.tmem_cols = P->tmem_cols;
  b.chunk_bytes = b.ncs * P->wr * (int)P->elt;
  b.pairs_off = P->pairs_off;
  if (P->use_tma && !encode_rf_map(P, rf, nf, &b.tmap))
    return fail(PA_ECUDA, "cuTensorMapEncodeTiled rejected the RF layout");
  b.rf = rf;
  b.rf_dtype = (int)d.rf_dtype;
  b.vec_ok = (d.n_samples % 4) == 0;
  b.nearest = d.interp == PA_INTERP_NEAREST;
  b.lane_rows_log2 = P->lane_rows_log2;
  b.n_elem = d.n_elem;
  b.n_samples = d.n_samples;
  b.frame_elems = (long long)d.n_elem * d.n_samples;
  b.table = P->table;
  b.ftab = P->ftab;
  b.full = P->full ? 1 : 0;
  b.steps = P->u1 - P->u0;
  b.wtab = P->wtab;
  b.table_stride = P->table_zb ? 1 << P->table_zb : P->nz_pad;
  b.table_zb = P->table_zb;
  b.table_nzp = P->nz_pad;
  b.table_zshift = P->table_zb ? P->table_zb : 31;
  b.table_zmask = P->table_zb ? (1 << P->table_zb) - 1 : 0x7fffffff;
  b.table_zblock = P->table_zb ? (long long)P->ndrows << P->table_zb : 0;
  b.items = P->items;
  b.slot_rg = P->slot_rg;
  b.ndrows = P->ndrows;
  b.dmin = P->dmin;
  b.m = P->m;
  b.R = P->R;
  b.nxt = P->nxt;
  b.nzt = P->nzt;
  b.tile_x = P->tile_x;
  b.tile_z = P->tile_z;
  b.warps = P->warps;
  b.slots = P->slots;
  b.ngroups = P->ngroups;
  b.nv = P->nv;
  b.u0 = P->u0;
  b.window = P->window;
  b.w4_inv = (int)(((1u << 20) + (unsigned)(P->window / 4) - 1) / (unsigned)(P->window / 4));
  b.lo = P->lo;
  b.urange = P->urange;
  b.vchunks = P->vchunks;
  b.out = out;
  b.planes = planes;
  b.plane_das = P->out_id[0] >= 0 ? s_raw * P->n_out + P->out_id[0] : -1;
  b.plane_dmas = P->out_id[1] >= 0 ? s_raw * P->n_out + P->out_id[1] : -1;
  b.plane_ho = P->out_id[2] >= 0 ? s_raw * P->n_out + P->out_id[2] : -1;
  b.nx = d.nx;
  b.nz = d.nz;
  b.n_frames = nf;
  b.n_items = P->n_tiles * P->ngroups * nf;
  b.counter = scratch + 1;
  b.err = scratch;
  b.timeouts = scratch + P->scratch_ints - 1;
  b.expect_extra = P->expect_extra;
  c->sb.func = bf_func(P->K, P->apod, P->comp, P->full);
  c->sb.grid = dim3(std::max(1, std::min(b.n_items, P->blocks_per_sm * P->num_sms)));
  c->sb.block = dim3(P->threads);
  c->sb.smem = P->smem;

  c->post = (stages & (PA_STAGE_ENV | PA_STAGE_LOG)) != 0;
  c->log = (stages & PA_STAGE_LOG) != 0;
  PostParams& q = c->q;
  q.out = out;
  q.planes = planes;
  q.n_out = P->n_out;
  q.s_src = s_raw;
  q.s_dst = s_env;
  q.nx = d.nx;
  q.nz = d.nz;
  q.m = P->M;
  q.log2m = P->log2M;
  q.tw = P->tw;
  q.n_tw = P->n_tw;
  q.mask = P->mask;
  q.maxslot = scratch + 2;
  q.n_frames = nf;
  q.warps_per_block = P->post_wpb;
  post_spec(q, &c->sq);
  LogParams& l = c->l;
  l.out = out;
  l.planes = planes;
  l.n_out = P->n_out;
  l.s_src = s_env;
  l.s_dst = stage_index(stages, PA_STAGE_LOG);
  l.plane_elems = (long long)d.nx * d.nz;
  l.maxslot = scratch + 2;
  l.dyn_range_db = P->dyn_range;
  l.n_frames = nf;
  log_spec(l, P->num_sms, &c->sl);
  return PA_OK;
}

pa_status launch_direct(pa_plan_s* P, ChunkLaunch& c, cudaStream_t st) {
  k_zero_ints<<<1, 256, 0, st>>>(c.zero, (int)c.zero_ints);
  PA_CUDA(cudaGetLastError());
  {
    ProfScope ps(P, 0, st);
    void* args[] = {&c.b};
    PA_CUDA(cudaLaunchKernel(c.sb.func, c.sb.grid, c.sb.block, args, c.sb.smem, st));
  }
  if (c.post) {
    ProfScope ps(P, 1, st);
    void* args[] = {&c.q};
    PA_CUDA(cudaLaunchKernel(c.sq.func, c.sq.grid, c.sq.block, args, c.sq.smem, st));
  }
  if (c.log) {
    ProfScope ps(P, 2, st);
    void* args[] = {&c.l};
    PA_CUDA(cudaLaunchKernel(c.sl.func, c.sl.grid, c.sl.block, args, c.sl.smem, st));
  }
  return PA_OK;
}

cudaKernelNodeParams node_params(const LaunchSpec& s, void** args) {
  cudaKernelNodeParams k{};
  k.func = const_cast<void*>(s.func);
  k.gridDim = s.grid;
  k.blockDim = s.block;
  k.sharedMemBytes = (unsigned)s.smem;
  k.kernelParams = args;
  k.extra = nullptr;
  return k;
}


// One chunk as a CUDA graph: clear -> fused kernel [-> post [-> log]].  An
// executable graph is kept per (frames, stages, timing); later calls only
// rewrite the node parameters (buffer pointers, and the timing events) and
// launch it.  While timing is on, each kernel node sits between two
// event-record nodes, so the kernels are timed on the path that serves.
pa_status launch_graph(pa_plan_s* P, ChunkLaunch& c, int nf, uint32_t stages, cudaStream_t st) {
  const uint32_t prof = P->prof;
  pa_plan_s::GraphEntry* ge = nullptr;
  for (auto& g : P->graphs)
    if (g.nf == nf && g.stages == stages && g.prof == prof) ge = &g;
  void* ab[] = {&c.b};
  void* aq[] = {&c.q};
  void* al[] = {&c.l};
  int zn = (int)c.zero_ints;
  void* az[] = {&c.zero, &zn};
  LaunchSpec sz;
  sz.func = reinterpret_cast<const void*>(k_zero_ints);
  sz.grid = dim3(1);
  sz.block = dim3(256);
  const cudaKernelNodeParams kz = node_params(sz, az);
  const cudaKernelNodeParams kb = node_params(c.sb, ab);
  const cudaKernelNodeParams kq = node_params(c.sq, aq);
  const cudaKernelNodeParams kl = node_params(c.sl, al);
  const bool has[3] = {true, c.post, c.log};
  bool timed[3];
  for (int k = 0; k < 3; ++k) timed[k] = has[k] && (prof >> k & 1u);
  std::pair<cudaEvent_t, cudaEvent_t> ev[3] = {};
  if (prof) {
    for (int k = 0; k < 3; ++k) {
      if (timed[k] && !take_events(P, &ev[k])) {
        for (int j = 0; j < k; ++j)
          if (ev[j].first) P->ev_free.push_back(ev[j]);
        return fail(PA_ECUDA, "timing events: out of resources");
      }
    }
  }
  auto give_back = [&]() {
    for (int k = 0; k < 3; ++k)
      if (ev[k].first) P->ev_free.push_back(ev[k]);
  };
  if (!ge) {
    // bounded cache: drop the oldest graph once 32 shapes are held (callers
    // that vary the batch size every call would otherwise grow it forever)
    if (P->graphs.size() >= 32) {
      cudaGraphExecDestroy(P->graphs.front().exec);
      cudaGraphDestroy(P->graphs.front().graph);
      P->graphs.erase(P->graphs.begin());
    }
    pa_plan_s::GraphEntry g;
    g.nf = nf;
    g.stages = stages;
    g.prof = prof;
    cudaGraph_t graph;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) {
      give_back();
      return fail(PA_ECUDA, "graph build: %s", cudaGetErrorString(e));
    }
    const cudaKernelNodeParams* kp[3] = {&kb, &kq, &kl};
    cudaGraphNode_t* kn[3] = {&g.n_bf, &g.n_post, &g.n_log};
    e = cudaGraphAddKernelNode(&g.n_memset, graph, nullptr, 0, &kz);
    cudaGraphNode_t prev = g.n_memset;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
      if (!has[k]) continue;
      if (timed[k]) {
        e = cudaGraphAddEventRecordNode(&g.n_ev[k][0], graph, &prev, 1, ev[k].first);
        prev = g.n_ev[k][0];
      }
      if (e == cudaSuccess) e = cudaGraphAddKernelNode(kn[k], graph, &prev, 1, kp[k]);
      if (e != cudaSuccess) break;
      prev = *kn[k];
      if (timed[k]) {
        e = cudaGraphAddEventRecordNode(&g.n_ev[k][1], graph, &prev, 1, ev[k].second);
        prev = g.n_ev[k][1];
      }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(graph);
      give_back();
      return fail(PA_ECUDA, "graph build: %s", cudaGetErrorString(e));
    }
    g.graph = graph;
    ++P->graph_builds;
    P->graphs.push_back(g);
    ge = &P->graphs.back();
  } else {
    cudaError_t e = cudaGraphExecKernelNodeSetParams(ge->exec, ge->n_memset, &kz);
    if (e == cudaSuccess) e = cudaGraphExecKernelNodeSetParams(ge->exec, ge->n_bf, &kb);
    if (e == cudaSuccess && c.post)
      e = cudaGraphExecKernelNodeSetParams(ge->exec, ge->n_post, &kq);
    if (e == cudaSuccess && c.log) e = cudaGraphExecKernelNodeSetParams(ge->exec, ge->n_log, &kl);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
      if (!timed[k]) continue;
      e = cudaGraphExecEventRecordNodeSetEvent(ge->exec, ge->n_ev[k][0], ev[k].first);
      if (e == cudaSuccess)
        e = cudaGraphExecEventRecordNodeSetEvent(ge->exec, ge->n_ev[k][1], ev[k].second);
    }
    if (e != cudaSuccess) {
      give_back();
      return fail(PA_ECUDA, "graph update: %s", cudaGetErrorString(e));
    }
  }
  const cudaError_t e = cudaGraphLaunch(ge->exec, st);
  if (e != cudaSuccess) {
    give_back();
    return fail(PA_ECUDA, "graph launch: %s", cudaGetErrorString(e));
  }
  for (int k = 0; k < 3; ++k)
    if (ev[k].first) P->ev_used.push_back({k, ev[k]});
  return PA_OK;
}

pa_status run_chunk(pa_plan_s* P, const void* rf, int nf, float* out, uint32_t stages,
                    cudaStream_t st, int* scratch) {
  ChunkLaunch c;
  pa_status ps = prepare_chunk(P, rf, nf, out, stages, scratch, &c);
  if (ps != PA_OK) return ps;
  if (P->use_graph) return launch_graph(P, c, nf, stages, st);
  return launch_direct(P, c, st);
}

// Tapered schedule: short first and last chunks (the first upload and the
// last download overlap no compute), evenly sized middle chunks, none above
// cap frames.
std::vector<int32_t> taper_schedule(int n, int cap) {
  std::vector<int32_t> sched;
  const int edge = std::min(cap, std::max(1, n / 5));
  const int mid = n - 2 * edge;
  if (mid < 0) {  // one or two frames
    for (int f = 0; f < n; ++f) sched.push_back(1);
    return sched;
  }
  sched.push_back(edge);
  const int nm = mid == 0 ? 0 : std::max(2, (mid + cap - 1) / cap);
  for (int q = 0; q < nm; ++q) {
    const int c = (mid * (q + 1)) / nm - (mid * q) / nm;
    if (c > 0) sched.push_back(c);
  }
  sched.push_back(edge);
  return sched;
}

// Host-path link rate assumed by the candidate schedules: about 200 GB/s each
// way between pinned Grace memory and the GPU (measured 206 GB/s up, 192 GB/s
// down on GB300).
constexpr double kLinkBytesPerUs = 2.0e5;

// The tuning state of one (frames, stages) shape, created on first use with
// its candidates: the tapered schedule and the pipeline model's best
// schedules for kernel times of 0.6x to 2.8x the per-frame copy time,
// per-chunk launch costs of 8 and 40 us and wave shares of 0 and 1.  None of
// these is known in advance (measured on GB300: 38 us per chunk and no wave
// effect for 512 x 512 images at k = 3; about 50 us and a full wave effect
// at 1024 x 1024, k = 4); the tuning calls measure the outcome.
pa_plan_s::HostTune* host_tune(pa_plan_s* P, int nf, uint32_t stages) {
  for (auto& t : P->tunes)
    if (t.nf == nf && t.stages == stages) return &t;
  if (P->tunes.size() >= 32) P->tunes.erase(P->tunes.begin());  // bounded, oldest first
  pa_plan_s::HostTune t;
  t.nf = nf;
  t.stages = stages;
  const int cap = std::max(1, P->d.max_batch);
  auto add = [&t](std::vector<int32_t> c) {
    if (!c.empty() && std::find(t.cand.begin(), t.cand.end(), c) == t.cand.end())
      t.cand.push_back(std::move(c));
  };
  add(taper_schedule(nf, cap));
  if (nf > 2) {
    pa_pipe_model m{};
    m.items_per_frame = std::max(1, P->n_tiles * P->ngroups);
    m.resident = std::max(1, P->blocks_per_sm * P->num_sms);
    m.n_sets = kHostSets;
    const double rf_frame = (double)P->d.n_elem * P->d.n_samples * P->elt;
    const double out_frame = (double)popcount3(stages) * P->n_out * P->d.nx * P->d.nz * 4.0;
    m.upload_us = rf_frame / kLinkBytesPerUs;
    m.download_us = out_frame / kLinkBytesPerUs;
    const double copy_us = std::max(m.upload_us, m.download_us);
    for (double x : {0.6, 0.9, 1.3, 1.9, 2.8})
      for (double launch : {8.0, 40.0})
        for (double q : {0.0, 1.0}) {
          m.kernel_us = x * copy_us;
          m.launch_us = launch;
          m.wave_share = q;
          add(pipe_search(m, nf, cap));
        }
  }
  t.best_ms.assign(t.cand.size(), -1.0);
  for (int i = 0; i < (int)t.cand.size(); ++i) t.order.push_back(i);
  if (t.cand.size() == 1) t.chosen = 0;
  P->tunes.push_back(std::move(t));
  return &P->tunes.back();
}

// One tuning call of candidate `cur` took `ms`.  A cold call (it built a
// graph or grew the staging buffers) is not counted unless the candidate was
// cold three times in a row.
void host_tune_record(pa_plan_s::HostTune* t, int cur, double ms, bool cold) {
  if (cold && ++t->attempts < 3) return;
  t->attempts = 0;
  double& b = t->best_ms[cur];
  b = b < 0 ? ms : std::min(b, ms);
  if (++t->pos < t->order.size()) return;
  if (!t->second_round) {  // time the three fastest once more
    t->second_round = true;
    std::vector<int> idx(t->cand.size());
    for (int i = 0; i < (int)idx.size(); ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(),
                     [t](int a, int c) { return t->best_ms[a] < t->best_ms[c]; });
    for (int i = 0; i < std::min<int>(3, (int)idx.size()); ++i) t->order.push_back(idx[i]);
    return;
  }
  t->chosen = (int)(std::min_element(t->best_ms.begin(), t->best_ms.end()) - t->best_ms.begin());
}

void drop_host_graphs(pa_plan_s* P) {
  for (auto& g : P->host_graphs) {
    cudaGraphExecDestroy(g.exec);
    cudaGraphDestroy(g.graph);
  }
  P->host_graphs.clear();
}

bool is_pinned(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// The graph of one host-path call: per chunk c (buffer set b = c mod sets)
// an upload, the launch sequence (clear, fused kernel, post, log) and a
// download, with the ordering of the stream form: a launch sequence after
// its upload and after the previous chunk's launch sequence, a download
// after its launch sequence, an upload into set b after the download that
// last used set b.
pa_status build_host_graph(pa_plan_s* P, pa_plan_s::HostGraph& hg, const void* rf_host,
                           float* out_host, int chunk, int nsets) {
  const pa_plan_desc& d = P->d;
  const size_t rf_frame = (size_t)d.n_elem * d.n_samples * P->elt;
  const size_t out_frame = (size_t)popcount3(hg.stages) * P->n_out * d.nx * d.nz;
  cudaGraph_t graph;
  PA_CUDA(cudaGraphCreate(&graph, 0));
  cudaError_t e = cudaSuccess;
  cudaGraphNode_t prev_last = nullptr;
  int f0 = 0;
  for (size_t c = 0; c < hg.sched.size() && e == cudaSuccess; ++c) {
    const int nf = hg.sched[c];
    const int b = (int)(c % nsets);
    char* rf_d = (char*)P->h_rf + (size_t)b * chunk * rf_frame;
    float* out_d = P->h_out + (size_t)b * chunk * out_frame;
    const size_t up_off = (size_t)f0 * rf_frame, up_bytes = nf * rf_frame;  // bytes
    const size_t down_off = (size_t)f0 * out_frame;                          // floats
    const size_t down_bytes = nf * out_frame * sizeof(float);
    cudaGraphNode_t up = nullptr, down = nullptr;
    {
      cudaGraphNode_t dep = c >= (size_t)nsets ? hg.down[c - nsets] : nullptr;
      e = cudaGraphAddMemcpyNode1D(&up, graph, dep ? &dep : nullptr, dep ? 1 : 0, rf_d,
                                   (const char*)rf_host + up_off, up_bytes, cudaMemcpyHostToDevice);
    }
    ChunkLaunch cl;
    if (e == cudaSuccess) {
      const pa_status ps = prepare_chunk(P, rf_d, nf, out_d, hg.stages, P->scratch[b], &cl);
      if (ps != PA_OK) {
        cudaGraphDestroy(graph);
        return ps;
      }
    }
    cudaGraphNode_t last = nullptr;
    if (e == cudaSuccess) {
      void* ab[] = {&cl.b};
      void* aq[] = {&cl.q};
      void* al[] = {&cl.l};
      int zn = (int)cl.zero_ints;
      void* az[] = {&cl.zero, &zn};
      LaunchSpec sz;
      sz.func = reinterpret_cast<const void*>(k_zero_ints);
      sz.grid = dim3(1);
      sz.block = dim3(256);
      const cudaKernelNodeParams kz = node_params(sz, az);
      const cudaKernelNodeParams kb = node_params(cl.sb, ab);
      cudaGraphNode_t deps[2] = {up, prev_last};
      cudaGraphNode_t nz = nullptr, nb = nullptr;
      e = cudaGraphAddKernelNode(&nz, graph, deps, prev_last ? 2 : 1, &kz);
      if (e == cudaSuccess) e = cudaGraphAddKernelNode(&nb, graph, &nz, 1, &kb);
      last = nb;
      if (e == cudaSuccess && cl.post) {
        const cudaKernelNodeParams kq = node_params(cl.sq, aq);
        cudaGraphNode_t nq = nullptr;
        e = cudaGraphAddKernelNode(&nq, graph, &last, 1, &kq);
        last = nq;
      }
      if (e == cudaSuccess && cl.log) {
        const cudaKernelNodeParams kl = node_params(cl.sl, al);
        cudaGraphNode_t nl = nullptr;
        e = cudaGraphAddKernelNode(&nl, graph, &last, 1, &kl);
        last = nl;
      }
    }
    if (e == cudaSuccess)
      e = cudaGraphAddMemcpyNode1D(&down, graph, &last, 1, out_host + down_off, out_d, down_bytes,
                                   cudaMemcpyDeviceToHost);
    hg.up.push_back(up);
    hg.down.push_back(down);
    hg.up_dev.push_back(rf_d);
    hg.down_dev.push_back(out_d);
    hg.up_off.push_back(up_off);
    hg.down_off.push_back(down_off);
    hg.up_bytes.push_back(up_bytes);
    hg.down_bytes.push_back(down_bytes);
    prev_last = last;
    f0 += nf;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&hg.exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(PA_ECUDA, "host-path graph build: %s", cudaGetErrorString(e));
  }
  hg.graph = graph;
  hg.rf_host = rf_host;
  hg.out_host = out_host;
  ++P->graph_builds;
  return PA_OK;
}

// End of a host-path call: the tuning record, then the bounded waits that
// ran out during the call (the kernel stopped early).
pa_status host_call_done(pa_plan_s* P, pa_plan_s::HostTune* tune, bool tuning, int cur,
                         std::chrono::steady_clock::time_point t_start, bool cold) {
  if (tuning)
    host_tune_record(tune, cur,
                     std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() -
                                                               t_start).count(),
                     cold);
  if (P->use_tma) {
    long long total = 0;
    for (int b = 0; b < kHostSets; ++b) {
      if (!P->scratch[b]) continue;
      int n = 0;
      PA_CUDA(cudaMemcpy(&n, P->scratch[b] + P->scratch_ints - 1, sizeof n, cudaMemcpyDeviceToHost));
      total += n;
    }
    if (total > P->timeouts_seen) {
      const long long fresh = total - P->timeouts_seen;
      P->timeouts_seen = total;
      return fail(PA_ETIMEOUT, "%lld thread block(s) gave up waiting for their RF staging copies",
                  fresh);
    }
  }
  return PA_OK;
}

}  // namespace

// ------------------------------------------------------------ dispatchers
namespace pa {
void set_error_message(const char* msg) { g_err = msg ? msg : ""; }

int* plan_timeout_counter(pa_plan_s* P) {
  return P && P->scratch[0] ? P->scratch[0] + P->scratch_ints - 1 : nullptr;
}

size_t plan_device_bytes(const pa_plan_s* P) { return P ? P->device_bytes : 0; }

pa_status plan_bf_params(pa_plan_s* P, const void* rf, int nf, float* out, uint32_t stages,
                         BfParams* b, int* k, bool* lattice_fp32_plain) {
  ChunkLaunch c;
  const pa_status s = prepare_chunk(P, rf, nf, out, stages, P->scratch[0], &c);
  if (s != PA_OK) return s;
  *b = c.b;
  *k = P->K;
  *lattice_fp32_plain = !P->full && !P->apod && !P->comp && P->d.rf_dtype == PA_RF_F32 &&
                        P->d.interp == PA_INTERP_LINEAR;
  return PA_OK;
}

// A compensated plan's fused-kernel blocks hold tmem_cols TMEM columns each.
// Whatever blocks share an SM, their registers add up to at most the SM's
// register file, so if every block's columns are within its register share
// of the SM's 512 columns (cols * regs_sm <= 512 * regs_block), blocks of
// any mix of such kernels never ask for more TMEM than the SM has.  A plan
// outside that bound (blocks of 3 or fewer warps) is TMEM-dense: its blocks
// can fill an SM's TMEM while registers remain, so a block of another
// compensated kernel landing there would wait in tcgen05.alloc.
void plan_tmem(const pa_plan_s* P, int* cols, bool* dense) {
  *cols = P ? P->tmem_cols : 0;
  *dense = false;
  if (!P || !P->tmem_cols) return;
  cudaFuncAttributes a;
  int regs_sm = 65536;
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, P->device);
  if (cudaFuncGetAttributes(&a, bf_func(P->K, P->apod, P->comp, P->full)) != cudaSuccess) {
    cudaGetLastError();
    *dense = true;  // unknown: treat as dense (serialised with other compensated batches)
    return;
  }
  const size_t warps = (size_t)(P->threads + 31) / 32;
  const size_t regs_block = (size_t)((a.numRegs * 32 + 255) / 256) * 256 * warps;
  *dense = (size_t)P->tmem_cols * (size_t)regs_sm > (size_t)kTmemColsPerSm * regs_block;
}

cudaError_t bf_launch(int order, bool apod, bool comp, bool full, const BfParams& p, int grid,
                      int block, size_t smem, cudaStream_t s) {
  switch (order) {
    case 1: return bf_launch_k1(apod, comp, full, p, grid, block, smem, s);
    case 2: return bf_launch_k2(apod, comp, full, p, grid, block, smem, s);
    case 3: return bf_launch_k3(apod, comp, full, p, grid, block, smem, s);
    case 4: return bf_launch_k4(apod, comp, full, p, grid, block, smem, s);
    case 5: return bf_launch_k5(apod, comp, full, p, grid, block, smem, s);
    case 6: return bf_launch_k6(apod, comp, full, p, grid, block, smem, s);
    case 7: return bf_launch_k7(apod, comp, full, p, grid, block, smem, s);
    case 8: return bf_launch_k8(apod, comp, full, p, grid, block, smem, s);
  }
  return cudaErrorInvalidValue;
}
const void* bf_func(int order, bool apod, bool comp, bool full) {
  switch (order) {
    case 1: return bf_func_k1(apod, comp, full);
    case 2: return bf_func_k2(apod, comp, full);
    case 3: return bf_func_k3(apod, comp, full);
    case 4: return bf_func_k4(apod, comp, full);
    case 5: return bf_func_k5(apod, comp, full);
    case 6: return bf_func_k6(apod, comp, full);
    case 7: return bf_func_k7(apod, comp, full);
    case 8: return bf_func_k8(apod, comp, full);
  }
  return nullptr;
}
cudaError_t bf_occupancy(int order, bool apod, bool comp, bool full, int block, size_t smem,
                         int* n) {
  switch (order) {
    case 1: return bf_occupancy_k1(apod, comp, full, block, smem, n);
    case 2: return bf_occupancy_k2(apod, comp, full, block, smem, n);
    case 3: return bf_occupancy_k3(apod, comp, full, block, smem, n);
    case 4: return bf_occupancy_k4(apod, comp, full, block, smem, n);
    case 5: return bf_occupancy_k5(apod, comp, full, block, smem, n);
    case 6: return bf_occupancy_k6(apod, comp, full, block, smem, n);
    case 7: return bf_occupancy_k7(apod, comp, full, block, smem, n);
    case 8: return bf_occupancy_k8(apod, comp, full, block, smem, n);
  }
  return cudaErrorInvalidValue;
}
}  // namespace pa

// ------------------------------------------------------------------ C ABI
extern "C" {

pa_status pa_plan(const pa_plan_desc* desc, void* cuda_stream, pa_plan_t* out) {
  if (!out) return fail(PA_EINVAL, "null output handle");
  *out = nullptr;
  pa_status s = validate(desc);
  if (s != PA_OK) return s;
  pa_plan_s* P = new (std::nothrow) pa_plan_s();
  if (!P) return fail(PA_ENOMEM, "host allocation failed");
  P->d = *desc;
  configure(P);
  s = build_plan(P, (cudaStream_t)cuda_stream);
  if (s != PA_OK) {
    const std::string keep = g_err;
    free_plan(P);
    g_err = keep;
    return s;
  }
  *out = P;
  return PA_OK;
}

pa_status pa_plan_footprint(const pa_plan_desc* desc, int32_t n_frames, size_t* bytes) {
  if (!bytes) return fail(PA_EINVAL, "null bytes pointer");
  pa_status s = validate(desc);
  if (s != PA_OK) return s;
  if (n_frames < 0) return fail(PA_EINVAL, "n_frames < 0");
  pa_plan_s P;
  P.d = *desc;
  configure(&P);
  if ((s = check_table_size(&P)) != PA_OK) return s;
  size_t b = table_bytes(&P);
  b += (3 + (size_t)P.d.max_batch * 3) * sizeof(int);  // scratch, as pa_plan allocates it
  const size_t elt = desc->rf_dtype == PA_RF_F32 ? 4 : 2;
  b += (size_t)n_frames * desc->n_elem * desc->n_samples * elt;
  b += (size_t)n_frames * 3 * P.n_out * desc->nx * desc->nz * sizeof(float);
  *bytes = b;
  return PA_OK;
}

pa_status pa_plan_get_info(pa_plan_t P, pa_plan_info* info) {
  if (!P || !info) return fail(PA_EINVAL, "null argument");
  info->lattice_m = P->full ? 0 : P->m;
  info->tile_x = P->tile_x;
  info->tile_z = P->tile_z;
  info->window = P->window;
  info->n_tiles = P->n_tiles;
  info->threads = P->threads;
  info->blocks_per_sm = P->blocks_per_sm;
  info->fft_size = P->M;
  info->n_outputs = P->n_out;
  info->warnings = P->warnings;
  info->nominal_pairs = (int64_t)P->d.nx * P->d.nz * P->d.n_elem;
  info->active_pairs = P->active_pairs;
  info->executed_pairs = P->executed_pairs;
  info->device_bytes = P->device_bytes;
  info->tma_staging = P->use_tma ? 1 : 0;
  info->chunk_steps = P->nc;
  info->lane_rows = 1 << P->lane_rows_log2;
  info->tmem_columns = P->tmem_cols;
  info->delay_table = P->full ? PA_TABLE_FULL : PA_TABLE_LATTICE;
  info->table_bytes = delay_table_bytes(P);
  {
    int cols = 0;
    bool dense = false;
    plan_tmem(P, &cols, &dense);
    info->tmem_dense = dense ? 1 : 0;
  }
  info->device_error_flags = 0;
  {
    DeviceGuard g(P->device);
    for (int b = 0; b < kHostSets; ++b) {
      if (!P->scratch[b]) continue;
      int flag = 0;
      PA_CUDA(cudaDeviceSynchronize());
      PA_CUDA(cudaMemcpy(&flag, P->scratch[b], sizeof flag, cudaMemcpyDeviceToHost));
      info->device_error_flags |= (uint32_t)flag;
    }
  }
  return PA_OK;
}

pa_status pa_beamform(pa_plan_t P, const void* rf_dev, int32_t n_frames, float* out_dev,
                      uint32_t stages, void* cuda_stream) {
  if (!P) return fail(PA_EINVAL, "null plan");
  if (n_frames < 0) return fail(PA_EINVAL, "n_frames < 0");
  if ((stages & 7u) == 0 || (stages & ~7u)) return fail(PA_EINVAL, "stages mask 0x%x invalid", stages);
  if (n_frames == 0) return PA_OK;
  if (!rf_dev || !out_dev) return fail(PA_EINVAL, "null buffer");
  if (((uintptr_t)rf_dev & 15) || ((uintptr_t)out_dev & 15))
    return fail(PA_EINVAL, "buffers must be 16-byte aligned");
  DeviceGuard g(P->device);
  const pa_plan_desc& d = P->d;
  const size_t rf_frame = (size_t)d.n_elem * d.n_samples * P->elt;
  const size_t out_frame = (size_t)popcount3(stages) * P->n_out * d.nx * d.nz;
  for (int f0 = 0; f0 < n_frames; f0 += d.max_batch) {
    const int nf = std::min(d.max_batch, n_frames - f0);
    pa_status s = run_chunk(P, (const char*)rf_dev + (size_t)f0 * rf_frame, nf,
                            out_dev + (size_t)f0 * out_frame, stages, (cudaStream_t)cuda_stream,
                            P->scratch[0]);
    if (s != PA_OK) return s;
  }
  return PA_OK;
}

pa_status pa_beamform_host(pa_plan_t P, const void* rf_host, int32_t n_frames, float* out_host,
                           uint32_t stages, void* cuda_stream) {
  if (!P) return fail(PA_EINVAL, "null plan");
  if (n_frames < 0) return fail(PA_EINVAL, "n_frames < 0");
  if ((stages & 7u) == 0 || (stages & ~7u)) return fail(PA_EINVAL, "stages mask 0x%x invalid", stages);
  if (n_frames == 0) return PA_OK;
  if (!rf_host || !out_host) return fail(PA_EINVAL, "null buffer");
  DeviceGuard g(P->device);
  const pa_plan_desc& d = P->d;
  cudaStream_t user = (cudaStream_t)cuda_stream;
  pa_plan_s::HostTune* tune = host_tune(P, n_frames, stages);
  const bool tuning = tune->fixed.empty() && tune->chosen < 0;
  const int cur = tuning ? tune->order[tune->pos] : -1;
  const std::vector<int32_t> sched = tune->current();
  const long long builds0 = P->graph_builds;
  bool grew = false;
  const auto t_start = std::chrono::steady_clock::now();
  // buffers sized for the largest chunk of any candidate, so trying
  // candidates does not reallocate
  int chunk = 1, sets_needed = 1;
  for (const auto& c : tune->cand) {
    chunk = std::max(chunk, *std::max_element(c.begin(), c.end()));
    sets_needed = std::max(sets_needed, (int)c.size());
  }
  for (int32_t c : tune->fixed) chunk = std::max(chunk, c);
  sets_needed = std::min(kHostSets, std::max(sets_needed, (int)tune->fixed.size()));
  const int nsets = std::min<int>(kHostSets, (int)sched.size());
  const size_t rf_frame = (size_t)d.n_elem * d.n_samples * P->elt;
  const size_t out_frame = (size_t)popcount3(stages) * P->n_out * d.nx * d.nz;
  const size_t need_rf = (size_t)sets_needed * chunk * rf_frame;
  const size_t need_out = (size_t)sets_needed * chunk * out_frame * sizeof(float);
  if (need_rf > P->h_rf_bytes) {
    grew = true;
    drop_host_graphs(P);
    cudaFree(P->h_rf);
    P->device_bytes -= P->h_rf_bytes;
    P->h_rf_bytes = 0;
    PA_CUDA(cudaMalloc(&P->h_rf, need_rf));
    P->h_rf_bytes = need_rf;
    P->device_bytes += need_rf;
  }
  if (need_out > P->h_out_bytes) {
    grew = true;
    drop_host_graphs(P);
    cudaFree(P->h_out);
    P->device_bytes -= P->h_out_bytes;
    P->h_out_bytes = 0;
    PA_CUDA(cudaMalloc(&P->h_out, need_out));
    P->h_out_bytes = need_out;
    P->device_bytes += need_out;
  }
  if (!P->h_ev) PA_CUDA(cudaEventCreateWithFlags(&P->h_ev, cudaEventDisableTiming));
  for (int b = 0; b < nsets; ++b) {
    if (!P->hs[b]) PA_CUDA(cudaStreamCreateWithFlags(&P->hs[b], cudaStreamNonBlocking));
    if (!P->h_done[b]) PA_CUDA(cudaEventCreateWithFlags(&P->h_done[b], cudaEventDisableTiming));
    if (!P->scratch[b]) {
      pa_status s = dalloc(P, &P->scratch[b], P->scratch_ints);
      if (s != PA_OK) return s;
      PA_CUDA(cudaMemset(P->scratch[b], 0, P->scratch_ints * sizeof(int)));
    }
  }
  if (P->use_graph && P->prof == 0 && is_pinned(rf_host) && is_pinned(out_host)) {
    // pinned buffers: the whole call is one graph launch on the caller's stream
    pa_plan_s::HostGraph* hg = nullptr;
    for (auto& g : P->host_graphs)
      if (g.nf == n_frames && g.stages == stages && g.sched == sched) hg = &g;
    if (!hg) {
      if (P->host_graphs.size() >= 64) {  // bounded, oldest first
        cudaGraphExecDestroy(P->host_graphs.front().exec);
        cudaGraphDestroy(P->host_graphs.front().graph);
        P->host_graphs.erase(P->host_graphs.begin());
      }
      pa_plan_s::HostGraph g;
      g.nf = n_frames;
      g.stages = stages;
      g.sched = sched;
      pa_status s = build_host_graph(P, g, rf_host, out_host, chunk, nsets);
      if (s != PA_OK) return s;
      P->host_graphs.push_back(std::move(g));
      hg = &P->host_graphs.back();
    } else if (hg->rf_host != rf_host || hg->out_host != out_host) {
      for (size_t c = 0; c < hg->sched.size(); ++c) {
        PA_CUDA(cudaGraphExecMemcpyNodeSetParams1D(hg->exec, hg->up[c], hg->up_dev[c],
                                                   (const char*)rf_host + hg->up_off[c],
                                                   hg->up_bytes[c], cudaMemcpyHostToDevice));
        PA_CUDA(cudaGraphExecMemcpyNodeSetParams1D(hg->exec, hg->down[c],
                                                   out_host + hg->down_off[c], hg->down_dev[c],
                                                   hg->down_bytes[c], cudaMemcpyDeviceToHost));
      }
      hg->rf_host = rf_host;
      hg->out_host = out_host;
    }
    PA_CUDA(cudaGraphLaunch(hg->exec, user));
    PA_CUDA(cudaStreamSynchronize(user));
    return host_call_done(P, tune, tuning, cur, t_start, grew || P->graph_builds != builds0);
  }
  // the internal streams start after work already queued on the caller's stream
  PA_CUDA(cudaEventRecord(P->h_ev, user));
  for (int b = 0; b < nsets; ++b) PA_CUDA(cudaStreamWaitEvent(P->hs[b], P->h_ev, 0));
  int f0 = 0;
  for (size_t c = 0; c < sched.size(); ++c) {
    const int nf = sched[c];
    const int b = (int)(c % nsets);
    cudaStream_t st = P->hs[b];
    char* rf_d = (char*)P->h_rf + (size_t)b * chunk * rf_frame;
    float* out_d = P->h_out + (size_t)b * chunk * out_frame;
    PA_CUDA(cudaMemcpyAsync(rf_d, (const char*)rf_host + (size_t)f0 * rf_frame, nf * rf_frame,
                            cudaMemcpyHostToDevice, st));
    // the launch sequence waits for the previous chunk's (measured on GB300,
    // cfg2, 32 FP32 frames: 1.013 ms per call against 1.097 ms when
    // neighbouring chunks' kernels overlap)
    if (c > 0) PA_CUDA(cudaStreamWaitEvent(st, P->h_done[(c - 1) % nsets], 0));
    pa_status s = run_chunk(P, rf_d, nf, out_d, stages, st, P->scratch[b]);
    if (s != PA_OK) return s;
    PA_CUDA(cudaEventRecord(P->h_done[b], st));
    PA_CUDA(cudaMemcpyAsync(out_host + (size_t)f0 * out_frame, out_d,
                            nf * out_frame * sizeof(float), cudaMemcpyDeviceToHost, st));
    f0 += nf;
  }
  for (int b = 0; b < nsets; ++b) PA_CUDA(cudaStreamSynchronize(P->hs[b]));
  return host_call_done(P, tune, tuning, cur, t_start, grew || P->graph_builds != builds0);
}


pa_status pa_plan_set_host_schedule(pa_plan_t P, int32_t n_frames, uint32_t stages,
                                    const int32_t* chunks, int32_t n_chunks) {
  if (!P) return fail(PA_EINVAL, "null plan");
  if (n_frames < 1) return fail(PA_EINVAL, "n_frames < 1");
  if ((stages & 7u) == 0 || (stages & ~7u)) return fail(PA_EINVAL, "stages mask 0x%x invalid", stages);
  if (n_chunks < 0 || (n_chunks > 0 && !chunks)) return fail(PA_EINVAL, "invalid chunk list");
  std::vector<int32_t> v(chunks, chunks + n_chunks);
  long long sum = 0;
  for (int32_t c : v) {
    if (c < 1 || c > P->d.max_batch)
      return fail(PA_EINVAL, "chunk of %d frames outside 1..max_batch (%d)", c, P->d.max_batch);
    sum += c;
  }
  if (n_chunks > 0 && sum != n_frames)
    return fail(PA_EINVAL, "chunks sum to %lld frames, not %d", sum, n_frames);
  pa_plan_s::HostTune* t = host_tune(P, n_frames, stages);
  t->fixed = v;  // empty: back to tuning (or to the tuned choice)
  return PA_OK;
}

pa_status pa_plan_host_schedule(pa_plan_t P, int32_t n_frames, uint32_t stages, int32_t* chunks,
                                int32_t max_chunks, int32_t* n_chunks, int32_t* state) {
  if (!P || !chunks || !n_chunks || !state) return fail(PA_EINVAL, "null argument");
  if (n_frames < 1) return fail(PA_EINVAL, "n_frames < 1");
  if ((stages & 7u) == 0 || (stages & ~7u)) return fail(PA_EINVAL, "stages mask 0x%x invalid", stages);
  pa_plan_s::HostTune* t = host_tune(P, n_frames, stages);
  const std::vector<int32_t>& s = t->current();
  if ((int)s.size() > max_chunks)
    return fail(PA_EINVAL, "schedule has %d chunks, room for %d", (int)s.size(), max_chunks);
  std::copy(s.begin(), s.end(), chunks);
  *n_chunks = (int32_t)s.size();
  *state = !t->fixed.empty() ? 3 : (t->chosen >= 0 ? 2 : 1);
  return PA_OK;
}

pa_status pa_plan_use_graph(pa_plan_t P, int32_t enable) {
  if (!P) return fail(PA_EINVAL, "null plan");
  P->use_graph = enable != 0;
  return PA_OK;
}

pa_status pa_plan_profile(pa_plan_t P, int32_t enable) {
  if (!P) return fail(PA_EINVAL, "null plan");
  if (enable < 0 || enable > 2) return fail(PA_EINVAL, "profile mode %d not in 0..2", (int)enable);
  P->prof = enable == 0 ? 0u : enable == 1 ? 7u : 1u;
  return PA_OK;
}

pa_status pa_plan_profile_read(pa_plan_t P, double ms[3], int64_t launches[3]) {
  if (!P || !ms || !launches) return fail(PA_EINVAL, "null argument");
  DeviceGuard g(P->device);
  for (int k = 0; k < 3; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  for (auto& e : P->ev_used) {
    PA_CUDA(cudaEventSynchronize(e.second.second));
    float t = 0.f;
    PA_CUDA(cudaEventElapsedTime(&t, e.second.first, e.second.second));
    ms[e.first] += t;
    launches[e.first] += 1;
    P->ev_free.push_back(e.second);
  }
  P->ev_used.clear();
  return PA_OK;
}

pa_status pa_destroy(pa_plan_t P) {
  free_plan(P);
  return PA_OK;
}

const char* pa_status_str(pa_status s) {
  switch (s) {
    case PA_OK: return "ok";
    case PA_EINVAL: return "invalid argument";
    case PA_ENOMEM: return "out of device memory";
    case PA_ECUDA: return "CUDA error";
    case PA_ETIMEOUT: return "timed out";
    case PA_EUNSUPPORTED: return "unsupported";
    case PA_EBUSY: return "busy";
  }
  return "unknown status";
}

const char* pa_last_error(void) { return g_err.c_str(); }

int32_t pa_version(void) { return 105; }

}  // extern "C"
