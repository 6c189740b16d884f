// pa_metrics.cu -- image-quality metrics of Section 3 (SNR Eq. 10, CR
// Eq. 11, gCNR Eq. 12, lateral FWHM) on device-resident images.
//
// Work is split into "slots": one slot is one region (target or background)
// of one ROI pair on one image.  Each slot's bounding box of pixels is cut
// into G chunks, one thread block per chunk, so large regions spread over the
// whole GPU while small ones cost a block each.  Reductions are written per
// block and summed in block order afterwards, so results do not depend on
// scheduling.  Region membership is decided once per image column: the
// pixels of a disc, rectangle or annulus in one column form one row interval
// (minus an inner interval for the annulus), found by binary search with the
// exact FP64 test, so the passes read member pixels only, warp by column with
// coalesced loads and no per-pixel floating-point test.  Launches:
//   ranges   per (region, column): the member row interval(s)
// and per chunk of ROI pairs:
//   pass 1   count, sum and the largest value (with its pixel) per block
//   reduce   per slot: count, mean, maximum
//   pass 2   per block: sum of squared deviations from the slot's mean; the
//            256-bin amplitude histogram (integer counts, exact) per slot
//   final    one thread per ROI pair: Eqs. 10-12, and the FWHM walk along
//            the row of the target maximum
// The bytes moved are 2 x 4 B per member pixel, plus the row walks.
#include <math.h>

#include <cmath>

#include <algorithm>
#include <vector>

#include "pa_internal.cuh"

namespace {

constexpr int kBins = 256;
constexpr int kThreads = 256;
constexpr int kMaxChunks = 64;
// ROI pairs per launch sequence: bounds the histogram scratch to
// 2 x 256 x 4 B x 16384 = 32 MiB.
constexpr long long kPairsPerLaunch = 16384;

struct MRegion {
  int shape;
  int j0, j1, l0, l1;  // bounding box of pixel indices, [j0, j1) x [l0, l1)
  long long col0;      // first entry of this region's columns in the range table
  double xc, zc, a, b;
};

// Member rows of one column: [lo, hi) without [hlo, hhi).
struct ColRange {
  int lo, hi, hlo, hhi;
};

struct MGeom {
  int nx, nz, n_roi, chunks;
  long long pair0;  // first (image, roi) pair of this launch sequence
  double x0, z0, dx, dz;
};

struct Part1 {
  long long cnt;
  double sum;
  unsigned long long key;  // ordered value bits << 32 | ~(pixel index)
};

struct SlotStat {
  long long cnt;
  double mean;
  unsigned long long key;
};

__device__ __forceinline__ unsigned int ordered_bits(float v) {
  const unsigned int u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_value(unsigned long long key) {
  const unsigned int o = (unsigned int)(key >> 32);
  const unsigned int u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
  return __uint_as_float(u);
}

// Pixel-centre membership, FP64 with explicit round-to-nearest operations
// (no fused multiply-add), so the decision matches a plain IEEE evaluation.
// Within one column every test below is monotone in |z - zc|, so each shape's
// member rows form one interval.
__device__ __forceinline__ double px(const MGeom& g, int j) {
  return __dadd_rn(g.x0, __dmul_rn((double)j + 0.5, g.dx));
}
__device__ __forceinline__ double pz(const MGeom& g, int l) {
  return __dadd_rn(g.z0, __dmul_rn((double)l + 0.5, g.dz));
}
// rect: |ez| <= b (the |ex| <= a part is per column); disc of radius rad:
// ex^2 + ez^2 <= rad^2
__device__ __forceinline__ bool row_in(int shape, double ex2, double zc, double rad, const MGeom& g,
                                       int l) {
  const double ez = __dsub_rn(pz(g, l), zc);
  if (shape == PA_REGION_RECT) return fabs(ez) <= rad;
  return __dadd_rn(ex2, __dmul_rn(ez, ez)) <= __dmul_rn(rad, rad);
}

// Interval of rows l in [0, nz) with row_in true, as [lo, hi) (empty: lo == hi).
__device__ int2 row_interval(int shape, double ex2, double zc, double rad, const MGeom& g) {
  // the test is weakest at the row nearest the centre (or at an end of the
  // column when the centre lies beyond it); rounding may move that by one
  double lc = (zc - g.z0) / g.dz - 0.5;
  lc = fmin(fmax(lc, 0.0), (double)(g.nz - 1));
  int lm = (int)rint(lc), seed = -1;
  for (int d = 0; d <= 2 && seed < 0; ++d) {
    if (lm - d >= 0 && row_in(shape, ex2, zc, rad, g, lm - d)) seed = lm - d;
    else if (lm + d < g.nz && row_in(shape, ex2, zc, rad, g, lm + d)) seed = lm + d;
  }
  if (seed < 0) return make_int2(0, 0);
  int lo = 0, hi = seed;  // first member row in [0, seed]
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (row_in(shape, ex2, zc, rad, g, mid)) hi = mid;
    else lo = mid + 1;
  }
  const int first = lo;
  lo = seed;
  hi = g.nz - 1;  // last member row in [seed, nz - 1]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (row_in(shape, ex2, zc, rad, g, mid)) lo = mid;
    else hi = mid - 1;
  }
  return make_int2(first, lo + 1);
}

__global__ void k_m_ranges(MGeom g, const MRegion* regs, int n_regions, ColRange* ranges) {
  const int r = blockIdx.y;
  if (r >= n_regions) return;
  const MRegion R = regs[r];
  const int j = R.j0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= R.j1) return;
  const double ex = __dsub_rn(px(g, j), R.xc);
  const double ex2 = __dmul_rn(ex, ex);
  ColRange c{0, 0, 0, 0};
  if (R.shape == PA_REGION_RECT) {
    if (fabs(ex) <= R.a) {
      const int2 v = row_interval(PA_REGION_RECT, 0.0, R.zc, R.b, g);
      c.lo = v.x;
      c.hi = v.y;
    }
  } else if (R.shape == PA_REGION_DISC) {
    const int2 v = row_interval(PA_REGION_DISC, ex2, R.zc, R.a, g);
    c.lo = v.x;
    c.hi = v.y;
  } else {  // annulus: disc(b) without disc(a)
    const int2 v = row_interval(PA_REGION_DISC, ex2, R.zc, R.b, g);
    const int2 h = row_interval(PA_REGION_DISC, ex2, R.zc, R.a, g);
    c.lo = v.x;
    c.hi = v.y;
    c.hlo = h.x;
    c.hhi = h.y;
  }
  ranges[R.col0 + (j - R.j0)] = c;
}

struct SlotRef {
  long long pair;  // global (image, roi) pair index
  int side;        // 0 target, 1 background
  const MRegion* reg;
  const float* img;
};

__device__ __forceinline__ SlotRef slot_ref(const MGeom& g, const MRegion* regs,
                                            const float* images, long long slot) {
  SlotRef s;
  s.pair = g.pair0 + slot / 2;
  s.side = (int)(slot & 1);
  const long long img = s.pair / g.n_roi;
  const int roi = (int)(s.pair % g.n_roi);
  s.reg = regs + 2 * roi + s.side;
  s.img = images + (size_t)img * g.nx * g.nz;
  return s;
}

template <typename T, typename Op>
__device__ __forceinline__ T block_reduce(T v, T* sh, Op op) {
  for (int o = 16; o >= 1; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  T r = sh[0];
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i) r = op(r, sh[i]);  // fixed order
  return r;
}

// Calls f(j, l, q) for every member pixel of the block's share of the
// slot's region: warp w of chunk c takes columns c * warps + w, stepping by
// chunks * warps; lanes walk the column's row interval(s).
template <typename F>
__device__ __forceinline__ void for_members(const MGeom& g, const MRegion& r, const ColRange* ranges,
                                            int chunk, F&& f) {
  const int warps = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int width = r.j1 - r.j0;
  for (int c = chunk * warps + w; c < width; c += g.chunks * warps) {
    const ColRange cr = ranges[r.col0 + c];
    const int j = r.j0 + c;
    const long long qj = (long long)j * g.nz;
    const int e1 = cr.hhi > cr.hlo ? min(cr.hi, cr.hlo) : cr.hi;  // rows before the hole
    for (int l = cr.lo + lane; l < e1; l += 32) f(j, l, qj + l);
    if (cr.hhi > cr.hlo)
      for (int l = max(cr.lo, cr.hhi) + lane; l < cr.hi; l += 32) f(j, l, qj + l);
  }
}

__global__ void __launch_bounds__(kThreads) k_m_pass1(MGeom g, const MRegion* regs,
                                                      const ColRange* ranges, const float* images,
                                                      Part1* part) {
  __shared__ long long sh_c[kThreads / 32];
  __shared__ double sh_s[kThreads / 32];
  __shared__ unsigned long long sh_k[kThreads / 32];
  const long long slot = blockIdx.x / g.chunks;
  const int chunk = blockIdx.x % g.chunks;
  const SlotRef s = slot_ref(g, regs, images, slot);
  const MRegion r = *s.reg;
  long long cnt = 0;
  double sum = 0.0;
  unsigned long long key = 0;
  for_members(g, r, ranges, chunk, [&](int, int, long long q) {
    const float v = __ldg(s.img + q);
    ++cnt;
    sum += (double)v;
    const unsigned long long k = ((unsigned long long)ordered_bits(v) << 32) |
                                 (unsigned long long)(0xffffffffu - (unsigned int)q);
    key = k > key ? k : key;
  });
  cnt = block_reduce(cnt, sh_c, [](long long x, long long y) { return x + y; });
  sum = block_reduce(sum, sh_s, [](double x, double y) { return x + y; });
  key = block_reduce(key, sh_k,
                     [](unsigned long long x, unsigned long long y) { return x > y ? x : y; });
  if (threadIdx.x == 0) part[blockIdx.x] = Part1{cnt, sum, key};
}

__global__ void k_m_reduce(long long n_slots, int chunks, const Part1* part, SlotStat* st) {
  const long long slot = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= n_slots) return;
  long long cnt = 0;
  double sum = 0.0;
  unsigned long long key = 0;
  for (int c = 0; c < chunks; ++c) {
    const Part1 p = part[slot * chunks + c];
    cnt += p.cnt;
    sum += p.sum;
    key = p.key > key ? p.key : key;
  }
  st[slot] = SlotStat{cnt, cnt > 0 ? sum / (double)cnt : 0.0, key};
}

// Normalised-amplitude bin of Eq. 12: floor(v * 256 / vmax), FP32 with an
// IEEE-rounded division, clamped to [0, 255].
__device__ __forceinline__ int amp_bin(float v, float vmax) {
  if (!(vmax > 0.f) || !(v > 0.f)) return 0;
  const float x = __fdiv_rn(v * 256.0f, vmax);
  return x >= 255.0f ? 255 : (int)x;
}

__global__ void __launch_bounds__(kThreads) k_m_pass2(MGeom g, const MRegion* regs,
                                                      const ColRange* ranges, const float* images,
                                                      const SlotStat* st, double* part2, int* hist) {
  __shared__ int h[kBins];
  __shared__ double sh_s[kThreads / 32];
  const long long slot = blockIdx.x / g.chunks;
  const int chunk = blockIdx.x % g.chunks;
  const SlotRef s = slot_ref(g, regs, images, slot);
  const MRegion r = *s.reg;
  const SlotStat mine = st[slot];
  const SlotStat a = st[slot & ~1ll], b = st[slot | 1ll];
  float vmax = -INFINITY;
  if (a.cnt > 0) vmax = key_value(a.key);
  if (b.cnt > 0) vmax = fmaxf(vmax, key_value(b.key));
  for (int i = threadIdx.x; i < kBins; i += blockDim.x) h[i] = 0;
  __syncthreads();
  double ss = 0.0;
  for_members(g, r, ranges, chunk, [&](int, int, long long q) {
    const float v = __ldg(s.img + q);
    const double e = (double)v - mine.mean;
    ss += e * e;
    atomicAdd(&h[amp_bin(v, vmax)], 1);
  });
  ss = block_reduce(ss, sh_s, [](double x, double y) { return x + y; });
  if (threadIdx.x == 0) part2[blockIdx.x] = ss;
  __syncthreads();
  int* dst = hist + (size_t)slot * kBins;
  for (int i = threadIdx.x; i < kBins; i += blockDim.x)
    if (h[i]) atomicAdd(dst + i, h[i]);
}

__global__ void k_m_final(MGeom g, long long n_pairs, const float* images, const SlotStat* st,
                          const double* part2, const int* hist, pa_metrics* out) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pairs) return;
  const long long pair = g.pair0 + p;
  const float* img = images + (size_t)(pair / g.n_roi) * g.nx * g.nz;
  const SlotStat si = st[2 * p], so = st[2 * p + 1];
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  pa_metrics m;
  m.n_in = si.cnt;
  m.n_out = so.cnt;
  m.mu_in = si.cnt > 0 ? si.mean : nan;
  m.mu_out = so.cnt > 0 ? so.mean : nan;
  double ss = 0.0;
  for (int c = 0; c < g.chunks; ++c) ss += part2[(2 * p + 1) * g.chunks + c];
  m.sigma_out = so.cnt > 0 ? sqrt(ss / (double)so.cnt) : nan;
  m.snr_db = 20.0 * log10(m.mu_in / m.sigma_out);
  m.cr_db = 20.0 * log10(m.mu_in / m.mu_out);
  if (si.cnt > 0 && so.cnt > 0) {
    // sum_b min(c_in / n_in, c_out / n_out) = sum_b min(c_in n_out, c_out n_in) / (n_in n_out)
    const int* hi = hist + (size_t)(2 * p) * kBins;
    const int* ho = hi + kBins;
    long long ov = 0;
    for (int b = 0; b < kBins; ++b) {
      const long long u = (long long)hi[b] * so.cnt, v = (long long)ho[b] * si.cnt;
      ov += u < v ? u : v;
    }
    m.gcnr = 1.0 - (double)ov / ((double)si.cnt * (double)so.cnt);
  } else {
    m.gcnr = nan;
  }
  m.peak = nan;
  m.fwhm_m = nan;
  m.peak_j = m.peak_l = -1;
  if (si.cnt > 0) {
    const unsigned int q = 0xffffffffu - (unsigned int)(si.key & 0xffffffffull);
    const int j0 = (int)(q / (unsigned int)g.nz), l0 = (int)(q % (unsigned int)g.nz);
    const float pk = key_value(si.key);
    m.peak = (double)pk;
    m.peak_j = j0;
    m.peak_l = l0;
    const double half = 0.5 * (double)pk;
    const float* row = img + l0;  // element j of the row at row[j * nz]
    auto at = [&](int j) { return (double)row[(size_t)j * g.nz]; };
    auto xp = [&](int j) { return __dadd_rn(g.x0, __dmul_rn((double)j + 0.5, g.dx)); };
    int jl = j0;
    while (jl > 0 && at(jl - 1) >= half) --jl;
    int jr = j0;
    while (jr < g.nx - 1 && at(jr + 1) >= half) ++jr;
    if (jl > 0 && jr < g.nx - 1) {
      const double pl = at(jl - 1), ql = at(jl);
      const double pr = at(jr + 1), qr = at(jr);
      const double xl = __dadd_rn(xp(jl - 1), __dmul_rn(__ddiv_rn(__dsub_rn(half, pl), __dsub_rn(ql, pl)), g.dx));
      const double xr = __dsub_rn(xp(jr + 1), __dmul_rn(__ddiv_rn(__dsub_rn(half, pr), __dsub_rn(qr, pr)), g.dx));
      m.fwhm_m = __dsub_rn(xr, xl);
    }
  }
  out[pair] = m;
}

pa_status mfail(pa_status s, const char* msg) {
  pa::set_error_message(msg);
  return s;
}

bool finite_d(double v) { return std::isfinite(v); }

// Conservative index range of pixel centres in [c - h, c + h] on a grid of n
// cells starting at o with step d; the membership test decides exactly.
void index_range(double c, double h, double o, double d, int n, int* lo, int* hi) {
  const double a = (c - h - o) / d - 0.5, b = (c + h - o) / d - 0.5;
  double l = std::floor(a) - 1.0, u = std::ceil(b) + 2.0;
  l = std::max(0.0, std::min((double)n, l));
  u = std::max(0.0, std::min((double)n, u));
  *lo = (int)l;
  *hi = std::max(*lo, (int)u);
}

}  // namespace

extern "C" pa_status pa_image_metrics(const pa_grid* grid, const float* images_dev,
                                      int32_t n_images, const pa_roi* rois, int32_t n_roi,
                                      pa_metrics* out_dev, void* cuda_stream) {
  if (!grid || !rois) return mfail(PA_EINVAL, "pa_image_metrics: null grid or rois");
  if (n_images < 0) return mfail(PA_EINVAL, "pa_image_metrics: n_images < 0");
  if (n_roi < 1 || n_roi > PA_METRICS_MAX_ROIS)
    return mfail(PA_EINVAL, "pa_image_metrics: n_roi outside 1..PA_METRICS_MAX_ROIS");
  const pa_grid G = *grid;
  if (G.nx < 1 || G.nz < 1 || !finite_d(G.x0_m) || !finite_d(G.x1_m) || !finite_d(G.z0_m) ||
      !finite_d(G.z1_m) || !(G.x1_m > G.x0_m) || !(G.z1_m > G.z0_m))
    return mfail(PA_EINVAL, "pa_image_metrics: bad grid");
  if ((long long)G.nx * G.nz > 0xffffffffll)
    return mfail(PA_EINVAL, "pa_image_metrics: image larger than 2^32 pixels");
  if (n_images == 0) return PA_OK;
  if (!images_dev || !out_dev) return mfail(PA_EINVAL, "pa_image_metrics: null buffer");

  MGeom g{};
  g.nx = G.nx;
  g.nz = G.nz;
  g.n_roi = n_roi;
  g.x0 = G.x0_m;
  g.z0 = G.z0_m;
  g.dx = (G.x1_m - G.x0_m) / G.nx;
  g.dz = (G.z1_m - G.z0_m) / G.nz;
  std::vector<MRegion> regs(2 * (size_t)n_roi);
  long long max_area = 0, n_cols = 0;
  int max_width = 0;
  for (int r = 0; r < n_roi; ++r) {
    for (int side = 0; side < 2; ++side) {
      const pa_region& in = side ? rois[r].background : rois[r].target;
      MRegion& o = regs[2 * r + side];
      if (in.shape != PA_REGION_RECT && in.shape != PA_REGION_DISC && in.shape != PA_REGION_ANNULUS)
        return mfail(PA_EINVAL, "pa_image_metrics: unknown region shape");
      if (!finite_d(in.xc_m) || !finite_d(in.zc_m) || !finite_d(in.a_m) || !finite_d(in.b_m) ||
          in.a_m < 0 || in.b_m < 0)
        return mfail(PA_EINVAL, "pa_image_metrics: region extents must be finite and >= 0");
      o.shape = in.shape;
      o.xc = in.xc_m;
      o.zc = in.zc_m;
      o.a = in.a_m;
      o.b = in.b_m;
      const double hx = in.shape == PA_REGION_ANNULUS ? in.b_m : in.a_m;
      const double hz = in.shape == PA_REGION_DISC ? in.a_m : in.b_m;
      index_range(in.xc_m, hx, g.x0, g.dx, g.nx, &o.j0, &o.j1);
      index_range(in.zc_m, hz, g.z0, g.dz, g.nz, &o.l0, &o.l1);
      o.col0 = n_cols;
      n_cols += o.j1 - o.j0;
      max_width = std::max(max_width, o.j1 - o.j0);
      max_area = std::max(max_area, (long long)(o.j1 - o.j0) * (o.l1 - o.l0));
    }
  }
  // blocks per region: about 8192 bounding-box pixels each, at least one
  // column per warp
  const long long by_area = (max_area + 8191) / 8192, by_cols = (max_width + 7) / 8;
  g.chunks = (int)std::max<long long>(1, std::min<long long>({(long long)kMaxChunks, by_area, by_cols}));

  cudaStream_t st = (cudaStream_t)cuda_stream;
  const long long n_pairs = (long long)n_images * n_roi;
  const long long pairs_per = std::min(n_pairs, kPairsPerLaunch);
  const long long slots_per = 2 * pairs_per;
  const size_t b_regs = regs.size() * sizeof(MRegion);
  const size_t b_cols = (size_t)std::max<long long>(n_cols, 1) * sizeof(ColRange);
  const size_t b_p1 = (size_t)slots_per * g.chunks * sizeof(Part1);
  const size_t b_st = (size_t)slots_per * sizeof(SlotStat);
  const size_t b_p2 = (size_t)slots_per * g.chunks * sizeof(double);
  const size_t b_h = (size_t)slots_per * kBins * sizeof(int);
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t total = up(b_regs) + up(b_cols) + up(b_p1) + up(b_st) + up(b_p2) + up(b_h);
  char* base = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&base, total, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return mfail(e == cudaErrorMemoryAllocation ? PA_ENOMEM : PA_ECUDA, cudaGetErrorString(e));
  }
  MRegion* d_regs = (MRegion*)base;
  ColRange* d_cols = (ColRange*)(base + up(b_regs));
  Part1* d_p1 = (Part1*)((char*)d_cols + up(b_cols));
  SlotStat* d_st = (SlotStat*)((char*)d_p1 + up(b_p1));
  double* d_p2 = (double*)((char*)d_st + up(b_st));
  int* d_h = (int*)((char*)d_p2 + up(b_p2));
  e = cudaMemcpyAsync(d_regs, regs.data(), b_regs, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && max_width > 0) {
    const dim3 grid_r((unsigned)((max_width + 127) / 128), (unsigned)regs.size());
    k_m_ranges<<<grid_r, 128, 0, st>>>(g, d_regs, (int)regs.size(), d_cols);
    e = cudaGetLastError();
  }
  for (long long p0 = 0; e == cudaSuccess && p0 < n_pairs; p0 += pairs_per) {
    const long long np = std::min(pairs_per, n_pairs - p0);
    const long long ns = 2 * np;
    g.pair0 = p0;
    const long long blocks = ns * g.chunks;
    e = cudaMemsetAsync(d_h, 0, (size_t)ns * kBins * sizeof(int), st);
    if (e != cudaSuccess) break;
    k_m_pass1<<<(unsigned)blocks, kThreads, 0, st>>>(g, d_regs, d_cols, images_dev, d_p1);
    k_m_reduce<<<(unsigned)((ns + 127) / 128), 128, 0, st>>>(ns, g.chunks, d_p1, d_st);
    k_m_pass2<<<(unsigned)blocks, kThreads, 0, st>>>(g, d_regs, d_cols, images_dev, d_st, d_p2,
                                                     d_h);
    k_m_final<<<(unsigned)((np + 127) / 128), 128, 0, st>>>(g, np, images_dev, d_st, d_p2, d_h,
                                                           out_dev);
    e = cudaGetLastError();
  }
  const cudaError_t ef = cudaFreeAsync(base, st);
  if (e == cudaSuccess) e = ef;
  if (e != cudaSuccess) return mfail(PA_ECUDA, cudaGetErrorString(e));
  return PA_OK;
}
