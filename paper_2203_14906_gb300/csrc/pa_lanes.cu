// pa_lanes.cu -- the other thread mapping of the fused pass, for measurement:
// channels on lanes, power sums reduced across lanes by warp shuffles.
//
// The fused kernel (pa_bf_kernel.cuh) gives each thread 4 pixels of one depth
// row and walks the aperture in registers, so a pixel's sums never cross
// lanes and one lattice-table entry serves 4 pairs.  Here a pixel is shared
// by L lanes instead: lane g of a pixel's group takes channels g, g + L,
// g + 2L, ..., keeps its own DAS / DMAS / DMAS-3 sums, and the L partial sums
// are added by a shuffle butterfly (log2 L steps per sum) before one lane
// forms the outputs (Eq. 3 and Eq. 7 as in the fused kernel's epilogue).
// 32 / L pixels of one column (neighbouring depth rows) are in flight per
// warp.  Each block stages every channel window of its (tile, frame) in
// shared memory at once, as (r[n], r[n+1] - r[n]) slots like the fused
// kernel, so the two mappings differ in how pairs meet lanes, not in the
// data they read.  Only the plain FP32 lattice form at k = 3 is covered.
#include "pa_bf_kernel.cuh"

namespace pa {
namespace {

template <int L>
__global__ void __launch_bounds__(256) k_lanes(const __grid_constant__ BfParams p) {
  constexpr int NA = NAcc<3>::value;
  constexpr int P = 32 / L;  // pixels in flight per warp
  extern __shared__ __align__(16) unsigned char smem[];
  const int tile_id = blockIdx.x, frame = blockIdx.y;
  const int tx = tile_id % p.nxt, tz = tile_id / p.nxt;
  const int W = p.window;
  int* s_cb = reinterpret_cast<int*>(smem);
  const int slots_off = ((p.nv * 4 + 15) / 16) * 16;
  float2* slots = reinterpret_cast<float2*>(smem + slots_off);
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(slots);
  const int* lo_t = p.lo + (size_t)tile_id * p.nv;
  const float* rf = reinterpret_cast<const float*>(p.rf);
  for (int v = threadIdx.x; v < p.nv; v += blockDim.x)
    s_cb[v] = (int)sbase + v * W * 8 - __ldg(lo_t + v) * 8;
  for (int idx = threadIdx.x; idx < p.nv * W; idx += blockDim.x) {
    const int v = idx / W, q = idx - v * W;
    const int i = v + p.u0, n = __ldg(lo_t + v) + q;
    float r0 = 0.f, r1 = 0.f;
    if (i >= 0 && i < p.n_elem) {
      const float* row = rf + ((size_t)frame * p.n_elem + i) * p.n_samples;
      if (n >= 0 && n < p.n_samples) r0 = __ldg(row + n);
      if (n + 1 >= 0 && n + 1 < p.n_samples) r1 = __ldg(row + n + 1);
    }
    slots[(size_t)v * W + q] = make_float2(r0, r1 - r0);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int g = lane % L, pl = lane / L;
  const int npix = p.tile_x * p.tile_z;
  const size_t plane = (size_t)p.nx * p.nz;
  const size_t fbase = (size_t)frame * p.planes * plane;
  for (int base = warp * P; base < npix; base += nwarps * P) {
    const int pix = base + pl;
    const int zr = pix % p.tile_z, cl = pix / p.tile_z;
    const int j = tx * p.tile_x + cl, z = tz * p.tile_z + zr;
    float acc[NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) acc[q] = 0.f;
    for (int i = g; i < p.n_elem; i += L) {
      const int d = j - p.m * i;
      const int2 e = __ldg(p.table + table_index(d - p.dmin, z, p.ndrows, p.table_nzp, p.table_zb));
      const int addr = s_cb[i - p.u0] + e.x;
      float2 r;
      asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "r"(addr));
      pair_update<3>(acc, fmaf(__int_as_float(e.y), r.y, r.x));
    }
#pragma unroll
    for (int off = L / 2; off >= 1; off >>= 1)
#pragma unroll
      for (int q = 0; q < NA; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
    if (g == 0 && j < p.nx && z < p.nz) {
      float das, dmas, ho;
      combine<3>(acc, das, dmas, ho);
      const size_t px = fbase + (size_t)j * p.nz + z;
      if (p.plane_das >= 0) p.out[px + (size_t)p.plane_das * plane] = das;
      if (p.plane_dmas >= 0) p.out[px + (size_t)p.plane_dmas * plane] = dmas;
      if (p.plane_ho >= 0) p.out[px + (size_t)p.plane_ho * plane] = ho;
    }
  }
}

template <int L>
cudaError_t launch_lanes(const BfParams& b, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_lanes<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_lanes<L><<<dim3(b.nxt * b.nzt, b.n_frames), 256, smem, st>>>(b);
  return cudaGetLastError();
}

}  // namespace
}  // namespace pa

extern "C" pa_status pa_lanes_raw(pa_plan_t plan, const void* rf_dev, int32_t n_frames,
                                  float* out_dev, int32_t lanes_per_pixel, void* cuda_stream) {
  using namespace pa;
  if (!plan || !rf_dev || !out_dev || n_frames < 1) {
    set_error_message("pa_lanes_raw: null argument or no frames");
    return PA_EINVAL;
  }
  if (lanes_per_pixel != 4 && lanes_per_pixel != 8 && lanes_per_pixel != 32) {
    set_error_message("pa_lanes_raw: lanes_per_pixel must be 4, 8 or 32");
    return PA_EINVAL;
  }
  BfParams b;
  int k = 0;
  bool plain = false;
  const pa_status s = plan_bf_params(plan, rf_dev, n_frames, out_dev, PA_STAGE_RAW, &b, &k, &plain);
  if (s != PA_OK) return s;
  if (k != 3 || !plain) {
    set_error_message("pa_lanes_raw: only the plain FP32 lattice form at k = 3");
    return PA_EUNSUPPORTED;
  }
  const size_t smem = ((size_t)b.nv * 4 + 15) / 16 * 16 + (size_t)b.nv * b.window * 8;
  if (smem > 227 * 1024) {
    set_error_message("pa_lanes_raw: the tile's RF windows do not fit shared memory");
    return PA_EUNSUPPORTED;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaError_t e = lanes_per_pixel == 4    ? launch_lanes<4>(b, smem, st)
                  : lanes_per_pixel == 8 ? launch_lanes<8>(b, smem, st)
                                         : launch_lanes<32>(b, smem, st);
  if (e != cudaSuccess) {
    set_error_message(cudaGetErrorString(e));
    return PA_ECUDA;
  }
  return PA_OK;
}
