// pa_post.cu -- band-pass + Hilbert envelope + log compression (Section 3:
// the beamformed images are band-pass filtered, envelope-detected through
// the Hilbert transform and log-compressed before display).
//
// k_post: one warp per depth column.  The column is zero-padded to
// M = 2^ceil(log2 nz) in shared memory, transformed by a radix-2
// decimation-in-time FFT (bit-reversed load, natural-order spectrum),
// multiplied by the plan's real mask H = band-pass x analytic weights
// (1 at DC and M/2, 2 on positive bins, 0 on negative bins), and
// transformed back by a decimation-in-frequency inverse FFT (natural
// input, bit-reversed output).  The envelope |y[z]| / M for z < nz is
// written and the column maximum is merged into the image maximum with an
// atomic max on the float bits (the envelope is non-negative).  The column
// is read completely before it is written, so source and destination may
// be the same plane.
//
// k_log: 20 log10(env / image max), clipped to [-DR, 0]; elementwise.
#include "pa_internal.cuh"

namespace pa {

__device__ __forceinline__ int bit_reverse(int n, int log2m) {
  return log2m == 0 ? 0 : (int)(__brev((unsigned)n) >> (32 - log2m));
}

__global__ void __launch_bounds__(256) k_post(const PostParams p) {
  extern __shared__ __align__(16) float2 sbuf[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * p.warps_per_block + warp;
  const int o = blockIdx.y, f = blockIdx.z;
  if (j >= p.nx) return;  // warps are independent: no block barrier below
  const int M = p.m, L = p.log2m, half = M >> 1;
  float2* buf = sbuf + (size_t)warp * M;
  const size_t plane = (size_t)p.nx * p.nz;
  const float* src = p.out + ((size_t)f * p.planes + (size_t)p.s_src * p.n_out + o) * plane +
                     (size_t)j * p.nz;
  float* dst = p.out + ((size_t)f * p.planes + (size_t)p.s_dst * p.n_out + o) * plane +
               (size_t)j * p.nz;

  for (int n = lane; n < M; n += 32) {
    const float x = (n < p.nz) ? src[n] : 0.f;
    buf[bit_reverse(n, L)] = make_float2(x, 0.f);
  }
  __syncwarp();

  // forward DIT, butterfly span h = 1, 2, ..., M/2; twiddle e^{-2 pi i pos/(2h)}
  for (int h = 1, tws = half; h < M; h <<= 1, tws >>= 1) {
    for (int b = lane; b < half; b += 32) {
      const int pos = b & (h - 1);
      const int i0 = ((b - pos) << 1) + pos;
      const int i1 = i0 + h;
      const float2 w = __ldg(p.tw + pos * tws);
      const float2 a = buf[i0], c = buf[i1];
      const float tr = c.x * w.x - c.y * w.y;
      const float ti = c.x * w.y + c.y * w.x;
      buf[i0] = make_float2(a.x + tr, a.y + ti);
      buf[i1] = make_float2(a.x - tr, a.y - ti);
    }
    __syncwarp();
  }

  const float* mk = p.mask + (size_t)o * M;
  for (int b = lane; b < M; b += 32) {
    const float hb = __ldg(mk + b);
    const float2 v = buf[b];
    buf[b] = make_float2(v.x * hb, v.y * hb);
  }
  __syncwarp();

  // inverse DIF, span h = M/2, ..., 1; twiddle e^{+2 pi i pos/(2h)}
  for (int h = half, tws = 1; h >= 1; h >>= 1, tws <<= 1) {
    for (int b = lane; b < half; b += 32) {
      const int pos = b & (h - 1);
      const int i0 = ((b - pos) << 1) + pos;
      const int i1 = i0 + h;
      const float2 w = __ldg(p.tw + pos * tws);
      const float2 a = buf[i0], c = buf[i1];
      buf[i0] = make_float2(a.x + c.x, a.y + c.y);
      const float dx = a.x - c.x, dy = a.y - c.y;
      buf[i1] = make_float2(dx * w.x + dy * w.y, dy * w.x - dx * w.y);
    }
    __syncwarp();
  }

  const float inv_m = 1.0f / (float)M;
  float mx = 0.f;
  for (int n = lane; n < p.nz; n += 32) {
    const float2 y = buf[bit_reverse(n, L)];
    const float env = sqrtf(y.x * y.x + y.y * y.y) * inv_m;
    dst[n] = env;
    mx = fmaxf(mx, env);
  }
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, s));
  if (lane == 0) atomicMax(p.maxslot + (size_t)f * p.n_out + o, __float_as_int(mx));
}

__global__ void __launch_bounds__(256) k_log(const LogParams p) {
  const int img = blockIdx.y;  // frame * n_out + output
  const int f = img / p.n_out, o = img - f * p.n_out;
  const float mx = __int_as_float(p.maxslot[img]);
  const float inv = mx > 0.f ? 1.0f / mx : 0.f;
  const float dr = p.dyn_range_db;
  const float* src = p.out + ((size_t)f * p.planes + (size_t)p.s_src * p.n_out + o) * p.plane_elems;
  float* dst = p.out + ((size_t)f * p.planes + (size_t)p.s_dst * p.n_out + o) * p.plane_elems;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < p.plane_elems;
       q += (long long)gridDim.x * blockDim.x) {
    const float env = src[q];
    float v = -dr;
    if (mx > 0.f && env > 0.f) v = fminf(0.f, fmaxf(-dr, 20.0f * log10f(env * inv)));
    dst[q] = v;
  }
}

cudaError_t post_configure(size_t smem) {
  return cudaFuncSetAttribute(k_post, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t post_launch(const PostParams& p, cudaStream_t s) {
  const size_t smem = (size_t)p.warps_per_block * p.m * sizeof(float2);
  dim3 grid((p.nx + p.warps_per_block - 1) / p.warps_per_block, p.n_out, p.n_frames);
  k_post<<<grid, p.warps_per_block * 32, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t log_launch(const LogParams& p, int num_sms, cudaStream_t s) {
  long long blocks = (p.plane_elems + 255) / 256;
  const long long images = (long long)p.n_frames * p.n_out;
  const long long target = (long long)num_sms * 8;
  long long per_img = (target + images - 1) / images;
  if (per_img < 1) per_img = 1;
  if (blocks > per_img) blocks = per_img;
  dim3 grid((unsigned)blocks, (unsigned)images);
  k_log<<<grid, 256, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace pa
