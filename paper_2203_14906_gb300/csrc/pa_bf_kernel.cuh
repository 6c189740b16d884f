// pa_bf_kernel.cuh -- fused delay-gather + interpolation + signed root +
// power-sum kernel with an FP64 e_k epilogue (Sections 2.1-2.3: Eq. 1 DAS,
// Eq. 3 real-time DMAS, Eqs. 7-9 O(N) DMAS-k).
//
// Delay tables: LATTICE (one entry per lattice offset and depth, shared by
// the kC pairs of a thread at one channel step, see below) or FULL (one
// entry per pixel and element, Section 5's precomputed delays for any grid);
// the FULL kernel reads kC entries per step, one per pair, as 32 contiguous
// bytes.
//
// Work decomposition (one persistent CTA loop over work items):
//   item   = (pixel tile, residue group, frame), taken from an atomic counter
//   tile   = tile_x columns x 32 depth rows; lane = depth row
//   thread = kC pixels of one row at columns jt, jt+m, ..., jt+(kC-1)m, where
//            m = pitch / dx.  At channel step u, pixel c pairs with channel
//            i = u + c and all kC pairs share the lattice offset
//            d = jt - m u, so one delay-table entry (n0, a) serves kC pairs.
//   chunk  = nc channel steps (per plan); the RF sample window of every channel the
//            chunk touches is staged in shared memory as overlapping FP32
//            pairs (r[n], r[n+1]) so one 64-bit LDS fetches both
//            interpolation taps.  Slots outside [0, Ns-2] hold zeros, which
//            reproduces the rule "s = 0 when a tap leaves the record".
// Per pair the arithmetic is FP32: interpolation, apodisation, one MUFU
// lg2/ex2 (or rsqrt) pair for the roots, power sums; Kahan-compensated
// sums are folded every kFoldBlocks*kC channels when requested, into totals
// held in tensor memory (TMEM).  Per pixel,
// the power sums p_1..p_k are turned into e_k in FP64 (see combine).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "pa_internal.cuh"

namespace pa {

// ---- hardware approximations (PTX instructions, no library code) -------
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Accumulator layout: [0] DAS = sum s, [1] q1 = sum sgn(s)|s|^(1/2),
// [2] q2 = sum |s|, [3 + (m-1)] p_m = sum x^m for m = 1..k-1.  The last
// power sum p_k is never accumulated: x^k = s for odd k (p_k = DAS) and
// x^k = |s| for even k (p_k = q2).  Every order accumulates DAS and DMAS.
template <int K>
struct NAcc {
  static constexpr int value = (K <= 2) ? 3 : K + 2;
};

template <int K>
__device__ __forceinline__ void pair_update(float* v, float s) {
  v[0] += s;
  {
    const float as = fabsf(s);
    v[2] += as;
    if constexpr (K <= 2) {
      v[1] += copysignf(sqrt_approx(as), s);
    } else if constexpr (K == 3) {
      const float y = ex2_approx(lg2_approx(as) * (1.0f / 6.0f));  // |s|^(1/6)
      const float y2 = y * y;                                      // |s|^(1/3)
      const float x = copysignf(y2, s);                            // cube root
      v[1] = fmaf(x, y, v[1]);    // sgn(s)|s|^(1/2)
      v[3] += x;                  // p1
      v[4] = fmaf(y2, y2, v[4]);  // p2
    } else if constexpr (K == 4) {
      const float y = rsqrt_approx(rsqrt_approx(as));  // |s|^(1/4)
      const float y2 = y * y;                          // |s|^(1/2)
      const float x = copysignf(y, s);
      v[1] = fmaf(x, y, v[1]);    // sgn(s)|s|^(1/2)
      v[3] += x;                  // p1
      v[4] += y2;                 // p2
      v[5] = fmaf(x, y2, v[5]);   // p3
    } else if constexpr (K == 5) {
      const float y = ex2_approx(lg2_approx(as) * 0.1f);  // |s|^(1/10)
      const float y2 = y * y;                             // |s|^(1/5)
      const float x = copysignf(y2, s);
      const float x2 = y2 * y2;
      v[1] = fmaf(x, y2 * y, v[1]);  // x y^3 = sgn(s)|s|^(1/2)
      v[3] += x;                     // p1
      v[4] += x2;                    // p2
      v[5] = fmaf(x, x2, v[5]);      // p3
      v[6] = fmaf(x2, x2, v[6]);     // p4
    } else {  // orders 6..8: generic root and powers
      const float x = copysignf(ex2_approx(lg2_approx(as) * (1.0f / K)), s);
      v[1] += copysignf(sqrt_approx(as), s);
      float xp = x;
      v[3] += x;
#pragma unroll
      for (int mm = 2; mm < K; ++mm) {
        xp *= x;
        v[2 + mm] += xp;
      }
    }
  }
}

// a^2 - 2 b (a, b >= 0) in FP32 with an error-free square: a^2 = h + l
// exactly, so the result is rounded about twice.
__device__ __forceinline__ float wsq_minus_2(float a, float b) {
  const float h = a * a;
  const float l = fmaf(a, a, -h);
  return (h - 2.0f * b) + l;
}

// Outputs of one pixel from its FP32 sums V: V[0] DAS, V[1] sum sgn sqrt|s|,
// V[2] sum |s|, V[3..] the power sums p1.. of the k-th roots.
//   DAS as is; DMAS (Eq. 3) in FP32 with an error-free square (q1^2 = h + l
//   exactly, so (q1^2 - q2) / 2 is rounded about once, as an FP64 evaluation
//   rounded to FP32 would be); e_k in FP64 from the power sums: k = 3, 4, 5
//   written out (Eqs. 7-9 in power sums; for k = 4, 5 the term p2^2 - 2 p4
//   enters as one FP32 value formed like DMAS), other orders by Newton's identities
//   m e_m = sum_{i=1}^m (-1)^(i-1) e_{m-i} p_i.  FP64 is used for e_k only:
//   on GB300 its rate is a small fraction of FP32, and for small apertures
//   (apodised images) the epilogue dominates the kernel.
template <int K>
__device__ __forceinline__ void combine(const float* V, float& das, float& dmas, float& ho) {
  das = V[0];
  {
    const float h = V[1] * V[1];
    const float l = fmaf(V[1], V[1], -h);
    dmas = 0.5f * ((h - V[2]) + l);
  }
  if constexpr (K == 1) {
    ho = das;
  } else if constexpr (K == 2) {
    ho = dmas;
  } else if constexpr (K == 3) {
    // e3 = (p1^3 - 3 p1 p2 + 2 p3) / 6.  p1^2 is exact in FP64 and each FMA
    // rounds once; scalings by powers of two are exact in FP32 and are done
    // there, as is the final division (the result is FP32): fewer FP64 ops.
    const double p1 = V[3], p2 = V[4], p3x2 = 2.0f * V[0];
    const double t = fma(p1, p1, -3.0 * p2);
    ho = (float)fma(t, p1, p3x2) * (1.0f / 6.0f);
  } else if constexpr (K == 4) {
    // e4 = (p1^4 - 6 p1^2 p2 + 8 p1 p3 + 3 w) / 24, w = p2^2 - 2 p4, p4 = sum |s|
    // (even k).  w, a square minus a sum of positives like DMAS, is formed
    // the way DMAS is: in FP32 with an error-free square (rounded about
    // twice); the terms that cancel are summed in FP64.  Two FP64-pipe
    // instructions fewer per pixel (measured on GB300, apodised 64-frame
    // k = 4 batch, fused kernel: 2.676 -> 2.563 ms).
    const double w = wsq_minus_2(V[4], V[2]);
    const double p1 = V[3], p2 = V[4], p3x8 = 8.0f * V[5];
    const double t = p1 * p1;
    double e = fma(-6.0, p2, t) * t;
    e = fma(p1, p3x8, e);
    ho = (float)fma(3.0, w, e) * (1.0f / 24.0f);
  } else if constexpr (K == 5) {
    // e5 = (p1 (p1^4 - 10 p1^2 p2 + 15 w) + 20 p3 (p1^2 - p2) + 24 p5) / 120,
    // w = p2^2 - 2 p4 as for k = 4, p5 = sum s (odd k); 8 p5 is exact in
    // FP32 (24 p5 = 3 (8 p5))
    const double w = wsq_minus_2(V[4], V[6]);
    const double p1 = V[3], p2 = V[4], p3 = V[5], p5x8 = 8.0f * V[0];
    const double t = p1 * p1;
    double e = fma(-10.0, p2, t) * t;
    e = fma(15.0, w, e) * p1;
    e = fma(20.0 * p3, t - p2, e);
    ho = (float)fma(3.0, p5x8, e) * (1.0f / 120.0f);
  } else {
    double p[K + 1];
#pragma unroll
    for (int mm = 1; mm < K; ++mm) p[mm] = V[2 + mm];
    p[K] = (K & 1) ? V[0] : V[2];
    double e[K + 1];
    e[0] = 1.0;
#pragma unroll
    for (int mm = 1; mm <= K; ++mm) {
      double acc = e[mm - 1] * p[1];
#pragma unroll
      for (int i = 2; i <= mm; ++i) {
        const double t = e[mm - i] * p[i];
        acc = (i & 1) ? acc + t : acc - t;
      }
      e[mm] = acc * (1.0 / mm);
    }
    ho = (float)e[K];
  }
}

// ---- RF staging ---------------------------------------------------------
// Samples are widened to FP32 on the way into shared memory; the storage type
// only changes the load.
template <int DT>
__device__ __forceinline__ float rf_load(const void* rf, size_t idx) {
  if constexpr (DT == PA_RF_F32) {
    return __ldg(reinterpret_cast<const float*>(rf) + idx);
  } else {
    const unsigned short u = __ldg(reinterpret_cast<const unsigned short*>(rf) + idx);
    if constexpr (DT == PA_RF_BF16) return __uint_as_float(((unsigned)u) << 16);
    return __half2float(__ushort_as_half(u));
  }
}

// Four consecutive samples at element idx (idx % 4 == 0, row start aligned).
template <int DT>
__device__ __forceinline__ void rf_load4(const void* rf, size_t idx, float* r) {
  if constexpr (DT == PA_RF_F32) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(rf) + idx));
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
  } else {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const unsigned short*>(rf) + idx));
    const unsigned w[4] = {v.x & 0xffffu, v.x >> 16, v.y & 0xffffu, v.y >> 16};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if constexpr (DT == PA_RF_BF16) r[t] = __uint_as_float(w[t] << 16);
      else r[t] = __half2float(__ushort_as_half((unsigned short)w[t]));
    }
  }
}

static_assert(kC == 4, "channel-base loads below read 2 x int4");

// Stage the sample windows of virtual channels [v0, v0 + ncs) of one tile.
// Slot q of staged channel cv holds (r[n], r[n+1] - r[n]) for n = lo + q, so
// the interpolated sample is one FMA, s = r[n] + a (r[n+1] - r[n]); samples
// outside [0, Ns) (and virtual channels) are zero.  The plan-time table never
// points a pair at a slot with exactly one tap inside the record, so a delay
// whose taps leave the record reads (0, 0).  s_cb[cv] is the 32-bit shared
// address of sample 0 of the channel's window, so the slot of sample n0 lives
// at s_cb[cv] + 8 n0 (lattice table); with the full table, whose entries
// hold n0 - lo, it is the address of the window's first slot.  Work is
// spread over the whole block, four slots per thread-iteration.  A first
// pass writes, per staged channel, the frame-relative index of its window's
// first sample when the whole window (and the sample after it) lies inside
// the record and vector loads apply, else -1 (s_off); after one barrier the
// iterations of those channels need no bounds checks or row arithmetic.
template <int DT>
__device__ __forceinline__ void stage_chunk(const BfParams& p, int frame, int tile_id, int v0,
                                            int* s_cb, int* s_off, unsigned char* smem,
                                            uint32_t sbase) {
  constexpr size_t kElt = DT == PA_RF_F32 ? 4 : 2;
  const int W = p.window, W4 = W >> 2;
  const int ns = p.n_samples;
  const int* lo_t = p.lo + (size_t)tile_id * p.nv;
  const size_t frame_base = (size_t)frame * p.n_elem;
  const void* frame_rf = reinterpret_cast<const char*>(p.rf) + frame_base * (size_t)ns * kElt;
  for (int c = threadIdx.x; c < p.ncs; c += blockDim.x) {
    const int v = v0 + c;
    const int lo = v < p.nv ? __ldg(lo_t + v) : 0;
    s_cb[c] = (int)sbase + p.pairs_off + c * W * 8 - (p.full ? 0 : lo * 8);
    const int i = v + p.u0;
    const long long o = (long long)i * ns + lo;
    const bool inside = p.vec_ok && v < p.nv && i >= 0 && i < p.n_elem && lo >= 0 &&
                        lo + 4 * W4 <= ns - 1 && o + 4 * W4 < 0x7fffffffll;
    s_off[c] = inside ? (int)o : -1;
  }
  __syncthreads();
  const int total = p.ncs * W4;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int cv = (int)(((unsigned)idx * (unsigned)p.w4_inv) >> 20);  // idx / W4
    const int q = idx - cv * W4;
    const int off = s_off[cv];
    float r[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (off >= 0) {
      const size_t e = (size_t)(unsigned)(off + 4 * q);
      rf_load4<DT>(frame_rf, e, r);
      r[4] = rf_load<DT>(frame_rf, e + 4);
    } else {
      // a window that leaves the record, a virtual channel, or unaligned rows
      const int v = v0 + cv;
      const int i = v + p.u0;
      const bool real = v < p.nv && i >= 0 && i < p.n_elem;
      const int n = (v < p.nv ? __ldg(lo_t + v) : 0) + 4 * q;
      if (real) {
        const size_t row = (size_t)i * (size_t)ns;
        if (p.vec_ok && n >= 0 && n + 4 <= ns - 1) {
          rf_load4<DT>(frame_rf, row + n, r);
          r[4] = rf_load<DT>(frame_rf, row + n + 4);
        } else {
#pragma unroll
          for (int t = 0; t < 5; ++t) {
            const int k = n + t;
            if (k >= 0 && k < ns) r[t] = rf_load<DT>(frame_rf, row + k);
          }
        }
      }
    }
    float4* dst = reinterpret_cast<float4*>(smem + p.pairs_off + (size_t)(cv * W + 4 * q) * 8);
    dst[0] = make_float4(r[0], r[1] - r[0], r[1], r[2] - r[1]);
    dst[1] = make_float4(r[2], r[3] - r[2], r[3], r[4] - r[3]);
  }
}

// ---- TMA staging ----------------------------------------------------------
// One 1-D box of wr samples per staged channel, loaded by the tensor memory
// accelerator straight from the 3-D RF map into the raw buffer; coordinates
// outside the record (negative or >= Ns samples, channels outside [0, N))
// read as zeros.  One mbarrier counts the bytes of a chunk.
__device__ __forceinline__ void mbar_init(uint32_t mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t mbar, int bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, int parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n"
      " selp.u32 %0, 1, 0, P;\n}"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for the chunk with a bound of about one second of SM clock; returns
// false if the bytes never arrived.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, int parity) {
  const long long t0 = clock64();
  while (!mbar_try(mbar, parity)) {
    if (clock64() - t0 > 2000000000LL) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_box(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                        uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar)
      : "memory");
}

// The boxes of a chunk are issued by ncs threads spread over the warps
// (staged channel cv = lane * nwarps + warp; the plan keeps ncs <= 32 nwarps,
// so every staged channel has an issuing lane), so no warp falls behind the
// others; each issuing thread keeps its channel's next window start in a
// register, loaded one chunk ahead.
__device__ __forceinline__ int tma_channel(int ncs) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int cv = lane * nwarps + warp;
  return cv < ncs ? cv : -1;
}

__device__ __forceinline__ int window_start(const BfParams& p, int tile_id, int k, int cv) {
  const int v = k * p.nc + cv;
  return v < p.nv ? __ldg(p.lo + (size_t)tile_id * p.nv + v) : 0;
}

// Issue the boxes of chunk k of (tile, frame); every thread calls it.
__device__ __forceinline__ void tma_issue_chunk(const BfParams& p, int frame, int k, int cv, int lo,
                                                int* s_lo, uint32_t raw_s, uint32_t mbar) {
  if (threadIdx.x == 0) mbar_expect(mbar, p.chunk_bytes + p.expect_extra);
  if (cv >= 0) {
    const int elt = p.rf_dtype == PA_RF_F32 ? 4 : 2;
    s_lo[cv] = lo;
    tma_box(raw_s + (uint32_t)(cv * p.rp * elt), &p.tmap, lo, k * p.nc + cv + p.u0, frame, mbar);
  }
}

// Raw samples of a chunk -> (r[n], r[n+1] - r[n]) slots and channel bases.
template <int DT>
__device__ __forceinline__ void convert_chunk(const BfParams& p, int* s_cb, const int* s_lo,
                                              unsigned char* smem, uint32_t sbase) {
  const int W = p.window, W4 = W >> 2;
  for (int c = threadIdx.x; c < p.ncs; c += blockDim.x)
    s_cb[c] = (int)sbase + p.pairs_off + c * W * 8 - (p.full ? 0 : s_lo[c] * 8);
  const int total = p.ncs * W4;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int cv = (int)(((unsigned)idx * (unsigned)p.w4_inv) >> 20);  // idx / W4
    const int q = idx - cv * W4;
    const int base = cv * p.rp + 4 * q;
    float r[5];
    if constexpr (DT == PA_RF_F32) {
      const float* raw = reinterpret_cast<const float*>(smem + kRawOff);
      const float4 v = *reinterpret_cast<const float4*>(raw + base);
      r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
      r[4] = raw[base + 4];
    } else {
      const unsigned short* raw = reinterpret_cast<const unsigned short*>(smem + kRawOff);
      const uint2 v = *reinterpret_cast<const uint2*>(raw + base);
      const unsigned w[5] = {v.x & 0xffffu, v.x >> 16, v.y & 0xffffu, v.y >> 16, raw[base + 4]};
#pragma unroll
      for (int t = 0; t < 5; ++t) {
        if constexpr (DT == PA_RF_BF16) r[t] = __uint_as_float(w[t] << 16);
        else r[t] = __half2float(__ushort_as_half((unsigned short)w[t]));
      }
    }
    float4* dst = reinterpret_cast<float4*>(smem + p.pairs_off + (size_t)(cv * W + 4 * q) * 8);
    dst[0] = make_float4(r[0], r[1] - r[0], r[1], r[2] - r[1]);
    dst[1] = make_float4(r[2], r[3] - r[2], r[3], r[4] - r[3]);
  }
}

struct ItemInfo {
  int tile_id, grp, frame, tz, tx;
};

// Work item = (tile, residue group) x frame, frame fastest; the host-built
// item table lists (tile, group) pairs deepest tiles first.
__device__ __forceinline__ ItemInfo decode_item(const BfParams& p, int item) {
  ItemInfo it;
  const int tg = item / p.n_frames;
  it.frame = item - tg * p.n_frames;
  const int4 e = __ldg(p.items + tg);
  it.tile_id = e.x;
  it.grp = e.y;
  it.tx = e.z;
  it.tz = e.w;
  return it;
}

// ---- Tensor memory (TMEM) for the Kahan totals of compensated sums -------
// The kernel does no matrix work, so the SM's 256 KB of tensor memory is
// free to hold the Kahan totals and compensation terms.  Warp w reaches TMEM
// lanes 32 (w % 4) .. 32 (w % 4) + 31 (lane = its own lane); warps w and
// w + 4 share those lanes and split the columns.  Accumulator q of a thread
// lives in 8 consecutive 32-bit columns: the totals of its kC = 4 pixels,
// then their compensation terms.  Every load and store waits for its own
// completion inside the same asm statement, so no TMEM access is in flight
// once a thread passes a barrier.
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, int ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               ::"r"(dst_smem), "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, int ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n"
      "tcgen05.wait::st.sync.aligned;" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
      : "memory");
}

// Kahan fold of the partial sums into the running totals held in TMEM.  The
// warp executes it converged: the plans that use it give every lane of a warp
// the same channel-step range (one slot per warp, or slots without
// apodisation, whose ranges are all the full aperture).  LAZY: the first
// fold of a work item folds into zero totals without loading them, so
// nothing has to zero TMEM before the item (apodised plans, whose items
// mostly end before their first fold); otherwise the totals are zeroed when
// the item starts and every fold loads them (no branch in the fold).
template <int NA, bool LAZY>
__device__ __forceinline__ void kahan_fold_tmem(float (&acc)[kC][NA], uint32_t tmem, bool first) {
  static_assert(kC == 4, "totals and compensation terms of one accumulator fill 8 columns");
  __syncwarp();
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    float t[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (!LAZY || !first) tmem_ld8(tmem + 8 * q, t);
#pragma unroll
    for (int c = 0; c < kC; ++c) {
      const float y = acc[c][q] - t[4 + c];
      const float s = t[c] + y;
      t[4 + c] = (s - t[c]) - y;
      t[c] = s;
      acc[c][q] = 0.f;
    }
    tmem_st8(tmem + 8 * q, t);
  }
}

// The last fold of a work item, straight into the values the epilogue
// combines: totals plus the remaining partial sums, compensated, rounded
// once to FP32 (total minus compensation), nothing stored back.
template <int NA>
__device__ __forceinline__ void kahan_final_tmem(float (&acc)[kC][NA], uint32_t tmem) {
  __syncwarp();
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    float t[8];
    tmem_ld8(tmem + 8 * q, t);
#pragma unroll
    for (int c = 0; c < kC; ++c) {
      const float y = acc[c][q] - t[4 + c];
      const float s = t[c] + y;
      acc[c][q] = s - ((s - t[c]) - y);
    }
  }
}

// Compensated sums keep their Kahan totals in TMEM.  Measured on GB300
// against the earlier forms (BF16 RF, fused kernel per launch): totals in
// registers for k = 3 (128 registers, 2 blocks per SM) 0.752 -> 0.676 ms at
// 3 blocks per SM; totals in shared memory for k = 4 / 5 / 8 (cfg2 geometry,
// 32 frames) 0.893 / 1.010 / 2.199 -> 0.752 / 0.866 / 1.514 ms, the
// apodised 64-frame k = 4 batch 2.91 -> 2.75 ms.
template <int K, bool COMP>
struct TmemSums {
  static constexpr bool value = COMP;
};

// Resident 256-thread blocks per SM the register allocation targets: four
// (64 registers) for plain orders <= 3, three (80 registers) for compensated
// orders <= 3 (at 64 registers, four blocks per SM, they spill: cfg2 k = 3
// BF16 0.717 ms with TMA staging and 0.750 ms with loads, against 0.663 ms
// at 80) and for orders 4-5, two for orders >= 6.
#ifndef PA_MINB4_MAX_K
#define PA_MINB4_MAX_K 3
#endif
template <int K, bool COMP>
struct MinBlocks {
  static constexpr int value = K >= 6 ? 2 : (K <= PA_MINB4_MAX_K && !COMP ? 4 : 3);
};

template <int K, bool APOD, bool COMP, bool FULL>
__global__ void __launch_bounds__(256, (MinBlocks<K, COMP>::value))
    k_bf_fused(const __grid_constant__ BfParams p) {
  constexpr int NA = NAcc<K>::value;
  extern __shared__ __align__(128) unsigned char smem[];
  // [0] item to run next, [1] its first chunk is already loading, [2] the
  // item after it (taken from the counter one item ahead)
  int* s_item = reinterpret_cast<int*>(smem);
  int* s_cb = reinterpret_cast<int*>(smem + kCbOff);
  int* s_lo = reinterpret_cast<int*>(smem + kLoOff);
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t mbar = sbase + kMbarOff;
  const int my_cv = tma_channel(p.ncs);
  const uint32_t raw_s = sbase + kRawOff;
  const int pairs_off = (int)sbase + p.pairs_off;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
#ifdef PA_CHECK_BOUNDS
  const int smem_hi = pairs_off + p.ncs * p.window * 8 - 8;  // shared addresses
#endif
  int phase = 0;
  constexpr bool TSUM = TmemSums<K, COMP>::value;
  if constexpr (TSUM) {
    if (warp == 0) {  // the whole warp allocates; the address lands in shared memory
      tmem_alloc(sbase + kTmemOff, p.tmem_cols);
      tc_fence_before_sync();
    }
  }
  if (threadIdx.x == 0) {
    if (p.use_tma) mbar_init(mbar);
    s_item[0] = atomicAdd(p.counter, 1);
    s_item[1] = 0;
    s_item[2] = 0;
  }
  __syncthreads();
  uint32_t tmem = 0;  // this warp's TMEM lanes and columns (compensated orders <= 3)
  if constexpr (TSUM) {
    tc_fence_after_sync();
    tmem = *reinterpret_cast<const volatile uint32_t*>(smem + kTmemOff) +
           ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * NA * 8);
  }

  for (;;) {
    const int item = s_item[0];
    const bool prefetched = s_item[1] != 0;
    __syncthreads();
    if (item >= p.n_items) break;
    if (threadIdx.x == 0) s_item[2] = atomicAdd(p.counter, 1);
    const ItemInfo it = decode_item(p, item);
    const int tz = it.tz, tx = it.tx, tile_id = it.tile_id, grp = it.grp, frame = it.frame;
    // Lanes -> (warp slot, depth row): lane_rows consecutive rows of
    // 32 / lane_rows neighbouring slots per warp; the block's warps cover its
    // slots x the tile's 32 rows.  Fewer rows per lane group shrink the
    // span of a half-warp's 64-bit shared gather (the delay advances ~2
    // samples per row).
    const int lr_log2 = p.lane_rows_log2;
    const int spw_log2 = 5 - lr_log2;              // slots per warp
    const int sg = nwarps >> spw_log2;             // slot groups of the block
    const int sl = grp * nwarps + ((warp % sg) << spw_log2) + (lane >> lr_log2);
    const int zr = ((warp / sg) << lr_log2) + (lane & ((1 << lr_log2) - 1));
    const int2 rg = __ldg(p.slot_rg + sl);
    const int r_m = rg.x, g = rg.y;
    const int jt = tx * p.tile_x + g * p.m * kC + r_m;
    const int z = tz * p.tile_z + zr;
    const int2 ur = __ldg(p.urange + (size_t)tile_id * p.slots + sl);
    const int2 vk = __ldg(p.vchunks + (size_t)tile_id * p.ngroups + grp);

    float acc[kC][NA];
#pragma unroll
    for (int c = 0; c < kC; ++c)
#pragma unroll
      for (int q = 0; q < NA; ++q) acc[c][q] = 0.f;
    // Lazy TMEM totals for apodised plans: an item's narrow aperture rarely
    // reaches a fold.  Measured on GB300 (fused kernel per launch): the
    // throughput batch 2.711 -> 2.664 ms lazy; without apodisation the
    // branch cost more than it saved (cfg2 BF16 k = 3 0.661 -> 0.680 ms).
    constexpr bool LAZY = APOD;
    if constexpr (TSUM && !LAZY) {
      const float z8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int q = 0; q < NA; ++q) tmem_st8(tmem + 8 * q, z8);
    }
    int fold = 0;
    bool tsum_live = !LAZY;  // this item's totals are in TMEM

    // Table rows of this thread.  LATTICE: row t(u) = jt - dmin - m u at
    // depth z.  FULL: the kC entries of step u (pixel c, column jt + m c,
    // with channel u + c) are two 16-byte pairs, pixels 0-1 at fbase0 +
    // (u - u0) fstep and pixels 2-3 half a step further (fhalf): per tile,
    // step and half, the threads' pairs are contiguous.
    // The depth-blocked table layout is only ever chosen for orders <= 2 and
    // compensated plans without apodisation; the other instantiations keep
    // the row-major address (their code measured faster without the general
    // form).
    constexpr bool TBLOCKED = (K <= 2 || COMP) && !APOD;
    const int2* tcol;
    const float* wcol;
    if constexpr (TBLOCKED) {
      const size_t trow0 =  // table row 0 at depth z
          (size_t)(z >> p.table_zshift) * (size_t)p.table_zblock + (z & p.table_zmask);
      tcol = p.table + trow0;
      wcol = nullptr;
    } else {
      tcol = p.table + z;
      wcol = APOD ? p.wtab + z : nullptr;
    }
    const int row_u0 = jt - p.dmin;
    const int mstride = p.m * p.table_stride;
    const size_t fhalf = (size_t)32 * p.slots * 2;
    const size_t fstep = 2 * fhalf;
    const size_t fbase0 = (size_t)tile_id * (p.steps + 3) * fstep +
                          (((size_t)(warp / sg) * p.slots + sl) * (1 << lr_log2) +
                           (lane & ((1 << lr_log2) - 1))) * 2;

    int lo_next = 0;  // window start of my channel in the next chunk to issue
    if (p.use_tma && vk.x < vk.y) {
      if (!prefetched) {
        if (my_cv >= 0) lo_next = window_start(p, tile_id, vk.x, my_cv);
        tma_issue_chunk(p, frame, vk.x, my_cv, lo_next, s_lo, raw_s, mbar);
      }
      if (my_cv >= 0 && vk.x + 1 < vk.y) lo_next = window_start(p, tile_id, vk.x + 1, my_cv);
    }
    bool timed_out = false;
    for (int k = vk.x; k < vk.y; ++k) {
      if (p.use_tma) {
        // raw samples of chunk k landed?  (this barrier also frees the slots:
        // every warp has finished chunk k - 1)
        const bool ok = mbar_wait_bounded(mbar, phase);
        phase ^= 1;
        if (!__syncthreads_and(ok)) {
          if (threadIdx.x == 0) {
            atomicOr(p.err, 8);
            atomicAdd(p.timeouts, 1);
          }
          timed_out = true;
          break;
        }
        if (p.rf_dtype == PA_RF_F32) convert_chunk<PA_RF_F32>(p, s_cb, s_lo, smem, sbase);
        else if (p.rf_dtype == PA_RF_BF16) convert_chunk<PA_RF_BF16>(p, s_cb, s_lo, smem, sbase);
        else convert_chunk<PA_RF_F16>(p, s_cb, s_lo, smem, sbase);
        __syncthreads();
        // the raw buffer was read through the generic proxy; order that before
        // the next asynchronous-proxy writes into it
        if (my_cv >= 0 || threadIdx.x == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (k + 1 < vk.y) {
          tma_issue_chunk(p, frame, k + 1, my_cv, lo_next, s_lo, raw_s, mbar);
          if (my_cv >= 0 && k + 2 < vk.y) lo_next = window_start(p, tile_id, k + 2, my_cv);
        } else {
          // last chunk: start the first chunk of the next work item now
          const int nxt = s_item[2];
          int pre = 0;
          if (nxt < p.n_items) {
            const ItemInfo ni = decode_item(p, nxt);
            const int2 nvk = __ldg(p.vchunks + (size_t)ni.tile_id * p.ngroups + ni.grp);
            if (nvk.x < nvk.y) {
              const int lo = my_cv >= 0 ? window_start(p, ni.tile_id, nvk.x, my_cv) : 0;
              tma_issue_chunk(p, ni.frame, nvk.x, my_cv, lo, s_lo, raw_s, mbar);
              pre = 1;
            }
          }
          if (threadIdx.x == 0) {
            s_item[0] = nxt;
            s_item[1] = pre;
          }
        }
      } else {
        __syncthreads();
        if (p.rf_dtype == PA_RF_F32) stage_chunk<PA_RF_F32>(p, frame, tile_id, k * p.nc, s_cb, s_lo, smem, sbase);
        else if (p.rf_dtype == PA_RF_BF16) stage_chunk<PA_RF_BF16>(p, frame, tile_id, k * p.nc, s_cb, s_lo, smem, sbase);
        else stage_chunk<PA_RF_F16>(p, frame, tile_id, k * p.nc, s_cb, s_lo, smem, sbase);
        __syncthreads();
      }
      const int cu0 = p.u0 + k * p.nc;
      int u = max(cu0, ur.x);
      const int u_end = min(cu0 + p.nc, ur.y);
      if (u >= u_end) continue;

      if constexpr (FULL) {
        // Entries [and weights] of the kC pairs of step uu: two 16-byte loads.
        auto load_step = [&](int2 (&e)[kC], float (&w)[kC], int uu) {
          const size_t o = fbase0 + (size_t)(uu - p.u0) * fstep;
#ifdef PA_CHECK_BOUNDS
          if (o + fhalf + 2 > (size_t)(tile_id + 1) * (p.steps + 3) * fstep) atomicOr(p.err, 1);
#endif
          const int4 q0 = __ldg(reinterpret_cast<const int4*>(p.ftab + o));
          const int4 q1 = __ldg(reinterpret_cast<const int4*>(p.ftab + o + fhalf));
          e[0] = make_int2(q0.x, q0.y);
          e[1] = make_int2(q0.z, q0.w);
          e[2] = make_int2(q1.x, q1.y);
          e[3] = make_int2(q1.z, q1.w);
          if constexpr (APOD) {
            const float2 w0 = __ldg(reinterpret_cast<const float2*>(p.wtab + o));
            const float2 w1 = __ldg(reinterpret_cast<const float2*>(p.wtab + o + fhalf));
            w[0] = w0.x;
            w[1] = w0.y;
            w[2] = w1.x;
            w[3] = w1.y;
          }
        };
        // kC steps from uu; the entries of the step after next are loaded
        // while the current one is evaluated (the padding steps at the end
        // of the tile's table keep those loads in bounds).
        auto fblock = [&](auto near_tag, int2 (&e)[kC], int2 (&e1)[kC], float (&w)[kC],
                          float (&w1)[kC], int uu) {
          constexpr bool NEAR = decltype(near_tag)::value;
          int cb[2 * kC];
          {
            const int4* cbv = reinterpret_cast<const int4*>(s_cb + (uu - cu0));
            const int4 c0 = cbv[0], c1 = cbv[1];
            cb[0] = c0.x; cb[1] = c0.y; cb[2] = c0.z; cb[3] = c0.w;
            cb[4] = c1.x; cb[5] = c1.y; cb[6] = c1.z; cb[7] = c1.w;
          }
#pragma unroll
          for (int tt = 0; tt < kC; ++tt) {
            int2 e2[kC];
            float w2[kC];
            load_step(e2, w2, uu + tt + 2);
#pragma unroll
            for (int c = 0; c < kC; ++c) {
              int addr = cb[tt + c] + e[c].x;
#ifdef PA_CHECK_BOUNDS
              if (addr < pairs_off || addr > smem_hi) {
                atomicOr(p.err, 2);
                addr = pairs_off;
              }
#endif
              float s;
              if constexpr (NEAR) {
                asm volatile("ld.shared.f32 %0, [%1];" : "=f"(s) : "r"(addr));
              } else {
                float2 r;
                asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "r"(addr));
                s = fmaf(__int_as_float(e[c].y), r.y, r.x);
              }
              if constexpr (APOD) s *= w[c];
              pair_update<K>(acc[c], s);
            }
#pragma unroll
            for (int c = 0; c < kC; ++c) {
              e[c] = e1[c];
              e1[c] = e2[c];
              if constexpr (APOD) {
                w[c] = w1[c];
                w1[c] = w2[c];
              }
            }
          }
          if constexpr (COMP) {
            if (++fold == kFoldBlocks) {
              kahan_fold_tmem<NA, LAZY>(acc, tmem, !tsum_live);
              tsum_live = true;
              fold = 0;
            }
          }
        };
        int2 e[kC], e1[kC];
        float w[kC], w1[kC];
        load_step(e, w, u);
        load_step(e1, w1, u + 1);
        for (; u < u_end; u += kC) {
          if (p.nearest) fblock(std::true_type{}, e, e1, w, w1, u);
          else fblock(std::false_type{}, e, e1, w, w1, u);
        }
        continue;
      } else {

      // Table entries (n0, a) [and weight] of the kC steps starting at uu.
      auto load_entries = [&](int2 (&ee)[kC], float (&ww)[kC], int uu) {
        const int r0 = row_u0 - p.m * uu;
#ifdef PA_CHECK_BOUNDS
        if (r0 - (kC - 1) * p.m < 0 || r0 >= p.ndrows) atomicOr(p.err, 1);
#endif
        const int2* tp = tcol + (size_t)r0 * p.table_stride;
        const float* wp = APOD ? wcol + (size_t)r0 * p.table_stride : nullptr;
#pragma unroll
        for (int tt = 0; tt < kC; ++tt) {
          ee[tt] = __ldg(tp - tt * mstride);
          if constexpr (APOD) ww[tt] = __ldg(wp - tt * mstride);
        }
      };
      // kC channel steps x kC columns = kC^2 pairs.  NEAR: nearest-sample
      // delays (Eq. 1), one tap per pair and no interpolation.
      auto block = [&](auto near_tag, const int2 (&ee)[kC], const float (&ww)[kC], int uu) {
        constexpr bool NEAR = decltype(near_tag)::value;
        int cb[2 * kC];
        {
          // channel bases of channels uu .. uu + 2kC - 2 (uu - cu0 is a multiple of 4)
          const int4* cbv = reinterpret_cast<const int4*>(s_cb + (uu - cu0));
          const int4 c0 = cbv[0], c1 = cbv[1];
          cb[0] = c0.x; cb[1] = c0.y; cb[2] = c0.z; cb[3] = c0.w;
          cb[4] = c1.x; cb[5] = c1.y; cb[6] = c1.z; cb[7] = c1.w;
        }
#pragma unroll
        for (int tt = 0; tt < kC; ++tt) {
          const int off = ee[tt].x;
          const float a = __int_as_float(ee[tt].y);
#pragma unroll
          for (int c = 0; c < kC; ++c) {
            int addr = cb[tt + c] + off;
#ifdef PA_CHECK_BOUNDS
            if (addr < pairs_off || addr > smem_hi) {
              atomicOr(p.err, 2);
              addr = pairs_off;
            }
#endif
            float s;
            if constexpr (NEAR) {
              asm volatile("ld.shared.f32 %0, [%1];" : "=f"(s) : "r"(addr));
            } else {
              float2 r;
              asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "r"(addr));
              s = fmaf(a, r.y, r.x);
            }
            if constexpr (APOD) s *= ww[tt];
            pair_update<K>(acc[c], s);
          }
        }
        if constexpr (COMP) {
          if (++fold == kFoldBlocks) {
            kahan_fold_tmem<NA, LAZY>(acc, tmem, !tsum_live);
            tsum_live = true;
            fold = 0;
          }
        }
      };
      // Two blocks per iteration so the prefetched entries alternate between
      // two register sets instead of being copied.
      int2 ea[kC], eb[kC];
      float wa[kC], wb[kC];
      load_entries(ea, wa, u);
      for (; u < u_end; u += 2 * kC) {
        const bool has_b = u + kC < u_end;
        if (has_b) load_entries(eb, wb, u + kC);
        if (p.nearest) block(std::true_type{}, ea, wa, u);
        else block(std::false_type{}, ea, wa, u);
        if (!has_b) break;
        if (u + 2 * kC < u_end) load_entries(ea, wa, u + 2 * kC);
        if (p.nearest) block(std::true_type{}, eb, wb, u + kC);
        else block(std::false_type{}, eb, wb, u + kC);
      }
      }  // LATTICE
    }
    if (timed_out) break;
    // compensated sums: the TMEM totals combine with the last partial sums;
    // a lazy item that never folded (at most kFoldBlocks blocks of steps)
    // already holds its sums
    if constexpr (TSUM) {
      if (tsum_live) kahan_final_tmem<NA>(acc, tmem);
    }
    if (threadIdx.x == 0 && (!p.use_tma || vk.x >= vk.y)) {
      s_item[0] = s_item[2];
      s_item[1] = 0;
    }

    // ---- epilogue (FP64 e_k) and store -----------------------------------
    const size_t plane = (size_t)p.nx * p.nz;
    const size_t fbase = (size_t)frame * p.planes * plane;
#pragma unroll
    for (int c = 0; c < kC; ++c) {
      const int j = jt + p.m * c;
      if (j < p.nx && z < p.nz) {
        // plain sums, or compensated totals minus compensations rounded once
        // to FP32 (kahan_final_tmem)
        float V[NA];
#pragma unroll
        for (int q = 0; q < NA; ++q) V[q] = acc[c][q];
        float das, dmas, ho;
        combine<K>(V, das, dmas, ho);
        const size_t px = fbase + (size_t)j * p.nz + z;
        if (p.plane_das >= 0) p.out[px + (size_t)p.plane_das * plane] = das;
        if (p.plane_dmas >= 0) p.out[px + (size_t)p.plane_dmas * plane] = dmas;
        if (p.plane_ho >= 0) p.out[px + (size_t)p.plane_ho * plane] = ho;
      }
    }
    __syncthreads();  // s_item is rewritten before the next item starts
  }
  if constexpr (TSUM) {  // every thread's TMEM accesses completed before the barrier
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) {
      tc_fence_after_sync();
      tmem_dealloc(*reinterpret_cast<const volatile uint32_t*>(smem + kTmemOff), p.tmem_cols);
    }
  }
}

}  // namespace pa

// One translation unit per order: launch and occupancy wrappers.
#define PA_DEFINE_ORDER(K)                                                      \
  namespace pa {                                                                \
  template <bool FULL>                                                          \
  static void (*pick_form_k##K(bool apod, bool comp))(BfParams) {               \
    if (apod)                                                                   \
      return comp ? k_bf_fused<K, true, true, FULL> : k_bf_fused<K, true, false, FULL>; \
    return comp ? k_bf_fused<K, false, true, FULL> : k_bf_fused<K, false, false, FULL>; \
  }                                                                             \
  static void (*pick_k##K(bool apod, bool comp, bool full))(BfParams) {         \
    return full ? pick_form_k##K<true>(apod, comp) : pick_form_k##K<false>(apod, comp); \
  }                                                                             \
  cudaError_t bf_launch_k##K(bool apod, bool comp, bool full, const BfParams& p, \
                             int grid, int block, size_t smem, cudaStream_t s) { \
    void (*f)(BfParams) = pick_k##K(apod, comp, full);                          \
    f<<<grid, block, smem, s>>>(p);                                             \
    return cudaGetLastError();                                                  \
  }                                                                             \
  cudaError_t bf_occupancy_k##K(bool apod, bool comp, bool full, int block,     \
                                size_t smem, int* blocks_per_sm) {              \
    void (*f)(BfParams) = pick_k##K(apod, comp, full);                          \
    cudaError_t e = cudaFuncSetAttribute(                                       \
        f, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);            \
    if (e != cudaSuccess) return e;                                             \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f,      \
                                                         block, smem);          \
  }                                                                             \
  const void* bf_func_k##K(bool apod, bool comp, bool full) {                   \
    return reinterpret_cast<const void*>(pick_k##K(apod, comp, full));          \
  }                                                                             \
  }
