// pa_post.cu -- band-pass + Hilbert envelope + log compression (Section 3:
// the beamformed images are band-pass filtered, envelope-detected through
// the Hilbert transform and log-compressed before display).
//
// k_post: one warp per pair of depth columns (j, j+1).  The two real columns
// are packed into one complex sequence a + i b, zero-padded to
// M = 2^ceil(log2 nz) and transformed by a Stockham (self-sorting) FFT with
// radix-8 passes (radix 4 / 2 for the remainder), each pass keeping its
// butterflies in registers.  The two spectra are separated with the
// conjugate symmetry of real inputs, A[k] = (Z[k] + Z*[M-k]) / 2 and
// B[k] = (Z[k] - Z*[M-k]) / (2i), multiplied by the plan's real mask H
// (band-pass x analytic weights: 1 at DC and M/2, 2 on positive bins, 0 on
// negative bins) and conjugated; a forward FFT of conj(H A) is the complex
// conjugate of M IFFT(H A), so the envelope is |FFT(conj(H A))[z]| / M.  The
// column maximum is merged into the image maximum with an atomic max on the
// float bits (the envelope is non-negative).  Columns are read completely
// before anything is written, so source and destination may be one plane.
//
// k_log: 20 log10(env / image max), clipped to [-DR, 0]; elementwise.
#include "pa_internal.cuh"
#include "pa_logdb.cuh"

namespace pa {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by -i
__device__ __forceinline__ float2 cmul_mi(float2 a) { return make_float2(a.y, -a.x); }

// In-register forward DFT of R = 2, 4 or 8 points (decimation in frequency,
// then the bit-reversed results are put back in natural order).
template <int R>
__device__ __forceinline__ void dft_regs(float2 (&x)[R]) {
  if constexpr (R == 2) {
    const float2 a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  } else if constexpr (R == 4) {
    float2 t0 = cadd(x[0], x[2]), t2 = csub(x[0], x[2]);
    float2 t1 = cadd(x[1], x[3]), t3 = cmul_mi(csub(x[1], x[3]));
    x[0] = cadd(t0, t1);
    x[2] = csub(t0, t1);
    x[1] = cadd(t2, t3);
    x[3] = csub(t2, t3);
  } else {
    const float h = 0.70710678118654752f;
    float2 y[8];
    // span 4
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      y[n] = cadd(x[n], x[n + 4]);
      y[n + 4] = csub(x[n], x[n + 4]);
    }
    y[5] = make_float2(h * (y[5].x + y[5].y), h * (y[5].y - y[5].x));     // * e^{-i pi/4}
    y[6] = cmul_mi(y[6]);                                                // * e^{-i pi/2}
    y[7] = make_float2(h * (y[7].y - y[7].x), -h * (y[7].x + y[7].y));    // * e^{-3i pi/4}
    // span 2
    float2 z[8];
#pragma unroll
    for (int b = 0; b < 8; b += 4) {
      z[b] = cadd(y[b], y[b + 2]);
      z[b + 2] = csub(y[b], y[b + 2]);
      z[b + 1] = cadd(y[b + 1], y[b + 3]);
      z[b + 3] = cmul_mi(csub(y[b + 1], y[b + 3]));
    }
    // span 1, outputs in bit-reversed positions
    x[0] = cadd(z[0], z[1]);
    x[4] = csub(z[0], z[1]);
    x[2] = cadd(z[2], z[3]);
    x[6] = csub(z[2], z[3]);
    x[1] = cadd(z[4], z[5]);
    x[5] = csub(z[4], z[5]);
    x[3] = cadd(z[6], z[7]);
    x[7] = csub(z[6], z[7]);
  }
}

// In-register forward DFT of 16 points in natural order: 4 x 4 (n = 4a + b,
// k = c + 4d): DFT4 over a for each b, twiddles W16^(b c), DFT4 over b for
// each c.
__device__ __forceinline__ void dft16_regs(float2 (&x)[16]) {
  float2 y[4][4];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    float2 v[4] = {x[b], x[4 + b], x[8 + b], x[12 + b]};
    dft_regs<4>(v);
#pragma unroll
    for (int c = 0; c < 4; ++c) y[b][c] = v[c];
  }
  // W16^m = cos(pi m / 8) - i sin(pi m / 8)
  const float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
  y[1][1] = cmul(y[1][1], make_float2(c1, -s1));  // m = 1
  y[1][2] = cmul(y[1][2], make_float2(h, -h));    // m = 2
  y[1][3] = cmul(y[1][3], make_float2(s1, -c1));  // m = 3
  y[2][1] = cmul(y[2][1], make_float2(h, -h));    // m = 2
  y[2][2] = cmul_mi(y[2][2]);                     // m = 4
  y[2][3] = cmul(y[2][3], make_float2(-h, -h));   // m = 6
  y[3][1] = cmul(y[3][1], make_float2(s1, -c1));  // m = 3
  y[3][2] = cmul(y[3][2], make_float2(-h, -h));   // m = 6
  y[3][3] = cmul(y[3][3], make_float2(-c1, s1));  // m = 9
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float2 v[4] = {y[0][c], y[1][c], y[2][c], y[3][c]};
    dft_regs<4>(v);
#pragma unroll
    for (int d = 0; d < 4; ++d) x[c + 4 * d] = v[d];
  }
}

template <int R>
__device__ __forceinline__ void dft_any(float2 (&x)[R]) {
  if constexpr (R == 16) dft16_regs(x);
  else dft_regs<R>(x);
}

// Shared buffers hold element i at pidx(i, ps) = i + (i >> ps): one padding
// slot every 2^ps elements (post_pad_shift).  From 256 points on, one slot
// per 16: a half-warp's 64-bit access covers 16 elements (128 bytes), so the
// contiguous accesses, the first passes' stores (stride 8 or 16) and the
// strided passes are all free of bank conflicts (one slot per 8 left every
// contiguous access 2-way conflicted; counted on the kernel's access pattern
// per column pair: 768 -> 608 wavefronts at 512 points, 1920 -> 1024 at
// 1024 points; measured 0.107 -> 0.097 ms and 1.07 -> 0.94 ms per launch).
// Below 256 points one slot per 8 measured faster (more of their passes have
// sub-transform lengths of 8).
__device__ __forceinline__ int pidx(int i, int ps) { return i + (i >> ps); }

// Twiddle tables are stored per pass in access order: the pass over
// sub-transforms of length ns (> 1) with radix R owns ns (R - 1) entries,
// entry k (R - 1) + r - 1 = e^{-2 pi i r k / (ns R)}.  A group reads its
// R - 1 twiddles from consecutive addresses.
template <int R>
__device__ __forceinline__ void twiddles(const float2* twp, int k, float2 (&w)[R]) {
  const float2* t = twp + k * (R - 1);
#pragma unroll
  for (int r = 1; r < R; ++r) w[r] = t[r - 1];
}

// One Stockham pass of radix R over sub-transforms of length ns.
template <int R>
__device__ __forceinline__ void stockham_pass(const float2* in, float2* out, int m, int ns,
                                              const float2* twp, int lane, int ps) {
  const int groups = m / R;
  // With groups a multiple of 2^ps, pidx(j + r groups) = pidx(j) + r (groups
  // + groups / 2^ps); with ns = 1 or a multiple of 2^ps the same holds for
  // the stores.  Other passes index every element.
  const int pm = (1 << ps) - 1;
  const bool strided = (groups & pm) == 0 && (ns == 1 || (ns & pm) == 0);
  const int is = groups + (groups >> ps), os = ns + (ns >> ps);
  for (int j = lane; j < groups; j += 32) {
    const int k = j & (ns - 1);
    float2 x[R];
    if (strided) {
      const float2* ip = in + pidx(j, ps);
#pragma unroll
      for (int r = 0; r < R; ++r) x[r] = ip[r * is];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) x[r] = in[pidx(j + r * groups, ps)];
    }
    if (ns > 1) {
      float2 w[R];
      twiddles<R>(twp, k, w);
#pragma unroll
      for (int r = 1; r < R; ++r) x[r] = cmul(x[r], w[r]);
    }
    dft_regs<R>(x);
    const int base = (j - k) * R + k;
    if (strided) {
      float2* op = out + pidx(base, ps);
#pragma unroll
      for (int r = 0; r < R; ++r) op[r * os] = x[r];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) out[pidx(base + r * ns, ps)] = x[r];
    }
  }
}

// Forward FFT of buf_a; returns the buffer (buf_a or buf_b) holding the result.
__device__ float2* fft_forward(float2* buf_a, float2* buf_b, int m, int log2m, const float2* tw,
                               int lane, int ps) {
  // tw: shared-memory copy of e^{-2 pi i k / m}, k < m
  float2* in = buf_a;
  float2* out = buf_b;
  int ns = 1, rem = log2m;
  const float2* twp = tw;  // per-pass twiddle blocks, in pass order
  while (rem > 0) {
    if (rem >= 3) {
      stockham_pass<8>(in, out, m, ns, twp, lane, ps);
      if (ns > 1) twp += ns * 7;
      ns *= 8;
      rem -= 3;
    } else if (rem == 2) {
      stockham_pass<4>(in, out, m, ns, twp, lane, ps);
      if (ns > 1) twp += ns * 3;
      ns *= 4;
      rem -= 2;
    } else {
      stockham_pass<2>(in, out, m, ns, twp, lane, ps);
      if (ns > 1) twp += ns;
      ns *= 2;
      rem -= 1;
    }
    __syncwarp();
    float2* t = in;
    in = out;
    out = t;
  }
  return in;
}

// A team of TW warps (TW = 1, 2 or 4) transforms one packed column pair;
// tl = lane index within the team (0 .. 32 TW - 1).  Teams of two halve the
// registers and shared memory per warp, so more warps fit an SM.
struct Team {
  int tl;  // lane within the team
  int id;  // team index within the block (named barrier 1 + id for TW = 2)
};

template <int TW>
__device__ __forceinline__ void team_sync(const Team& tm) {
  if constexpr (TW == 1) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + tm.id), "r"(32 * TW) : "memory");
  }
}

// In-place Stockham pass: each team lane first reads the R inputs of all its
// groups into registers, the team synchronises, then the outputs overwrite
// the same buffer.  M = 32 MPL points (64 <= M <= 1024).
template <int R, int MPL, int TW>
__device__ __forceinline__ void stockham_pass_inplace(float2* buf, int m, int ns, const float2* twp,
                                                      const Team& tm) {
  constexpr int TL = 32 * TW;
  constexpr int GPL = (32 * MPL / R) >= TL ? (32 * MPL / R) / TL : 1;  // groups per team lane
  constexpr int PS = post_pad_shift(32 * MPL), PM = (1 << PS) - 1;
  const int groups = m / R;
  const int is = groups + (groups >> PS), os = ns + (ns >> PS);
  const bool strided = (groups & PM) == 0 && (ns == 1 || (ns & PM) == 0);
  float2 x[GPL][R];
#pragma unroll
  for (int t = 0; t < GPL; ++t) {
    const int j = tm.tl + TL * t;
    if (j < groups) {
      if (strided) {
        const float2* ip = buf + pidx(j, PS);
#pragma unroll
        for (int r = 0; r < R; ++r) x[t][r] = ip[r * is];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) x[t][r] = buf[pidx(j + r * groups, PS)];
      }
    }
  }
  team_sync<TW>(tm);
#pragma unroll
  for (int t = 0; t < GPL; ++t) {
    const int j = tm.tl + TL * t;
    if (j < groups) {
      const int k = j & (ns - 1);
      if (ns > 1) {
        float2 w[R];
        twiddles<R>(twp, k, w);
#pragma unroll
        for (int r = 1; r < R; ++r) x[t][r] = cmul(x[t][r], w[r]);
      }
      dft_regs<R>(x[t]);
      const int base = (j - k) * R + k;
      if (strided) {
        float2* op = buf + pidx(base, PS);
#pragma unroll
        for (int r = 0; r < R; ++r) op[r * os] = x[t][r];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) buf[pidx(base + r * ns, PS)] = x[t][r];
      }
    }
  }
  team_sync<TW>(tm);
}

// The same pass over two buffers (the inverse transforms of both columns of
// a pair): every team lane loads its groups of both, one barrier, then both
// are transformed and stored - half the barriers of two separate passes and
// twice the independent work between them.
template <int R, int MPL, int TW>
__device__ __forceinline__ void stockham_pass_inplace2(float2* bufa, float2* bufb, int m, int ns,
                                                       const float2* twp, const Team& tm) {
  constexpr int TL = 32 * TW;
  constexpr int GPL = (32 * MPL / R) >= TL ? (32 * MPL / R) / TL : 1;
  constexpr int PS = post_pad_shift(32 * MPL), PM = (1 << PS) - 1;
  const int groups = m / R;
  const int is = groups + (groups >> PS), os = ns + (ns >> PS);
  const bool strided = (groups & PM) == 0 && (ns == 1 || (ns & PM) == 0);
  float2 x[2][GPL][R];
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const float2* buf = b ? bufb : bufa;
#pragma unroll
    for (int t = 0; t < GPL; ++t) {
      const int j = tm.tl + TL * t;
      if (j < groups) {
        if (strided) {
          const float2* ip = buf + pidx(j, PS);
#pragma unroll
          for (int r = 0; r < R; ++r) x[b][t][r] = ip[r * is];
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) x[b][t][r] = buf[pidx(j + r * groups, PS)];
        }
      }
    }
  }
  team_sync<TW>(tm);
#pragma unroll
  for (int t = 0; t < GPL; ++t) {
    const int j = tm.tl + TL * t;
    if (j < groups) {
      const int k = j & (ns - 1);
      float2 w[R];
      if (ns > 1) twiddles<R>(twp, k, w);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        float2* buf = b ? bufb : bufa;
        if (ns > 1) {
#pragma unroll
          for (int r = 1; r < R; ++r) x[b][t][r] = cmul(x[b][t][r], w[r]);
        }
        dft_regs<R>(x[b][t]);
        if (strided) {
          float2* op = buf + pidx(base, PS);
#pragma unroll
          for (int r = 0; r < R; ++r) op[r * os] = x[b][t][r];
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) buf[pidx(base + r * ns, PS)] = x[b][t][r];
        }
      }
    }
  }
  team_sync<TW>(tm);
}

// ---- k_post_inplace: 64 <= M <= 1024, two M-point buffers per team ----
// Same algorithm as k_post below (pack two real columns, forward FFT, split
// the spectra with the conjugate symmetry, mask, conjugate, forward FFT of
// each half, modulus / M), arranged so that shared memory is crossed as few
// times as possible:
//   * the first radix-8 pass of the forward FFT reads its inputs straight
//     from the image columns (coalesced across the lanes);
//   * the spectrum split is fused into the first pass of both inverse
//     transforms (each input of that pass is formed from Z[n] and Z[M-n]);
//   * the last pass of each inverse transform writes the envelope straight
//     to the image.
// Every pass is a radix-8 Stockham pass except a final radix-4 / radix-2
// pass when log2 M is not a multiple of 3; the first pass (sub-transform
// length 1) needs no twiddles.

template <int MPL, int TW>
struct PostShape {
  static constexpr int M = 32 * MPL;
  static constexpr int LOG2 = MPL == 2 ? 6 : MPL == 4 ? 7 : MPL == 8 ? 8 : MPL == 16 ? 9 : 10;
  static constexpr int TL = 32 * TW;                    // team lanes
  // radix of the first pass: 16 for 1024 points (16 x 8 x 8: three passes
  // instead of four), else 8; the passes after it follow post_pass_radix
  static constexpr int R1 = post_first_radix(M);
  static constexpr int LR1 = R1 == 16 ? 4 : 3;
  static constexpr int G1 = M / R1;                     // groups of the first pass
  static constexpr int GPL = G1 >= TL ? G1 / TL : 1;    // groups per team lane
};

// First forward pass: x[r] = (a[n], b[n]), n = j + r M/8, zero past nz.
template <int MPL, int TW>
__device__ __forceinline__ void first_pass_from_columns(float2* A, const float* ca, const float* cb,
                                                        int nz, bool two, const Team& tm) {
  using S = PostShape<MPL, TW>;
  constexpr int PS = post_pad_shift(S::M);
#pragma unroll
  for (int t = 0; t < S::GPL; ++t) {
    const int j = tm.tl + S::TL * t;
    if (j >= S::G1) break;
    constexpr int R = S::R1;
    float2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int n = j + r * S::G1;
      const bool in = n < nz;
      x[r] = make_float2(in ? ca[n] : 0.f, (in && two) ? cb[n] : 0.f);
    }
    dft_any<R>(x);
    // outputs R j + r: pidx(R j + r) = pidx(R j) + r (R j is a multiple of
    // 2^PS, or of 8 with r < 8)
    float2* op = A + pidx(R * j, PS);
#pragma unroll
    for (int r = 0; r < R; ++r) op[r] = x[r];
  }
  team_sync<TW>(tm);
}

// Spectrum split fused into the first pass of both inverse transforms.
// Input n of the transform for column a is (h (Z[n] + conj Z[M-n]) / 2)*
// written out as below, for column b the same with -i; h = mask[n].  The
// column-b pass output goes to B at once (B is free); the column-a outputs
// wait in registers until every lane has read Z, then overwrite it in A.
template <int MPL, int TW>
__device__ __forceinline__ void split_first_pass(float2* A, float2* B, const float* mk,
                                                 const Team& tm) {
  using S = PostShape<MPL, TW>;
  constexpr int M = S::M, R = S::R1, PS = post_pad_shift(M);
  if constexpr (2 * S::G1 <= S::TL) {
    // fewer groups than half the team (1024 points: 64 radix-16 groups, 128
    // lanes): lanes below G1 transform column a, the next G1 lanes column b
    const bool colb = tm.tl >= S::G1;
    const int j = colb ? tm.tl - S::G1 : tm.tl;
    float2 x[R];
    if (j < S::G1) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int n = j + r * S::G1;
        const float2 zn = A[pidx(n, PS)], zm = A[pidx((M - n) & (M - 1), PS)];
        const float h = 0.5f * mk[n];
        x[r] = colb ? make_float2(h * (zn.y + zm.y), h * (zn.x - zm.x))
                    : make_float2(h * (zn.x + zm.x), -h * (zn.y - zm.y));
      }
      dft_any<R>(x);
      if (colb) {
        float2* op = B + pidx(R * j, PS);
#pragma unroll
        for (int r = 0; r < R; ++r) op[r] = x[r];
      }
    }
    team_sync<TW>(tm);  // every lane has read Z
    if (!colb && j < S::G1) {
      float2* op = A + pidx(R * j, PS);
#pragma unroll
      for (int r = 0; r < R; ++r) op[r] = x[r];
    }
    team_sync<TW>(tm);
    return;
  }
  float2 xa[S::GPL][R];
#pragma unroll
  for (int t = 0; t < S::GPL; ++t) {
    const int j = tm.tl + S::TL * t;
    if (j >= S::G1) break;
    float2 xb[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int n = j + r * S::G1;
      const float2 zn = A[pidx(n, PS)], zm = A[pidx((M - n) & (M - 1), PS)];
      const float h = 0.5f * mk[n];
      xa[t][r] = make_float2(h * (zn.x + zm.x), -h * (zn.y - zm.y));
      xb[r] = make_float2(h * (zn.y + zm.y), h * (zn.x - zm.x));
    }
    dft_any<R>(xb);
    float2* op = B + pidx(R * j, PS);
#pragma unroll
    for (int r = 0; r < R; ++r) op[r] = xb[r];
  }
  team_sync<TW>(tm);
#pragma unroll
  for (int t = 0; t < S::GPL; ++t) {
    const int j = tm.tl + S::TL * t;
    if (j >= S::G1) break;
    dft_any<R>(xa[t]);
    float2* op = A + pidx(R * j, PS);
#pragma unroll
    for (int r = 0; r < R; ++r) op[r] = xa[t][r];
  }
  team_sync<TW>(tm);
}

// Last pass (sub-transform length ns = M / R, so group j has k = j and its
// outputs land at j + r ns in natural order): modulus / M straight to the
// column, folded into the column maximum.
template <int R, int MPL, int TW>
__device__ __forceinline__ void last_pass_to_column(const float2* buf, const float2* twp, float* col,
                                                    int nz, float inv_m, float& mx, const Team& tm) {
  constexpr int M = 32 * MPL, ns = M / R, groups = M / R, TL = 32 * TW;
  constexpr int PS = post_pad_shift(M);
  constexpr bool strided = (groups & ((1 << PS) - 1)) == 0;
  constexpr int is = groups + (groups >> PS);
#pragma unroll
  for (int t = 0; t < (groups + TL - 1) / TL; ++t) {
    const int j = tm.tl + TL * t;
    if (j >= groups) break;
    float2 x[R];
    if constexpr (strided) {
      const float2* ip = buf + pidx(j, PS);
#pragma unroll
      for (int r = 0; r < R; ++r) x[r] = ip[r * is];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) x[r] = buf[pidx(j + r * groups, PS)];
    }
    float2 w[R];
    twiddles<R>(twp, j, w);
#pragma unroll
    for (int r = 1; r < R; ++r) x[r] = cmul(x[r], w[r]);
    dft_regs<R>(x);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int n = j + r * ns;
      const float e = sqrtf(x[r].x * x[r].x + x[r].y * x[r].y) * inv_m;
      if (n < nz) {
        col[n] = e;
        mx = fmaxf(mx, e);
      }
    }
  }
}

// Last pass of both inverse transforms: envelopes of columns a and b (b only
// when the pair has two columns).
template <int R, int MPL, int TW>
__device__ __forceinline__ void last_pass_to_columns2(const float2* bufa, const float2* bufb,
                                                      const float2* twp, float* cola, float* colb,
                                                      int nz, float inv_m, float& mx,
                                                      const Team& tm) {
  constexpr int M = 32 * MPL, ns = M / R, groups = M / R, TL = 32 * TW;
  constexpr int PS = post_pad_shift(M);
  constexpr bool strided = (groups & ((1 << PS) - 1)) == 0;
  constexpr int is = groups + (groups >> PS);
#pragma unroll
  for (int t = 0; t < (groups + TL - 1) / TL; ++t) {
    const int j = tm.tl + TL * t;
    if (j >= groups) break;
    float2 x[2][R];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const float2* buf = b ? bufb : bufa;
      if constexpr (strided) {
        const float2* ip = buf + pidx(j, PS);
#pragma unroll
        for (int r = 0; r < R; ++r) x[b][r] = ip[r * is];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) x[b][r] = buf[pidx(j + r * groups, PS)];
      }
    }
    float2 w[R];
    twiddles<R>(twp, j, w);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
#pragma unroll
      for (int r = 1; r < R; ++r) x[b][r] = cmul(x[b][r], w[r]);
      dft_regs<R>(x[b]);
      float* col = b ? colb : cola;
      if (!col) continue;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int n = j + r * ns;
        const float e = sqrtf(x[b][r].x * x[b][r].x + x[b][r].y * x[b][r].y) * inv_m;
        if (n < nz) {
          col[n] = e;
          mx = fmaxf(mx, e);
        }
      }
    }
  }
}

// The inverse transforms of both columns after their fused first pass, pass
// by pass together, the last pass writing both envelopes (colb null: the
// pair's second column lies outside the image).
template <int MPL, int TW>
__device__ __forceinline__ void rest_passes2(float2* bufa, float2* bufb, const float2* tw,
                                             float* cola, float* colb, int nz, float inv_m,
                                             float& mx, const Team& tm) {
  constexpr int M = 32 * MPL;
  using S = PostShape<MPL, TW>;
  int ns = S::R1, rem = S::LOG2 - S::LR1;
  const float2* twp = tw;
  while (rem > 0) {
    const int lr = rem >= 3 ? 3 : rem;
    if (lr == rem) {
      if (lr == 3) last_pass_to_columns2<8, MPL, TW>(bufa, bufb, twp, cola, colb, nz, inv_m, mx, tm);
      else if (lr == 2) last_pass_to_columns2<4, MPL, TW>(bufa, bufb, twp, cola, colb, nz, inv_m, mx, tm);
      else last_pass_to_columns2<2, MPL, TW>(bufa, bufb, twp, cola, colb, nz, inv_m, mx, tm);
      return;
    }
    if (lr == 3) stockham_pass_inplace2<8, MPL, TW>(bufa, bufb, M, ns, twp, tm);
    else if (lr == 2) stockham_pass_inplace2<4, MPL, TW>(bufa, bufb, M, ns, twp, tm);
    else stockham_pass_inplace2<2, MPL, TW>(bufa, bufb, M, ns, twp, tm);
    twp += ns * ((1 << lr) - 1);
    ns <<= lr;
    rem -= lr;
  }
}

// Passes after the first (twiddle blocks from the second pass on), the last
// one writing the envelope; to_column = false keeps every pass in shared
// memory (the forward transform).
template <int MPL, int TW>
__device__ __forceinline__ void rest_passes(float2* buf, const float2* tw, bool to_column,
                                            float* col, int nz, float inv_m, float& mx,
                                            const Team& tm) {
  constexpr int M = 32 * MPL;
  using S = PostShape<MPL, TW>;
  int ns = S::R1, rem = S::LOG2 - S::LR1;
  const float2* twp = tw;
  while (rem > 0) {
    const int lr = rem >= 3 ? 3 : rem;
    if (to_column && lr == rem) {
      if (lr == 3) last_pass_to_column<8, MPL, TW>(buf, twp, col, nz, inv_m, mx, tm);
      else if (lr == 2) last_pass_to_column<4, MPL, TW>(buf, twp, col, nz, inv_m, mx, tm);
      else last_pass_to_column<2, MPL, TW>(buf, twp, col, nz, inv_m, mx, tm);
      return;
    }
    if (lr == 3) stockham_pass_inplace<8, MPL, TW>(buf, M, ns, twp, tm);
    else if (lr == 2) stockham_pass_inplace<4, MPL, TW>(buf, M, ns, twp, tm);
    else stockham_pass_inplace<2, MPL, TW>(buf, M, ns, twp, tm);
    twp += ns * ((1 << lr) - 1);
    ns <<= lr;
    rem -= lr;
  }
}

template <int MPL, int TW>
__global__ void __launch_bounds__(256) k_post_inplace(const PostParams p) {
  extern __shared__ __align__(16) float2 sbuf[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int M = 32 * MPL;
  constexpr int MP = post_padded_len(M);
  float2* tw = sbuf;  // p.n_tw per-pass twiddles, then the mask, then buffers
  float* mk = reinterpret_cast<float*>(sbuf + p.n_tw);
  for (int k = threadIdx.x; k < p.n_tw; k += blockDim.x) tw[k] = __ldg(p.tw + k);
  for (int k = threadIdx.x; k < M; k += blockDim.x) mk[k] = __ldg(p.mask + (size_t)blockIdx.y * M + k);
  __syncthreads();
  const Team tm{(warp % TW) * 32 + lane, warp / TW};
  const int teams = p.warps_per_block / TW;
  const int j0 = 2 * (blockIdx.x * teams + tm.id);
  const int o = blockIdx.y, f = blockIdx.z;
  if (j0 >= p.nx) return;  // the whole team leaves; no block barrier below
  const bool two = j0 + 1 < p.nx;
  float2* A = sbuf + p.n_tw + M / 2 + (size_t)tm.id * 2 * MP;
  float2* B = A + MP;
  const size_t plane = (size_t)p.nx * p.nz;
  const float* src = p.out + ((size_t)f * p.planes + (size_t)p.s_src * p.n_out + o) * plane +
                     (size_t)j0 * p.nz;
  float* dst = p.out + ((size_t)f * p.planes + (size_t)p.s_dst * p.n_out + o) * plane +
               (size_t)j0 * p.nz;
  // forward transform of a + i b
  first_pass_from_columns<MPL, TW>(A, src, src + p.nz, p.nz, two, tm);
  float mx = 0.f;
  rest_passes<MPL, TW>(A, tw, false, nullptr, 0, 0.f, mx, tm);
  // split + masks, first inverse pass of both columns
  split_first_pass<MPL, TW>(A, B, mk, tm);
  const float inv_m = 1.0f / (float)M;
  if constexpr (M == 1024) {
    // both inverse transforms pass by pass together (registers stay at the
    // kernel's 80; at 512 points they rose from 64 to 78, a block per SM)
    rest_passes2<MPL, TW>(A, B, tw, dst, two ? dst + p.nz : nullptr, p.nz, inv_m, mx, tm);
  } else {
    rest_passes<MPL, TW>(A, tw, true, dst, p.nz, inv_m, mx, tm);
    if (two) rest_passes<MPL, TW>(B, tw, true, dst + p.nz, p.nz, inv_m, mx, tm);
  }
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, s));
  if (lane == 0) atomicMax(p.maxslot + (size_t)f * p.n_out + o, __float_as_int(mx));
}

// Shared memory: the M-entry twiddle table, then three M-point complex
// buffers per warp.
__global__ void __launch_bounds__(256) k_post(const PostParams p) {
  extern __shared__ __align__(16) float2 sbuf[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int M = p.m;
  const int ps = post_pad_shift(M);
  const int MP = post_padded_len(M);  // padded buffer length
  float2* tw = sbuf;  // p.n_tw per-pass twiddles, then the buffers
  for (int k = threadIdx.x; k < p.n_tw; k += blockDim.x) tw[k] = __ldg(p.tw + k);
  __syncthreads();
  const int j0 = 2 * (blockIdx.x * p.warps_per_block + warp);
  const int o = blockIdx.y, f = blockIdx.z;
  if (j0 >= p.nx) return;  // no block barrier below
  const bool two = j0 + 1 < p.nx;
  float2* b0 = sbuf + p.n_tw + (size_t)warp * 3 * MP;
  float2* b1 = b0 + MP;
  float2* b2 = b1 + MP;
  const size_t plane = (size_t)p.nx * p.nz;
  const float* src = p.out + ((size_t)f * p.planes + (size_t)p.s_src * p.n_out + o) * plane +
                     (size_t)j0 * p.nz;
  float* dst = p.out + ((size_t)f * p.planes + (size_t)p.s_dst * p.n_out + o) * plane +
               (size_t)j0 * p.nz;
  const bool vec = (p.nz & 3) == 0;  // column starts 16-byte aligned

  if (vec) {
    for (int n = 4 * lane; n < M; n += 128) {
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
      if (n < p.nz) {
        a = *reinterpret_cast<const float4*>(src + n);
        if (two) b = *reinterpret_cast<const float4*>(src + p.nz + n);
      }
      b0[pidx(n, ps)] = make_float2(a.x, b.x);
      b0[pidx(n + 1, ps)] = make_float2(a.y, b.y);
      b0[pidx(n + 2, ps)] = make_float2(a.z, b.z);
      b0[pidx(n + 3, ps)] = make_float2(a.w, b.w);
    }
  } else {
    for (int n = lane; n < M; n += 32) {
      const bool in_col = n < p.nz;
      const float a = in_col ? src[n] : 0.f;
      const float b = (in_col && two) ? src[p.nz + n] : 0.f;
      b0[pidx(n, ps)] = make_float2(a, b);
    }
  }
  __syncwarp();
  float2* Z = fft_forward(b0, b1, M, p.log2m, tw, lane, ps);
  float2* F = (Z == b0) ? b1 : b0;  // free buffer

  // Split the packed spectrum and apply the mask.  Bins k and M-k are handled
  // by the same lane, so conj(H B) can overwrite Z in place; conj(H A) goes
  // to b2.  H vanishes above M/2.
  const float* mk = p.mask + (size_t)o * M;
  const int half = M >> 1;
  for (int k = lane; k <= half; k += 32) {
    const int km = (M - k) & (M - 1);
    const float2 z = Z[pidx(k, ps)], zc = Z[pidx(km, ps)];
    const float hk = 0.5f * __ldg(mk + k);
    // A[k] = (z + conj zc) / 2,  B[k] = (z - conj zc) / (2i)
    b2[pidx(k, ps)] = make_float2(hk * (z.x + zc.x), -hk * (z.y - zc.y));
    Z[pidx(k, ps)] = make_float2(hk * (z.y + zc.y), hk * (z.x - zc.x));
    if (km != k) {
      const float hm = 0.5f * __ldg(mk + km);  // zero for km > M/2
      b2[pidx(km, ps)] = make_float2(hm * (zc.x + z.x), -hm * (zc.y - z.y));
      Z[pidx(km, ps)] = make_float2(hm * (zc.y + z.y), hm * (zc.x - z.x));
    }
  }
  __syncwarp();
  const float inv_m = 1.0f / (float)M;
  const float2* Ya = fft_forward(b2, F, M, p.log2m, tw, lane, ps);
  float mx = 0.f;
  auto emit = [&](const float2* Y, float* col) {
    if (vec) {
      for (int n = 4 * lane; n < p.nz; n += 128) {
        float e[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const float2 y = Y[pidx(n + t, ps)];
          e[t] = sqrtf(y.x * y.x + y.y * y.y) * inv_m;
          mx = fmaxf(mx, e[t]);
        }
        *reinterpret_cast<float4*>(col + n) = make_float4(e[0], e[1], e[2], e[3]);
      }
    } else {
      for (int n = lane; n < p.nz; n += 32) {
        const float2 y = Y[pidx(n, ps)];
        const float env = sqrtf(y.x * y.x + y.y * y.y) * inv_m;
        col[n] = env;
        mx = fmaxf(mx, env);
      }
    }
  };
  emit(Ya, dst);
  if (two) {
    __syncwarp();
    // Ya lives in b2 or F; the FFT of the B half ping-pongs between Z and the
    // buffer Ya does not use.
    float2* G = (Ya == b2) ? F : b2;
    emit(fft_forward(Z, G, M, p.log2m, tw, lane, ps), dst + p.nz);
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
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if ((p.plane_elems & 3) == 0) {  // planes start 16-byte aligned
    const long long n4 = p.plane_elems >> 2;
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    // two loads in flight per thread before either result is stored
    for (long long q = t0; q < n4; q += 2 * stride) {
      const long long q1 = q + stride;
      const float4 e = s4[q];
      const float4 e1 = q1 < n4 ? s4[q1] : e;
      d4[q] = make_float4(log_db(e.x, mx, inv, dr), log_db(e.y, mx, inv, dr),
                          log_db(e.z, mx, inv, dr), log_db(e.w, mx, inv, dr));
      if (q1 < n4)
        d4[q1] = make_float4(log_db(e1.x, mx, inv, dr), log_db(e1.y, mx, inv, dr),
                             log_db(e1.z, mx, inv, dr), log_db(e1.w, mx, inv, dr));
    }
  } else {
    for (long long q = t0; q < p.plane_elems; q += stride) dst[q] = log_db(src[q], mx, inv, dr);
  }
}

const void* post_inplace_func(int m);

cudaError_t post_configure(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k_post, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  for (int m = 64; m <= 1024 && e == cudaSuccess; m *= 2)
    e = cudaFuncSetAttribute(post_inplace_func(m), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
  return e;
}

const void* post_inplace_func(int m) {
  switch (m) {
    case 64: return reinterpret_cast<const void*>(k_post_inplace<2, 1>);
    case 128: return reinterpret_cast<const void*>(k_post_inplace<4, 1>);
    case 256: return reinterpret_cast<const void*>(k_post_inplace<8, 2>);
    case 512: return reinterpret_cast<const void*>(k_post_inplace<16, 2>);
    case 1024: return reinterpret_cast<const void*>(k_post_inplace<32, 4>);
  }
  return nullptr;
}

int post_buffers(int m) { return post_inplace_func(m) ? 2 : 3; }

// Warps per team (one packed column pair) of the in-place kernel: one up to
// 128 points, two for 256 and 512 (one radix-8 group per lane), four for
// 1024 (measured: 1.18 -> 1.07 ms per 192 cfg5 images against two); one for
// the fallback kernel.
int post_team_warps(int m) {
  if (!post_inplace_func(m) || m < 256) return 1;
  return m == 1024 ? 4 : 2;
}

void post_spec(const PostParams& p, LaunchSpec* ls) {
  const size_t mp = (size_t)post_padded_len(p.m);
  const void* f = post_inplace_func(p.m);
  ls->func = f ? f : reinterpret_cast<const void*>(k_post);
  // in place: two buffers per team of post_team_warps warps; fallback: three
  // buffers per warp
  const int tw_warps = post_team_warps(p.m);
  const int teams = p.warps_per_block / tw_warps;
  ls->smem = ((size_t)teams * post_buffers(p.m) * mp + p.n_tw) * sizeof(float2) +
             (f ? (size_t)p.m * sizeof(float) : 0);
  const int col_pairs = (p.nx + 1) / 2;
  ls->grid = dim3((col_pairs + teams - 1) / teams, p.n_out, p.n_frames);
  ls->block = dim3(p.warps_per_block * 32);
}

void log_spec(const LogParams& p, int num_sms, LaunchSpec* ls) {
  long long blocks = (p.plane_elems / 4 + 255) / 256 + 1;
  const long long images = (long long)p.n_frames * p.n_out;
  const long long target = (long long)num_sms * 32;
  long long per_img = (target + images - 1) / images;
  if (per_img < 1) per_img = 1;
  if (blocks > per_img) blocks = per_img;
  ls->func = reinterpret_cast<const void*>(k_log);
  ls->grid = dim3((unsigned)blocks, (unsigned)images);
  ls->block = dim3(256);
  ls->smem = 0;
}

cudaError_t post_launch(const PostParams& p, cudaStream_t s) {
  LaunchSpec ls;
  post_spec(p, &ls);
  void* args[] = {const_cast<PostParams*>(&p)};
  return cudaLaunchKernel(ls.func, ls.grid, ls.block, args, ls.smem, s);
}

cudaError_t log_launch(const LogParams& p, int num_sms, cudaStream_t s) {
  LaunchSpec ls;
  log_spec(p, num_sms, &ls);
  k_log<<<ls.grid, ls.block, ls.smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace pa
