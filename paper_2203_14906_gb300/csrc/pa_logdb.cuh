// pa_logdb.cuh -- log compression of one envelope sample (display stage of
// the pipeline): 20 log10(env / image max), clipped to [-dr, 0]; -dr where
// the envelope or the image maximum is 0.
#pragma once

namespace pa {

// 20 log10(x) = (20 / log2 10) log2(x), log2 by the hardware approximation
// (absolute error about 2^-22 in log2, ~1e-6 dB; denormal ratios flush to
// zero and clip to -dr like any ratio below -dr).
__device__ __forceinline__ float log_db(float env, float mx, float inv, float dr) {
  float l2;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l2) : "f"(env * inv));
  return (mx > 0.f && env > 0.f) ? fminf(0.f, fmaxf(-dr, 6.0205999132796239f * l2)) : -dr;
}

}  // namespace pa
