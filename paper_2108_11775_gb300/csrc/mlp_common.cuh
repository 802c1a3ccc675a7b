// The surrogate network's input encoding, shared by its training (mlp.cu) and
// inference (mlp_tc05.cu) kernels.
//
// u = (x - lo) s - 1 with the network's float32 lo and s (in_scale).  The
// encoding is [u_0..u_2, then for k = 0..5: sin(2^k pi u_j), cos(2^k pi u_j)],
// and sin(2^k pi u) = sin(2 pi tau), tau = 2^(k-1) ((x - lo) s - 1).  The
// product w = (x - lo) s is kept as w_hi + w_lo (an FMA gives the rounding
// error of the product exactly), 2^(k-1) w_hi - rint(2^(k-1) w_hi) is exact,
// and the - 2^(k-1) of the shift is an integer for k >= 1 (a half turn for
// k = 0): the only rounded steps left are the addition of the small w_lo term
// and the angle 2 pi r.  Without this, FP32's rounding of u (about 1e-7) would
// reach the k = 5 features multiplied by 32 pi.
#pragma once

#include "common.cuh"

namespace pdmp {

struct MlpEncIn {
  float whi[3], wlo[3];
};

__device__ __forceinline__ void mlp_enc_prepare(const float* x, const float* lo, const float* s, MlpEncIn& e) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float d = x[j] - lo[j];
    e.whi[j] = d * s[j];
    e.wlo[j] = fmaf(d, s[j], -e.whi[j]);
  }
}

// feature f (0 .. 38) of the encoding; 0 past the end (padding)
template <bool PRECISE>
__device__ __forceinline__ float mlp_enc_feature(int f, const MlpEncIn& e) {
  if (f >= 39) return 0.0f;
  if (f < 3) return (e.whi[f] - 1.0f) + e.wlo[f];
  const int k = (f - 3) / 6, m = (f - 3) % 6, j = m % 3;
  const float sc = 0.5f * (float)(1 << k);               // 2^(k-1), exact
  const float th_ = e.whi[j] * sc;
  float r = (th_ - rintf(th_)) + e.wlo[j] * sc;
  if (k == 0) r -= 0.5f;
  r -= rintf(r);                                        // [-1/2, 1/2] turn
  const float th = 6.28318530717958648f * r;
  if constexpr (PRECISE) return m < 3 ? sinf(th) : cosf(th);
  return m < 3 ? sin_approx(th) : cos_approx(th);
}

}  // namespace pdmp
