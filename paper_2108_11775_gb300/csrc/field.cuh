// Field records staged in shared memory, and the per-feature arithmetic of
// the occupancy logit s(x) = sum_m w_m phi_m(x) + bias (Sec. 3.1) and of its
// first and second input derivatives.
#pragma once
#include "common.cuh"

namespace pdmp {

// A staged feature record is D + 2 floats:
//   RBF: mu_0 .. mu_{D-1}, lw = log2|w| (-inf when w = 0), sg = sign(w) (0 when w = 0)
//   RFF: omega_0 .. omega_{D-1}, b, w
// Records past M are zero-weight padding (RBF: lw = -inf, sg = 0; RFF: w = 0),
// whose contributions are exactly zero.
template <int D>
struct RecLayout {
  static constexpr int kUsed = D + 2;                    // floats that carry data
  static constexpr int kFloats = (kUsed + 3) / 4 * 4;    // padded to whole float4s
};

// Copies staged record i (kFloats floats, 16-byte aligned) into registers
// with 128-bit shared-memory loads.
template <int D>
__device__ __forceinline__ void load_rec(const float* sm, int i, float* rec) {
  constexpr int R = RecLayout<D>::kFloats;
  const float4* q = reinterpret_cast<const float4*>(sm + i * R);
#pragma unroll
  for (int v = 0; v < R / 4; ++v) {
    const float4 t = q[v];
    rec[4 * v] = t.x;
    rec[4 * v + 1] = t.y;
    rec[4 * v + 2] = t.z;
    rec[4 * v + 3] = t.w;
  }
}

struct FieldArgs {
  const float* centres;
  const float* phase;
  const float* w;
  int64_t M;
  float gamma;
  float bias;
};

// Stages records [m0, m0 + tile) into smem (tile * (D + 2) floats), all
// threads of the block cooperating; the caller synchronises around it.
template <int KIND, int D>
__device__ __forceinline__ void stage_tile(const FieldArgs& fa, int64_t m0, int tile, float* sm) {
  constexpr int R = RecLayout<D>::kFloats;
  for (int i = threadIdx.x; i < tile; i += blockDim.x) {
    int64_t m = m0 + i;
    float* r = sm + i * R;
    if (m < fa.M) {
#pragma unroll
      for (int j = 0; j < D; ++j) r[j] = __ldg(fa.centres + m * D + j);
      float wm = __ldg(fa.w + m);
      if (KIND == PDMP_KIND_RBF) {
        r[D] = wm != 0.0f ? log2f(fabsf(wm)) : -INFINITY;
        r[D + 1] = wm > 0.0f ? 1.0f : (wm < 0.0f ? -1.0f : 0.0f);
      } else {
        r[D] = __ldg(fa.phase + m);
        r[D + 1] = wm;
      }
    } else {
#pragma unroll
      for (int j = 0; j < D; ++j) r[j] = 0.0f;
      r[D] = KIND == PDMP_KIND_RBF ? -INFINITY : 0.0f;
      r[D + 1] = 0.0f;
    }
#pragma unroll
    for (int j = D + 2; j < R; ++j) r[j] = 0.0f;
  }
}

// Accumulates one feature's contribution to s (without bias) and to
// gs = (RBF) sum_m w_m phi_m (x - mu_m)      [grad s = -2 gamma gs]
//      (RFF) sum_m -w_m sin(theta_m) omega_m [grad s = gs]
// ngl2e = -gamma * log2(e).
template <int KIND, int D>
__device__ __forceinline__ void accum_grad(const float* rec, const float* x, float ngl2e, float& s, float* gs) {
  if (KIND == PDMP_KIND_RBF) {
    float dx[D];
    float r2 = 0.0f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      dx[j] = x[j] - rec[j];
      r2 = fmaf(dx[j], dx[j], r2);
    }
    float e = ex2_approx(fmaf(r2, ngl2e, rec[D]));
    float we = __fmul_rn(rec[D + 1], e);   // explicit roundings: no contraction,
    s = __fadd_rn(s, we);                  // so every kernel rounds alike
#pragma unroll
    for (int j = 0; j < D; ++j) gs[j] = fmaf(we, dx[j], gs[j]);
  } else {
    float th = rec[D];
#pragma unroll
    for (int j = 0; j < D; ++j) th = fmaf(rec[j], x[j], th);
    th = reduce_2pi(th);
    float wc = __fmul_rn(rec[D + 1], cos_approx(th));
    float ws = __fmul_rn(rec[D + 1], sin_approx(th));
    s = __fadd_rn(s, wc);
#pragma unroll
    for (int j = 0; j < D; ++j) gs[j] = fmaf(-ws, rec[j], gs[j]);
  }
}

// Converts accumulated (s, gs) to grad s.
template <int KIND, int D>
__device__ __forceinline__ void finish_grad_s(const float* gs, float gamma, float* grad_s) {
#pragma unroll
  for (int j = 0; j < D; ++j) grad_s[j] = KIND == PDMP_KIND_RBF ? -2.0f * gamma * gs[j] : gs[j];
}

// log det of the symmetric positive definite D x D matrix whose lower
// triangle is in a (overwritten by its Cholesky factor); NaN when a pivot is
// not positive
template <int D>
__device__ __forceinline__ float chol_logdet(float (&a)[D][D]) {
  float acc = 0.0f;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    float p = a[j][j];
#pragma unroll
    for (int q = 0; q < j; ++q) p = fmaf(-a[j][q], a[j][q], p);
    if (!(p > 0.0f)) return nanf("");
    float l = sqrtf(p), inv = 1.0f / l;
    a[j][j] = l;
    acc += logf(p);
#pragma unroll
    for (int i = j + 1; i < D; ++i) {
      float v = a[i][j];
#pragma unroll
      for (int q = 0; q < j; ++q) v = fmaf(-a[i][q], a[j][q], v);
      a[i][j] = v * inv;
    }
  }
  return acc;
}

}  // namespace pdmp
