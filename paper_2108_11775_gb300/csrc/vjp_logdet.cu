// Differentiation through the Euler chain of Eq. (1):
//   * VJP   g_t = (I - eta Hess c(x_t)) g_{t+1}   (Hess c symmetric), with the
//           optional weight / bias gradient of sum_n <gT[n], x_T[n]>;
//   * log-det  sum_t log det(I - eta Hess c(x_t)) by a d x d Cholesky.
// Hess c = sigma'(s) Hess s + sigma''(s) grad s grad s^T.
// One sample per thread; states inside a checkpoint segment are recomputed
// into thread-local memory.
#include "field.cuh"
#include "kernels.cuh"

namespace pdmp {

constexpr int kVjpThreads = 128;
constexpr int kVjpTile = 128;

// -------------------------------------------------------------- forward step
template <int KIND, int D>
__device__ void grad_pass(const FieldArgs& fa, float ngl2e, const float* x, float* sm, float& s_out,
                          float* grad_s) {
  constexpr int R = RecLayout<D>::kFloats;
  float s = 0.0f, gs[D];
#pragma unroll
  for (int j = 0; j < D; ++j) gs[j] = 0.0f;
  for (int64_t m0 = 0; m0 < fa.M; m0 += kVjpTile) {
    __syncthreads();
    stage_tile<KIND, D>(fa, m0, kVjpTile, sm);
    __syncthreads();
    const int cnt = (int)min64(kVjpTile, fa.M - m0);
    for (int i = 0; i < cnt; ++i) {
      float rec[R];
      load_rec<D>(sm, i, rec);
      accum_grad<KIND, D>(rec, x, ngl2e, s, gs);
    }
  }
  s_out = s + fa.bias;
  finish_grad_s<KIND, D>(gs, fa.gamma, grad_s);
}

template <int KIND, int D>
__device__ __forceinline__ void euler_step(const FieldArgs& fa, float ngl2e, float eta, float* x, float* sm) {
  float s, g[D], d1, d2;
  grad_pass<KIND, D>(fa, ngl2e, x, sm, s, g);
  sigmoid_d12(s, d1, d2);
  // same rounding as the morph kernel: the increment is rounded, then added
  const float c = -eta * d1;
#pragma unroll
  for (int j = 0; j < D; ++j) x[j] = __fadd_rn(x[j], __fmul_rn(c, g[j]));
}

// ------------------------------------------------- Hessian-vector product pass
// Returns s (with bias), grad s and (Hess s) v at x.
//   RBF: Hess s v = 4 gamma^2 sum w phi (r.v) r - 2 gamma (sum w phi) v,  r = x - mu
//   RFF: Hess s v = -sum w cos(theta) (omega.v) omega
template <int KIND, int D>
__device__ void hvp_pass(const FieldArgs& fa, float ngl2e, const float* x, const float* v, float* sm, float& s_out,
                         float* grad_s, float* hsv) {
  constexpr int R = RecLayout<D>::kFloats;
  float s = 0.0f, G[D], P[D];
#pragma unroll
  for (int j = 0; j < D; ++j) { G[j] = 0.0f; P[j] = 0.0f; }
  for (int64_t m0 = 0; m0 < fa.M; m0 += kVjpTile) {
    __syncthreads();
    stage_tile<KIND, D>(fa, m0, kVjpTile, sm);
    __syncthreads();
    const int cnt = (int)min64(kVjpTile, fa.M - m0);
    for (int i = 0; i < cnt; ++i) {
      float rec[R];
      load_rec<D>(sm, i, rec);
      if (KIND == PDMP_KIND_RBF) {
        float dx[D], r2 = 0.0f, rv = 0.0f;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          dx[j] = x[j] - rec[j];
          r2 = fmaf(dx[j], dx[j], r2);
          rv = fmaf(dx[j], v[j], rv);
        }
        float we = rec[D + 1] * ex2_approx(fmaf(r2, ngl2e, rec[D]));
        s += we;
        float wrv = we * rv;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          G[j] = fmaf(we, dx[j], G[j]);
          P[j] = fmaf(wrv, dx[j], P[j]);
        }
      } else {
        float th = rec[D], ov = 0.0f;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          th = fmaf(rec[j], x[j], th);
          ov = fmaf(rec[j], v[j], ov);
        }
        th = reduce_2pi(th);
        float wc = rec[D + 1] * cos_approx(th);
        float ws = rec[D + 1] * sin_approx(th);
        s += wc;
        float q = wc * ov;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          G[j] = fmaf(-ws, rec[j], G[j]);
          P[j] = fmaf(-q, rec[j], P[j]);
        }
      }
    }
  }
  if (KIND == PDMP_KIND_RBF) {
    const float g2 = 2.0f * fa.gamma, g4 = 4.0f * fa.gamma * fa.gamma;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      grad_s[j] = -g2 * G[j];
      hsv[j] = g4 * P[j] - g2 * s * v[j];
    }
  } else {
#pragma unroll
    for (int j = 0; j < D; ++j) { grad_s[j] = G[j]; hsv[j] = P[j]; }
  }
  s_out = s + fa.bias;
}

// ------------------------------------------ weight-gradient pass (optional)
// Adds, for every feature m, the block's sum over its samples of
//   -eta (sigma''(s) phi_m (grad s . g) + sigma'(s) (grad phi_m . g))
// to row[m] (this block's row of the workspace; no other block touches it).
template <int KIND, int D>
__device__ void weight_grad_pass(const FieldArgs& fa, float ngl2e, const float* x, const float* g, float a_coef,
                                 float b_coef, bool active, float* sm, float* red, float* row) {
  // a_coef = -eta sigma'' (grad s . g), b_coef = -eta sigma'
  constexpr int R = RecLayout<D>::kFloats;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kWarps = kVjpThreads / 32;
  for (int64_t m0 = 0; m0 < fa.M; m0 += kVjpTile) {
    __syncthreads();
    stage_tile<KIND, D>(fa, m0, kVjpTile, sm);
    __syncthreads();
    const int cnt = (int)min64(kVjpTile, fa.M - m0);
    for (int i = 0; i < cnt; ++i) {
      float rec[R];
      load_rec<D>(sm, i, rec);
      float contrib = 0.0f;
      if (active) {
        float phi, dphig;
        if (KIND == PDMP_KIND_RBF) {
          float r2 = 0.0f, rg = 0.0f;
#pragma unroll
          for (int j = 0; j < D; ++j) {
            float dx = x[j] - rec[j];
            r2 = fmaf(dx, dx, r2);
            rg = fmaf(dx, g[j], rg);
          }
          phi = ex2_approx(r2 * ngl2e);
          dphig = -2.0f * fa.gamma * phi * rg;
        } else {
          float th = rec[D], og = 0.0f;
#pragma unroll
          for (int j = 0; j < D; ++j) {
            th = fmaf(rec[j], x[j], th);
            og = fmaf(rec[j], g[j], og);
          }
          th = reduce_2pi(th);
          phi = cos_approx(th);
          dphig = -sin_approx(th) * og;
        }
        contrib = fmaf(a_coef, phi, b_coef * dphig);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
      if (lane == 0) red[warp * kVjpTile + i] = contrib;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      float acc = 0.0f;
#pragma unroll
      for (int q = 0; q < kWarps; ++q) acc += red[q * kVjpTile + i];
      row[m0 + i] += acc;
    }
  }
}

// --------------------------------------------------------------------- VJP
template <int KIND, int D>
__global__ void __launch_bounds__(kVjpThreads)
k_morph_vjp(FieldArgs fa, const float* __restrict__ x0, int64_t N, int T, float eta, int kseg,
            const float* __restrict__ ckpt, const float* __restrict__ gT, float* __restrict__ g0,
            float* __restrict__ ws_rows /* nullptr or gridDim.x x (M + 1) */) {
  constexpr int R = RecLayout<D>::kFloats;
  __shared__ __align__(16) float sm[kVjpTile * R];
  __shared__ float red[(kVjpThreads / 32) * kVjpTile];
  const float ngl2e = -fa.gamma * kLog2e;
  const int64_t n = (int64_t)blockIdx.x * kVjpThreads + threadIdx.x;
  const bool active = n < N;
  float* row = ws_rows ? ws_rows + (int64_t)blockIdx.x * (fa.M + 1) : nullptr;
  if (row)
    for (int64_t m = threadIdx.x; m <= fa.M; m += blockDim.x) row[m] = 0.0f;

  float g[D], xs[kMaxSegment][D];
#pragma unroll
  for (int j = 0; j < D; ++j) g[j] = active ? gT[n * D + j] : 0.0f;
  float gb = 0.0f;
  const int nseg = T / kseg;
  for (int sgi = nseg - 1; sgi >= 0; --sgi) {
    // state at the start of the segment
    float x[D];
    if (sgi == 0 || ckpt == nullptr) {
#pragma unroll
      for (int j = 0; j < D; ++j) x[j] = active ? x0[n * D + j] : 0.0f;
      for (int t = 0; t < sgi * kseg; ++t) euler_step<KIND, D>(fa, ngl2e, eta, x, sm);
    } else {
      const float* src = ckpt + (int64_t)(sgi - 1) * N * D;
#pragma unroll
      for (int j = 0; j < D; ++j) x[j] = active ? src[n * D + j] : 0.0f;
    }
    for (int i = 0; i < kseg; ++i) {
#pragma unroll
      for (int j = 0; j < D; ++j) xs[i][j] = x[j];
      if (i + 1 < kseg) euler_step<KIND, D>(fa, ngl2e, eta, x, sm);
    }
    for (int i = kseg - 1; i >= 0; --i) {
      float xi[D];
#pragma unroll
      for (int j = 0; j < D; ++j) xi[j] = xs[i][j];
      float s, gsv[D], hsv[D], d1, d2;
      hvp_pass<KIND, D>(fa, ngl2e, xi, g, sm, s, gsv, hsv);
      sigmoid_d12(s, d1, d2);
      float gdot = 0.0f;
#pragma unroll
      for (int j = 0; j < D; ++j) gdot = fmaf(gsv[j], g[j], gdot);
      if (row) {
        weight_grad_pass<KIND, D>(fa, ngl2e, xi, g, -eta * d2 * gdot, -eta * d1, active, sm, red, row);
        gb = fmaf(-eta * d2, gdot, gb);
      }
#pragma unroll
      for (int j = 0; j < D; ++j) g[j] = g[j] - eta * fmaf(d1, hsv[j], d2 * gdot * gsv[j]);
    }
  }
  if (active)
#pragma unroll
    for (int j = 0; j < D; ++j) g0[n * D + j] = g[j];
  if (row) {
    float v = active ? gb : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      float acc = 0.0f;
      for (int q = 0; q < kVjpThreads / 32; ++q) acc += red[q];
      row[fa.M] = acc;
    }
  }
}

// sums the per-block rows in block order: out[m] = sum_b rows[b][m], m <= M
__global__ void k_sum_rows(const float* __restrict__ rows, int64_t nrows, int64_t width, float* __restrict__ gw,
                           float* __restrict__ gbias) {
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= width) return;
  float acc = 0.0f;
  for (int64_t b = 0; b < nrows; ++b) acc += rows[b * width + m];
  if (m + 1 < width) {
    if (gw) gw[m] = acc;
  } else if (gbias) {
    *gbias = acc;
  }
}

cudaError_t sum_vjp_rows(const float* rows, int64_t nrows, int64_t width, float* gw, float* gbias, cudaStream_t st) {
  k_sum_rows<<<(unsigned)((width + 255) / 256), 256, 0, st>>>(rows, nrows, width, gw, gbias);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ log-det
// Cholesky of the SPD d x d matrix a (row-major, lower triangle used);
// returns sum log diag(L)^2, or NaN after raising the flag if a pivot <= 0.
template <int KIND, int D>
__global__ void __launch_bounds__(kVjpThreads)
k_logdet(FieldArgs fa, const float* __restrict__ x0, int64_t N, int T, float eta, float* __restrict__ logdet,
         float* __restrict__ xT) {
  constexpr int R = RecLayout<D>::kFloats;
  __shared__ __align__(16) float sm[kVjpTile * R];
  const float ngl2e = -fa.gamma * kLog2e;
  const int64_t n = (int64_t)blockIdx.x * kVjpThreads + threadIdx.x;
  const bool active = n < N;
  float x[D];
#pragma unroll
  for (int j = 0; j < D; ++j) x[j] = active ? x0[n * D + j] : 0.0f;
  float total = 0.0f;
  bool bad = false;
  for (int t = 0; t < T; ++t) {
    float s = 0.0f, G[D], Q[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      G[i] = 0.0f;
#pragma unroll
      for (int j = 0; j < D; ++j) Q[i][j] = 0.0f;
    }
    for (int64_t m0 = 0; m0 < fa.M; m0 += kVjpTile) {
      __syncthreads();
      stage_tile<KIND, D>(fa, m0, kVjpTile, sm);
      __syncthreads();
      const int cnt = (int)min64(kVjpTile, fa.M - m0);
      for (int i = 0; i < cnt; ++i) {
        float rec[R];
        load_rec<D>(sm, i, rec);
        if (KIND == PDMP_KIND_RBF) {
          float dx[D], r2 = 0.0f;
#pragma unroll
          for (int j = 0; j < D; ++j) {
            dx[j] = x[j] - rec[j];
            r2 = fmaf(dx[j], dx[j], r2);
          }
          float we = rec[D + 1] * ex2_approx(fmaf(r2, ngl2e, rec[D]));
          s += we;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            G[a] = fmaf(we, dx[a], G[a]);
            float wa = we * dx[a];
#pragma unroll
            for (int b = 0; b <= a; ++b) Q[a][b] = fmaf(wa, dx[b], Q[a][b]);
          }
        } else {
          float th = rec[D];
#pragma unroll
          for (int j = 0; j < D; ++j) th = fmaf(rec[j], x[j], th);
          th = reduce_2pi(th);
          float wc = rec[D + 1] * cos_approx(th);
          float ws = rec[D + 1] * sin_approx(th);
          s += wc;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            G[a] = fmaf(-ws, rec[a], G[a]);
            float wa = wc * rec[a];
#pragma unroll
            for (int b = 0; b <= a; ++b) Q[a][b] = fmaf(wa, rec[b], Q[a][b]);
          }
        }
      }
    }
    // grad s and Hess s (lower triangle)
    float gsv[D], H[D][D];
    if (KIND == PDMP_KIND_RBF) {
      const float g2 = 2.0f * fa.gamma, g4 = 4.0f * fa.gamma * fa.gamma;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        gsv[a] = -g2 * G[a];
#pragma unroll
        for (int b = 0; b <= a; ++b) H[a][b] = g4 * Q[a][b] - (a == b ? g2 * s : 0.0f);
      }
    } else {
#pragma unroll
      for (int a = 0; a < D; ++a) {
        gsv[a] = G[a];
#pragma unroll
        for (int b = 0; b <= a; ++b) H[a][b] = -Q[a][b];
      }
    }
    float d1, d2;
    sigmoid_d12(s + fa.bias, d1, d2);
    float A[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) {
        if (b <= a) {
          float hc = fmaf(d1, H[a][b], d2 * gsv[a] * gsv[b]);
          A[a][b] = (a == b ? 1.0f : 0.0f) - eta * hc;
        } else {
          A[a][b] = 0.0f;
        }
      }
    float ld = chol_logdet<D>(A);
    if (!(ld == ld)) bad = true;
    total += ld;
    const float c = -eta * d1;
#pragma unroll
    for (int j = 0; j < D; ++j) x[j] = __fadd_rn(x[j], __fmul_rn(c, gsv[j]));
  }
  if (active) {
    if (bad) raise_flag(FLAG_NONPOSITIVE_PIVOT);
    logdet[n] = bad ? nanf("") : total;
    if (xT)
#pragma unroll
      for (int j = 0; j < D; ++j) xT[n * D + j] = x[j];
  }
}

// ---------------------------------------------------------------- launchers
template <int KIND, int D>
static cudaError_t launch_vjp(const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, int k,
                              const float* ckpt, const float* gT, float* g0, float* rows, float* gw, float* gbias,
                              cudaStream_t st) {
  int64_t blocks = (N + kVjpThreads - 1) / kVjpThreads;
  if (blocks == 0) {
    if (gw) cudaMemsetAsync(gw, 0, sizeof(float) * fa.M, st);
    if (gbias) cudaMemsetAsync(gbias, 0, sizeof(float), st);
    return cudaGetLastError();
  }
  k_morph_vjp<KIND, D><<<(unsigned)blocks, kVjpThreads, 0, st>>>(fa, x0, N, T, eta, k, ckpt, gT, g0, rows);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || rows == nullptr) return e;
  return sum_vjp_rows(rows, blocks, fa.M + 1, gw, gbias, st);
}

template <int KIND, int D>
static cudaError_t launch_logdet(const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* ld,
                                 float* xT, cudaStream_t st) {
  int64_t blocks = (N + kVjpThreads - 1) / kVjpThreads;
  if (blocks == 0) return cudaSuccess;
  k_logdet<KIND, D><<<(unsigned)blocks, kVjpThreads, 0, st>>>(fa, x0, N, T, eta, ld, xT);
  return cudaGetLastError();
}

int64_t vjp_blocks(int64_t N) { return (N + kVjpThreads - 1) / kVjpThreads; }

#define PDMP_DISPATCH(FN, ...)                                                                         \
  do {                                                                                                 \
    if (kind == PDMP_KIND_RBF) {                                                                       \
      if (d == 1) return FN<PDMP_KIND_RBF, 1>(__VA_ARGS__);                                             \
      if (d == 2) return FN<PDMP_KIND_RBF, 2>(__VA_ARGS__);                                             \
      if (d == 3) return FN<PDMP_KIND_RBF, 3>(__VA_ARGS__);                                             \
    } else {                                                                                           \
      if (d == 1) return FN<PDMP_KIND_RFF, 1>(__VA_ARGS__);                                             \
      if (d == 2) return FN<PDMP_KIND_RFF, 2>(__VA_ARGS__);                                             \
      if (d == 3) return FN<PDMP_KIND_RFF, 3>(__VA_ARGS__);                                             \
      if (d == 4) return FN<PDMP_KIND_RFF, 4>(__VA_ARGS__);                                             \
      if (d == 5) return FN<PDMP_KIND_RFF, 5>(__VA_ARGS__);                                             \
      if (d == 6) return FN<PDMP_KIND_RFF, 6>(__VA_ARGS__);                                             \
      if (d == 7) return FN<PDMP_KIND_RFF, 7>(__VA_ARGS__);                                             \
      if (d == 8) return FN<PDMP_KIND_RFF, 8>(__VA_ARGS__);                                             \
    }                                                                                                  \
    return cudaErrorInvalidValue;                                                                      \
  } while (0)

cudaError_t morph_vjp(int kind, int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, int k,
                      const float* ckpt, const float* gT, float* g0, float* rows, float* gw, float* gbias,
                      cudaStream_t st) {
  PDMP_DISPATCH(launch_vjp, fa, x0, N, T, eta, k, ckpt, gT, g0, rows, gw, gbias, st);
}

cudaError_t logdet(int kind, int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* ld,
                   float* xT, void* ws, cudaStream_t st) {
  if (kind == PDMP_KIND_RFF && d <= 7 && ws != nullptr) return logdet_rff_mma(d, fa, x0, N, T, eta, ld, xT, ws, st);
  if (kind == PDMP_KIND_RBF && (d == 2 || d == 3) && ws != nullptr)
    return logdet_rbf_fast(d, fa, x0, N, T, eta, ld, xT, ws, st);
  if (kind == PDMP_KIND_RFF && d == 7) return logdet_rff7_mma(fa, x0, N, T, eta, ld, xT, st);
  PDMP_DISPATCH(launch_logdet, fa, x0, N, T, eta, ld, xT, st);
}

}  // namespace pdmp
