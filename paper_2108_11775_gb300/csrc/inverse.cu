// Inverse of the T-step map (Eq. 2): every Euler step x_{t+1} = x_t - eta grad c(x_t)
// is undone, last step first, by the fixed point y = z + eta grad c(y), which
// is a contraction with rate eta L < 1.  Each iteration is one pass over the
// features for the block's samples; a block stops when every sample's update
// is at most tol (relative to 1 + |y|) or after maxit iterations.
#include "field.cuh"
#include "kernels.cuh"

namespace pdmp {

constexpr int kInvThreads = 128;
constexpr int kInvTile = 256;

template <int KIND, int D, int K>
__global__ void __launch_bounds__(kInvThreads)
k_morph_inverse(FieldArgs fa, const float* __restrict__ z0, int64_t N, int T, float eta, float tol, int maxit,
                float* __restrict__ y_out, int32_t* __restrict__ iters) {
  constexpr int R = RecLayout<D>::kFloats;
  __shared__ __align__(16) float sm[kInvTile * R];
  const float ngl2e = -fa.gamma * kLog2e;
  const int64_t base = (int64_t)blockIdx.x * (kInvThreads * K) + threadIdx.x;
  float z[K][D], y[K][D];
  bool act[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int64_t n = base + (int64_t)k * kInvThreads;
    act[k] = n < N;
#pragma unroll
    for (int j = 0; j < D; ++j) z[k][j] = act[k] ? z0[n * D + j] : 0.0f;
  }
  int worst = 0;
  for (int t = T - 1; t >= 0; --t) {
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int j = 0; j < D; ++j) y[k][j] = z[k][j];
    int it = 0;
    for (; it < maxit; ++it) {
      float s[K], gs[K][D];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        s[k] = 0.0f;
#pragma unroll
        for (int j = 0; j < D; ++j) gs[k][j] = 0.0f;
      }
      for (int64_t m0 = 0; m0 < fa.M; m0 += kInvTile) {
        __syncthreads();
        stage_tile<KIND, D>(fa, m0, kInvTile, sm);
        __syncthreads();
        const int cnt = (int)min64(kInvTile, fa.M - m0);
        for (int i = 0; i < cnt; ++i) {
          float rec[R];
          load_rec<D>(sm, i, rec);
#pragma unroll
          for (int k = 0; k < K; ++k) accum_grad<KIND, D>(rec, y[k], ngl2e, s[k], gs[k]);
        }
      }
      bool moving = false;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        float d1, d2, g[D];
        sigmoid_d12(s[k] + fa.bias, d1, d2);
        finish_grad_s<KIND, D>(gs[k], fa.gamma, g);
        const float c = eta * d1;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          const float yn = fmaf(c, g[j], z[k][j]);
          if (act[k] && fabsf(yn - y[k][j]) > tol * (1.0f + fabsf(yn))) moving = true;
          y[k][j] = yn;
        }
      }
      if (!__syncthreads_or(moving)) {
        ++it;
        break;
      }
    }
    worst = it > worst ? it : worst;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int j = 0; j < D; ++j) z[k][j] = y[k][j];
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int64_t n = base + (int64_t)k * kInvThreads;
    if (!act[k]) continue;
#pragma unroll
    for (int j = 0; j < D; ++j) y_out[n * D + j] = z[k][j];
    if (iters) iters[n] = worst;
  }
}

template <int KIND, int D>
static cudaError_t launch_inverse(const FieldArgs& fa, const float* z, int64_t N, int T, float eta, float tol,
                                  int maxit, float* y, int32_t* iters, cudaStream_t st) {
  constexpr int K = 2;
  const int64_t per = (int64_t)kInvThreads * K;
  const int64_t blocks = (N + per - 1) / per;
  if (blocks == 0) return cudaSuccess;
  k_morph_inverse<KIND, D, K><<<(unsigned)blocks, kInvThreads, 0, st>>>(fa, z, N, T, eta, tol, maxit, y, iters);
  return cudaGetLastError();
}

cudaError_t morph_inverse(int kind, int d, const FieldArgs& fa, const float* z, int64_t N, int T, float eta,
                          float tol, int maxit, float* y, int32_t* iters, cudaStream_t st) {
#define PDMP_CASE(KD, DD) \
  if (kind == KD && d == DD) return launch_inverse<KD, DD>(fa, z, N, T, eta, tol, maxit, y, iters, st);
  PDMP_CASE(PDMP_KIND_RBF, 1) PDMP_CASE(PDMP_KIND_RBF, 2) PDMP_CASE(PDMP_KIND_RBF, 3)
  PDMP_CASE(PDMP_KIND_RFF, 1) PDMP_CASE(PDMP_KIND_RFF, 2) PDMP_CASE(PDMP_KIND_RFF, 3) PDMP_CASE(PDMP_KIND_RFF, 4)
  PDMP_CASE(PDMP_KIND_RFF, 5) PDMP_CASE(PDMP_KIND_RFF, 6) PDMP_CASE(PDMP_KIND_RFF, 7) PDMP_CASE(PDMP_KIND_RFF, 8)
#undef PDMP_CASE
  return cudaErrorInvalidValue;
}

// log p_z(z) = log p_0(y) - log det J(y) at y = phi^{-1}(z) (change of
// variables through the T-step map, Sec. 3.2 "Drawing Samples"), for a uniform
// base density on the box [lo, hi]: on entry lp holds log det J(y), on exit
// log p_z; outside the box the density is 0 (-inf).
struct BoxArgs {
  float lo[8], hi[8];
  float log_vol;
  int d;
};

__global__ void k_uniform_log_density(const float* __restrict__ y, int64_t N, BoxArgs b, float* __restrict__ lp) {
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    bool inside = true;
    for (int j = 0; j < b.d; ++j) {
      const float v = y[n * b.d + j];
      inside = inside && v >= b.lo[j] && v <= b.hi[j];
    }
    lp[n] = inside ? -b.log_vol - lp[n] : -INFINITY;
  }
}

cudaError_t uniform_log_density(const float* y, int64_t N, int d, const double* lo, const double* hi, float* lp,
                                cudaStream_t st) {
  BoxArgs b{};
  double lv = 0.0;
  for (int j = 0; j < d; ++j) {
    b.lo[j] = (float)lo[j];
    b.hi[j] = (float)hi[j];
    lv += log(hi[j] - lo[j]);
  }
  b.log_vol = (float)lv;
  b.d = d;
  const int64_t blocks = min64((N + 255) / 256, 152 * 8);
  k_uniform_log_density<<<(unsigned)blocks, 256, 0, st>>>(y, N, b, lp);
  return cudaGetLastError();
}

}  // namespace pdmp
