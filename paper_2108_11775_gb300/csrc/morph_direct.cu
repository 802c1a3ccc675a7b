// Direct-form morph kernel: T Euler steps of Eq. (1),
//   x_{t+1} = x_t - eta * sigmoid'(s(x_t)) * grad s(x_t),
// for any field kind and dimension the library supports.  Each thread keeps
// K samples in registers for all T steps; the block streams the feature
// records through shared memory in tiles every step.
//
// This is the general path (any d, any sample layout).  The 2-D / 3-D RBF
// fast path lives in morph_rbf_fast.cu.
#include "field.cuh"
#include "kernels.cuh"

namespace pdmp {

constexpr int kDirectThreads = 128;
constexpr int kDirectTile = 256;

// TRACE: also write every state x_t to traj ((T+1) x N x D) and every FP32
// increment -eta sigma'(s) grad s, as computed before it is added, to steps
// (T x N x D).
template <int KIND, int D, int K, bool TRACE>
__global__ void __launch_bounds__(kDirectThreads)
k_morph_direct(FieldArgs fa, const float* x0, int64_t N, int T, float eta,
               float* xT, float* __restrict__ ckpt, int kck, float* __restrict__ traj, float* __restrict__ steps) {
  constexpr int R = RecLayout<D>::kFloats;
  __shared__ __align__(16) float sm[kDirectTile * R];
  const float ngl2e = -fa.gamma * kLog2e;
  const int64_t base = (int64_t)blockIdx.x * (kDirectThreads * K) + threadIdx.x;

  float x[K][D];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    int64_t n = base + (int64_t)k * kDirectThreads;
#pragma unroll
    for (int j = 0; j < D; ++j) x[k][j] = n < N ? x0[n * D + j] : 0.0f;
  }

  for (int t = 0; t < T; ++t) {
    if (TRACE) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        int64_t n = base + (int64_t)k * kDirectThreads;
        if (n < N)
#pragma unroll
          for (int j = 0; j < D; ++j) traj[((int64_t)t * N + n) * D + j] = x[k][j];
      }
    }
    float s[K], gs[K][D];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      s[k] = 0.0f;
#pragma unroll
      for (int j = 0; j < D; ++j) gs[k][j] = 0.0f;
    }
    for (int64_t m0 = 0; m0 < fa.M; m0 += kDirectTile) {
      __syncthreads();
      stage_tile<KIND, D>(fa, m0, kDirectTile, sm);
      __syncthreads();
      const int cnt = (int)min64(kDirectTile, fa.M - m0);
      for (int i = 0; i < cnt; ++i) {
        float rec[R];
        load_rec<D>(sm, i, rec);
#pragma unroll
        for (int k = 0; k < K; ++k) accum_grad<KIND, D>(rec, x[k], ngl2e, s[k], gs[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float d1, d2, g[D];
      sigmoid_d12(s[k] + fa.bias, d1, d2);
      finish_grad_s<KIND, D>(gs[k], fa.gamma, g);
      const float c = -eta * d1;
      const int64_t n = base + (int64_t)k * kDirectThreads;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        // explicit roundings: the increment is rounded, then added (no FMA
        // contraction), identically in the traced and untraced variants
        const float inc = __fmul_rn(c, g[j]);
        if (TRACE && n < N) steps[((int64_t)t * N + n) * D + j] = inc;
        x[k][j] = __fadd_rn(x[k][j], inc);
      }
    }
    if (ckpt != nullptr && (t + 1) % kck == 0) {
      float* dst = ckpt + (int64_t)((t + 1) / kck - 1) * N * D;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        int64_t n = base + (int64_t)k * kDirectThreads;
        if (n < N)
#pragma unroll
          for (int j = 0; j < D; ++j) dst[n * D + j] = x[k][j];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    int64_t n = base + (int64_t)k * kDirectThreads;
    if (n < N)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        if (xT) xT[n * D + j] = x[k][j];
        if (TRACE) traj[((int64_t)T * N + n) * D + j] = x[k][j];
      }
  }
}

template <int KIND, int D>
static cudaError_t launch_direct(const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* xT,
                                 float* ckpt, int k, float* traj, float* steps, cudaStream_t st) {
  constexpr int K = 4;
  int64_t per_block = (int64_t)kDirectThreads * K;
  int64_t blocks = (N + per_block - 1) / per_block;
  if (blocks == 0) return cudaSuccess;
  if (traj != nullptr)
    k_morph_direct<KIND, D, K, true><<<(unsigned)blocks, kDirectThreads, 0, st>>>(fa, x0, N, T, eta, xT, ckpt, k,
                                                                                  traj, steps);
  else
    k_morph_direct<KIND, D, K, false><<<(unsigned)blocks, kDirectThreads, 0, st>>>(fa, x0, N, T, eta, xT, ckpt, k,
                                                                                   nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t morph_direct(int kind, int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta,
                         float* xT, float* ckpt, int k, float* traj, float* steps, cudaStream_t st) {
#define PDMP_CASE(KD, DD) \
  if (kind == KD && d == DD) return launch_direct<KD, DD>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, st);
  PDMP_CASE(PDMP_KIND_RBF, 1) PDMP_CASE(PDMP_KIND_RBF, 2) PDMP_CASE(PDMP_KIND_RBF, 3)
  PDMP_CASE(PDMP_KIND_RFF, 1) PDMP_CASE(PDMP_KIND_RFF, 2) PDMP_CASE(PDMP_KIND_RFF, 3) PDMP_CASE(PDMP_KIND_RFF, 4)
  PDMP_CASE(PDMP_KIND_RFF, 5) PDMP_CASE(PDMP_KIND_RFF, 6) PDMP_CASE(PDMP_KIND_RFF, 7) PDMP_CASE(PDMP_KIND_RFF, 8)
#undef PDMP_CASE
  return cudaErrorInvalidValue;
}

}  // namespace pdmp

namespace pdmp {
// Chooses the kernel for a morph request.
// RFF fields with d <= 7 take the tensor-core kernel (1.10x the packed-pair
// kernel at d = 1, 1.55x at d = 7, measured on 2^20 samples, M = 4096);
// d = 8 (eight dimensions and the phase do not fit its eight k slots) the
// packed-pair one.
static bool rff_mma(int d) { return d <= 7; }

size_t morph_workspace(int kind, int d, int64_t M, int64_t N) {
  if (kind == PDMP_KIND_RBF && (d == 2 || d == 3) && N > 0) return morph_rbf_fast_workspace(d, M, N);
  if (kind == PDMP_KIND_RFF && N > 0) {
    const size_t a = morph_rff_fast_workspace(d, M), b = rff_mma(d) ? morph_rff_mma_workspace(M) : 0;
    return a > b ? a : b;
  }
  return 0;
}

cudaError_t morph_dispatch(int kind, int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta,
                           float* xT, float* ckpt, int k, float* traj, float* steps, void* ws, cudaStream_t st) {
  if (ws != nullptr && morph_workspace(kind, d, fa.M, N) > 0) {
    if (kind == PDMP_KIND_RBF) return morph_rbf_fast(d, fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
    if (rff_mma(d)) return morph_rff_mma(d, fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
    return morph_rff_fast(d, fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
  }
  return morph_direct(kind, d, fa, x0, N, T, eta, xT, ckpt, k, traj, steps, st);
}
}  // namespace pdmp
