// Occupancy queries c(x), s(x), grad c(x) (Sec. 3.1) and ground-truth labels
// from closed axis-aligned boxes.
#include "field.cuh"
#include "kernels.cuh"

namespace pdmp {

constexpr int kQueryThreads = 128;
constexpr int kQueryTile = 256;

template <int KIND, int D>
__global__ void __launch_bounds__(kQueryThreads)
k_query(FieldArgs fa, const float* __restrict__ x, int64_t N, float* __restrict__ c, float* __restrict__ s_out,
        float* __restrict__ grad) {
  constexpr int R = RecLayout<D>::kFloats;
  __shared__ __align__(16) float sm[kQueryTile * R];
  const float ngl2e = -fa.gamma * kLog2e;
  const int64_t n = (int64_t)blockIdx.x * kQueryThreads + threadIdx.x;
  float xv[D];
#pragma unroll
  for (int j = 0; j < D; ++j) xv[j] = n < N ? x[n * D + j] : 0.0f;
  float s = 0.0f, gs[D];
#pragma unroll
  for (int j = 0; j < D; ++j) gs[j] = 0.0f;
  for (int64_t m0 = 0; m0 < fa.M; m0 += kQueryTile) {
    __syncthreads();
    stage_tile<KIND, D>(fa, m0, kQueryTile, sm);
    __syncthreads();
    const int cnt = (int)min64(kQueryTile, fa.M - m0);
    for (int i = 0; i < cnt; ++i) {
      float rec[RecLayout<D>::kFloats];
      load_rec<D>(sm, i, rec);
      accum_grad<KIND, D>(rec, xv, ngl2e, s, gs);
    }
  }
  if (n >= N) return;
  s += fa.bias;
  if (s_out) s_out[n] = s;
  if (c) c[n] = sigmoid_f(s);
  if (grad) {
    float d1, d2, g[D];
    sigmoid_d12(s, d1, d2);
    finish_grad_s<KIND, D>(gs, fa.gamma, g);
#pragma unroll
    for (int j = 0; j < D; ++j) grad[n * D + j] = d1 * g[j];
  }
}

template <int KIND, int D>
static cudaError_t launch_query(const FieldArgs& fa, const float* x, int64_t N, float* c, float* s, float* grad,
                                cudaStream_t st) {
  int64_t blocks = (N + kQueryThreads - 1) / kQueryThreads;
  if (blocks == 0) return cudaSuccess;
  k_query<KIND, D><<<(unsigned)blocks, kQueryThreads, 0, st>>>(fa, x, N, c, s, grad);
  return cudaGetLastError();
}

cudaError_t occupancy_query(int kind, int d, const FieldArgs& fa, const float* x, int64_t N, float* c, float* s,
                            float* grad, cudaStream_t st) {
  if (kind == PDMP_KIND_RBF) {
    if (d == 1) return launch_query<PDMP_KIND_RBF, 1>(fa, x, N, c, s, grad, st);
    if (d == 2) return launch_query<PDMP_KIND_RBF, 2>(fa, x, N, c, s, grad, st);
    if (d == 3) return launch_query<PDMP_KIND_RBF, 3>(fa, x, N, c, s, grad, st);
  } else {
    if (d == 1) return launch_query<PDMP_KIND_RFF, 1>(fa, x, N, c, s, grad, st);
    if (d == 2) return launch_query<PDMP_KIND_RFF, 2>(fa, x, N, c, s, grad, st);
    if (d == 3) return launch_query<PDMP_KIND_RFF, 3>(fa, x, N, c, s, grad, st);
    if (d == 4) return launch_query<PDMP_KIND_RFF, 4>(fa, x, N, c, s, grad, st);
    if (d == 5) return launch_query<PDMP_KIND_RFF, 5>(fa, x, N, c, s, grad, st);
    if (d == 6) return launch_query<PDMP_KIND_RFF, 6>(fa, x, N, c, s, grad, st);
    if (d == 7) return launch_query<PDMP_KIND_RFF, 7>(fa, x, N, c, s, grad, st);
    if (d == 8) return launch_query<PDMP_KIND_RFF, 8>(fa, x, N, c, s, grad, st);
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ labels
constexpr int kLabelThreads = 256;
constexpr int kBoxTile = 256;

template <int D>
__global__ void __launch_bounds__(kLabelThreads)
k_box_labels(const float* __restrict__ boxes, int64_t nb, const float* __restrict__ x, int64_t N,
             uint8_t* __restrict__ label) {
  __shared__ float sb[kBoxTile * 2 * D];
  const int64_t n = (int64_t)blockIdx.x * kLabelThreads + threadIdx.x;
  float xv[D];
#pragma unroll
  for (int j = 0; j < D; ++j) xv[j] = n < N ? x[n * D + j] : 0.0f;
  bool inside_any = false;
  for (int64_t b0 = 0; b0 < nb; b0 += kBoxTile) {
    __syncthreads();
    const int cnt = (int)min64(kBoxTile, nb - b0);
    for (int i = threadIdx.x; i < cnt * 2 * D; i += blockDim.x) sb[i] = boxes[b0 * 2 * D + i];
    __syncthreads();
    for (int i = 0; i < cnt; ++i) {
      bool in = true;
#pragma unroll
      for (int j = 0; j < D; ++j) in = in && (sb[i * 2 * D + j] <= xv[j]) && (xv[j] <= sb[i * 2 * D + D + j]);
      inside_any = inside_any || in;
    }
  }
  if (n < N) label[n] = inside_any ? 1 : 0;
}

cudaError_t box_labels(int d, const float* boxes, int64_t nb, const float* x, int64_t N, uint8_t* label,
                       cudaStream_t st) {
  int64_t blocks = (N + kLabelThreads - 1) / kLabelThreads;
  if (blocks == 0) return cudaSuccess;
  switch (d) {
#define PDMP_CASE(DD) \
  case DD: k_box_labels<DD><<<(unsigned)blocks, kLabelThreads, 0, st>>>(boxes, nb, x, N, label); break;
    PDMP_CASE(1) PDMP_CASE(2) PDMP_CASE(3) PDMP_CASE(4) PDMP_CASE(5) PDMP_CASE(6) PDMP_CASE(7) PDMP_CASE(8)
#undef PDMP_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace pdmp
