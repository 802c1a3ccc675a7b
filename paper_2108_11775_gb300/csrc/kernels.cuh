// Host-side launchers implemented by the .cu files of libpdmp.
#pragma once
#include "field.cuh"

namespace pdmp {

// longest checkpoint segment the VJP keeps in thread-local memory
constexpr int kMaxSegment = 32;

// traj / steps: both NULL, or both set (diagnostic trace, see pdmp_morph_trace)
cudaError_t morph_direct(int kind, int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta,
                         float* xT, float* ckpt, int k, float* traj, float* steps, cudaStream_t st);
// fast RBF path (d = 2, 3): spatially sorted tiles, expanded exponent, f32x2
size_t morph_rbf_fast_workspace(int d, int64_t M, int64_t N);
cudaError_t morph_rbf_fast(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* xT,
                           float* ckpt, int k, float* traj, float* steps, void* ws, cudaStream_t st);
// workspace the dispatcher's fast path needs (0: the request takes the direct path)
size_t morph_workspace(int kind, int d, int64_t M, int64_t N);
// ws == nullptr selects the direct path
cudaError_t morph_dispatch(int kind, int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta,
                           float* xT, float* ckpt, int k, float* traj, float* steps, void* ws, cudaStream_t st);

int64_t vjp_blocks(int64_t N);
cudaError_t morph_vjp(int kind, int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, int k,
                      const float* ckpt, const float* gT, float* g0, float* rows, float* gw, float* gbias,
                      cudaStream_t st);
cudaError_t logdet(int kind, int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* ld,
                   float* xT, cudaStream_t st);

cudaError_t occupancy_query(int kind, int d, const FieldArgs& fa, const float* x, int64_t N, float* c, float* s,
                            float* grad, cudaStream_t st);
cudaError_t box_labels(int d, const float* boxes, int64_t nb, const float* x, int64_t N, uint8_t* label,
                       cudaStream_t st);

cudaError_t lipschitz_bound(int kind, int d, const FieldArgs& fa, const double* lo, const double* hi, int cells,
                            double* L, double* G, cudaStream_t st);

size_t fit_workspace(int64_t M, int64_t n);
cudaError_t fit_occupancy(int kind, int d, const FieldArgs& geom, const float* X, const uint8_t* y, int64_t n,
                          float l2, int power_iters, int iters, float* w_out, float* bias_out, float* loss_out,
                          float* alpha_out, void* ws, cudaStream_t st);

}  // namespace pdmp
