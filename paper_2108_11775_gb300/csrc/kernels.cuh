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
// bytes of the centre table at the start of that workspace (the sort's buffers follow)
size_t rbf_fast_table_bytes(int d, int64_t M);
size_t morph_rff_fast_workspace(int d, int64_t M);
// RFF with both contractions on the tensor cores (d = 1 .. 7)
size_t morph_rff_mma_workspace(int64_t M);
cudaError_t morph_rff_mma(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* xT,
                          float* ckpt, int k, float* traj, float* steps, void* ws, cudaStream_t st);
cudaError_t morph_rff_fast(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* xT,
                           float* ckpt, int k, float* traj, float* steps, void* ws, cudaStream_t st);
// grad c at N points by the fast RBF tile kernel (ws: morph_rbf_fast_workspace)
cudaError_t grad_rbf_fast(int d, const FieldArgs& fa, const float* x, int64_t N, float* g, void* ws,
                          cudaStream_t st);

// planar serial chains for the C-space pull-back (Eq. 3)
constexpr int kChainMax = 16;
size_t cspace_workspace(int d, int64_t M, int n, int p, int64_t N);
cudaError_t cspace_morph(const FieldArgs& fa, int kind, int n, int p, const float* base, const float* len,
                         const float* q0, int64_t N, int T, float eta, float* qT, void* ws, cudaStream_t st);
// The fast RBF morph with the exponent on tcgen05 (d = 2, 3) over samples in
// the sorted order perm (N < 2^31); eligible: whether the fast path takes it
// (only with PDMP_RBF_TC05=1 in the environment: slower than the FP32 tile
// kernel on the benchmarked workload).
bool morph_rbf_tc05_eligible(int d, int64_t N);
cudaError_t morph_rbf_tc05(int d, const FieldArgs& fa, const float* x0, const int32_t* perm, int64_t N, int T,
                           float eta, float* xT, float* ckpt, int k, float* traj, float* steps, float* s_out,
                           float* g_out, cudaStream_t st);
// s_out (optional): the logit at the last step's state, per sample
cudaError_t morph_rbf_fast(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* xT,
                           float* ckpt, int k, float* traj, float* steps, void* ws, cudaStream_t st,
                           float* s_out = nullptr);
// workspace the dispatcher's fast path needs (0: the request takes the direct path)
size_t morph_workspace(int kind, int d, int64_t M, int64_t N);
// ws == nullptr selects the direct path
cudaError_t morph_dispatch(int kind, int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta,
                           float* xT, float* ckpt, int k, float* traj, float* steps, void* ws, cudaStream_t st);

// ws: NULL (direct kernel) or morph_rbf_fast_workspace bytes (RBF, d = 2, 3: sorted tiles);
// work (device, may be NULL) is incremented by the feature evaluations performed
cudaError_t morph_inverse(int kind, int d, const FieldArgs& fa, const float* z, int64_t N, int T, float eta,
                          float tol, int maxit, float* y, int32_t* iters, void* ws, unsigned long long* work,
                          cudaStream_t st);

// the tanh occupancy network of Sec. 3.1 (d -> H -> H -> 1), float32 device arrays
struct TanhNetArgs {
  int d, H;
  const float *W1, *b1, *W2, *b2, *w3;
  float b3;
};
cudaError_t tanh_net_morph(const TanhNetArgs& net, const float* x0, int64_t N, int T, float eta, float* xT,
                           float* ckpt, int k, cudaStream_t st);
cudaError_t tanh_net_query(const TanhNetArgs& net, const float* x, int64_t N, float* c, float* s, float* g,
                           cudaStream_t st);

size_t morph_rbf_cull_workspace(int d, int64_t M, int64_t N);
// s_out, g_out (may be NULL): the logit and grad c of the last step's state, per sample
cudaError_t morph_rbf_cull(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float r_cut,
                           float* xT, float* ckpt, int k, void* ws, unsigned long long* work, cudaStream_t st,
                           float* s_out = nullptr, float* g_out = nullptr);
cudaError_t abs_weight_sum(const float* w, int64_t M, double* out, cudaStream_t st);

cudaError_t logdet_rff7_mma(const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* ld, float* xT,
                            cudaStream_t st);

cudaError_t uniform_log_density(const float* y, int64_t N, int d, const double* lo, const double* hi, float* lp,
                                cudaStream_t st);

int64_t vjp_blocks(int64_t N);
// gw[m] = sum_b rows[b][m] (m < width - 1), *gbias = sum_b rows[b][width - 1], in block order
cudaError_t sum_vjp_rows(const float* rows, int64_t nrows, int64_t width, float* gw, float* gbias, cudaStream_t st);
// the tensor-core VJP for RFF fields (d <= 7, segments k <= kVjpMmaMaxSegment; ws: morph_rff_mma_workspace).
// rows: nullptr, or vjp_rff_mma_blocks(N) x (M + 1) floats for the weight and bias gradient (gw, gbias)
constexpr int kVjpMmaMaxSegment = 16;
int64_t vjp_rff_mma_blocks(int64_t N);
// the staging wait's self-test (src, dst: 16 floats, 16-byte aligned; limit in clocks)
cudaError_t stage_wait_selftest(const float* src, float* dst, long long limit, int with_copy, cudaStream_t st);
cudaError_t vjp_rff_mma(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, int k,
                        const float* ckpt, const float* gT, float* g0, float* rows, float* gw, float* gbias, void* ws,
                        cudaStream_t st);
// the sorted-tile VJP for RBF fields (d = 2, 3, k <= kVjpMmaMaxSegment; ws: morph_rbf_fast_workspace).
// rows: nullptr, or vjp_rbf_fast_blocks(d, N) x (M + 1) floats for the weight and bias gradient (gw, gbias)
int64_t vjp_rbf_fast_blocks(int d, int64_t N);
cudaError_t vjp_rbf_fast(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, int k,
                         const float* ckpt, const float* gT, float* g0, float* rows, float* gw, float* gbias,
                         void* ws, cudaStream_t st);
cudaError_t morph_vjp(int kind, int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, int k,
                      const float* ckpt, const float* gT, float* g0, float* rows, float* gw, float* gbias,
                      cudaStream_t st);
// ws: NULL or the morph's workspace (RFF, d <= 7: the tensor-core kernel)
cudaError_t logdet(int kind, int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* ld,
                   float* xT, void* ws, cudaStream_t st);
cudaError_t logdet_rff_mma(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* ld,
                           float* xT, void* ws, cudaStream_t st);
// the inverse map for RFF fields (d <= 7) on the tensor cores (ws: morph_rff_mma_workspace)
cudaError_t inverse_rff_mma(int d, const FieldArgs& fa, const float* z, int64_t N, int T, float eta, float tol,
                            int maxit, float* y, int32_t* iters, unsigned long long* work, void* ws, cudaStream_t st);
// RBF, d = 2, 3 on sorted tiles (ws: morph_rbf_fast_workspace)
cudaError_t logdet_rbf_fast(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* ld,
                            float* xT, void* ws, cudaStream_t st);
// the inverse map with every step's log-det from its last fixed-point sweep
// (RBF, d = 2, 3 on sorted tiles; ws: morph_rbf_fast_workspace): y = phi^{-1}(z),
// ld = log det J(y)
cudaError_t log_density_rbf_fast(int d, const FieldArgs& fa, const float* z, int64_t N, int T, float eta, float tol,
                                 int maxit, float* y, float* ld, int32_t* iters, unsigned long long* work, void* ws,
                                 cudaStream_t st);

cudaError_t occupancy_query(int kind, int d, const FieldArgs& fa, const float* x, int64_t N, float* c, float* s,
                            float* grad, cudaStream_t st);
cudaError_t box_labels(int d, const float* boxes, int64_t nb, const float* x, int64_t N, uint8_t* label,
                       cudaStream_t st);

cudaError_t lipschitz_bound(int kind, int d, const FieldArgs& fa, const double* lo, const double* hi, int cells,
                            double* L, double* G, cudaStream_t st);

int batch_variants();
size_t batch_workspace(const pdmp_env* envs, int n, int variant);
cudaError_t batch_prepare(const pdmp_env* envs, int n, int variant, void* ws, pdmp_batch_plan* plan,
                          cudaStream_t st);
cudaError_t batch_run(const pdmp_batch_plan* plan, void* ws, cudaStream_t st);

// surrogate MLP (mlp.cu, surrogate.cu)
constexpr int64_t kMlpNW = 39 * 128 + 2 * 128 * 128 + 3 * 128;  // weights W1 (over the 39-wide encoding), W2, W3, W4
constexpr int64_t kMlpNB = 3 * 128 + 3;                         // biases b1, b2, b3, b4
cudaError_t mlp_forward(const pdmp_mlp* net, const float* x0, int64_t N, float* y, bool fp32_act, cudaStream_t st);
cudaError_t mlp_forward_tc05(const pdmp_mlp* net, const float* x0, int64_t N, float* y, bool fp32_act,
                             cudaStream_t st);
size_t mlp_train_workspace(int B);
cudaError_t mlp_gradient(const pdmp_mlp* net, const float* x0, const float* xT, int B, bool fp32_act, float* loss,
                         float* gW, float* gb, void* ws, cudaStream_t st);
cudaError_t mlp_train_step(const pdmp_mlp* net, const float* x0, const float* xT, int B, float lr, float beta1,
                           float beta2, float eps, int step, float* loss, void* ws, cudaStream_t st);
cudaError_t mlp_refresh(const pdmp_mlp* net, cudaStream_t st);
size_t surrogate_workspace(int d, int64_t M, int64_t N);
cudaError_t displacement_rms(const float* x0, const float* xT, int64_t N, int d, float* rms, cudaStream_t st);
// r_cut > 0: the residual check on the culled kernel (features farther than
// r_cut from a tile dropped); r_cut = 0: on the dense kernel
cudaError_t surrogate_infer(const pdmp_mlp* net, int d, const FieldArgs& fa, const float* x0, int64_t N, int T,
                            float eta, float tau_r, float r_cut, float* xT, int64_t* n_fallback, void* ws,
                            cudaStream_t st);
size_t residual_threshold_workspace(int d, int64_t M, int64_t N);
cudaError_t residual_threshold(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, int64_t k,
                               float* tau_r, float* xT, void* ws, cudaStream_t st);

size_t fit_workspace(int64_t M, int64_t n);
cudaError_t fit_occupancy(int kind, int d, const FieldArgs& geom, const float* X, const uint8_t* y, int64_t n,
                          float l2, int power_iters, int iters, float* w_out, float* bias_out, float* loss_out,
                          float* alpha_out, void* ws, cudaStream_t st);

}  // namespace pdmp
