/*
 * pdmp.h -- C ABI of libpdmp, the GB300 (sm_103a) library for the sample-
 * morphing hot path of "Parallelised Diffeomorphic Sampling-based Motion
 * Planning" (Lai, Zhi, Hermans, Ramos; arXiv 2108.11775).
 *
 * Conventions shared by every call
 * --------------------------------
 * Memory     Array arguments are DEVICE pointers unless a comment says "host".
 *            Float arrays are float32, row-major, torch-contiguous: a batch of
 *            N points in d dimensions is N x d with the d coordinates of a point
 *            adjacent.  The caller owns every buffer, including workspaces; the
 *            compute calls allocate no device memory.  The exceptions say so:
 *            pdmp_sampler_create allocates its batch buffers (freed by
 *            pdmp_sampler_destroy), pdmp_morph_noalloc and the small bound /
 *            radius reductions use fixed device arrays of the library.
 * Alignment  Every device array must be 16-byte aligned (cudaMalloc and torch
 *            allocations are).  Misaligned pointers give PDMP_ERR_INVALID_ARG.
 * Ordering   Every call is asynchronous on `stream` (a cudaStream_t; NULL is the
 *            legacy default stream) unless it says it synchronises.  Arguments
 *            are validated on the host before anything is launched; a call that
 *            returns an error has launched nothing.
 * Errors     Each call returns a pdmp_status.  Errors raised while kernels run
 *            are reported by pdmp_stream_status().  No kernel traps.
 *
 * The occupancy field (Sec. 3.1)
 * ------------------------------
 * c(x) = sigmoid(s(x)),  s(x) = sum_m w_m phi_m(x) + bias,  with
 *   RBF  phi_m(x) = exp(-gamma |x - mu_m|^2)       (centres = mu, M x d)
 *   RFF  phi_m(x) = cos(omega_m . x + b_m)          (centres = omega, M x d;
 *                                                    phase = b, M)
 * The map (Sec. 3.2, Eq. 1 integrated with Euler's method):
 *   x_{t+1} = x_t - eta * grad c(x_t),  t = 0 .. T-1.
 * Each step is a diffeomorphism when eta * L < 1, L a Lipschitz constant of
 * grad c (Sec. 3.2: Picard-Lindelof needs a Lipschitz gradient).
 */
#ifndef PDMP_H
#define PDMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t pdmp_status;

#define PDMP_OK                       0
#define PDMP_ERR_INVALID_ARG          1  /* bad size, pointer, alignment or option */
#define PDMP_ERR_STEP_TOO_LARGE       2  /* eta * L >= 1 for a field that carries L */
#define PDMP_ERR_WORKSPACE_TOO_SMALL  3
#define PDMP_ERR_CUDA                 4  /* a CUDA runtime call failed */
#define PDMP_ERR_NOT_CONVERGED        5
#define PDMP_ERR_TIMEOUT              6
#define PDMP_ERR_DEVICE_FLAG          7  /* a kernel recorded a numerical failure */
#define PDMP_ERR_UNSUPPORTED          8  /* valid request this library version does not handle */

/* Bits of the device flag (the detail of PDMP_ERR_DEVICE_FLAG). */
#define PDMP_FLAG_NONPOSITIVE_PIVOT   1  /* log-det: I - eta Hess c not positive definite at some step */
#define PDMP_FLAG_FIT_NONFINITE       2  /* fit: the loss became NaN or infinite */
#define PDMP_FLAG_NOT_CONVERGED       4  /* inverse: a block stopped at maxit iterations */
#define PDMP_FLAG_STAGE_TIMEOUT       8  /* a bounded wait for a shared-memory stage copy gave up (results invalid) */
#define PDMP_FLAG_MMA_TIMEOUT        16  /* a bounded wait for a tensor-core (tcgen05) MMA gave up (results invalid) */

#define PDMP_KIND_RBF 0
#define PDMP_KIND_RFF 1

/* The learned occupancy field.  All pointers are device pointers to float32.
 * RBF: d in {1, 2, 3}.  RFF: 1 <= d <= 8.  M >= 1.
 * `lipschitz` is optional: when > 0 it is a bound L on |Hess c|_2 over the
 * region the samples visit, and calls that take a step size reject
 * eta * L >= 1 with PDMP_ERR_STEP_TOO_LARGE. */
typedef struct {
  int32_t kind;            /* PDMP_KIND_RBF or PDMP_KIND_RFF */
  int32_t d;               /* dimension of x */
  int64_t M;               /* number of features */
  const float* centres;    /* RBF: mu (M x d).  RFF: omega (M x d) */
  const float* phase;      /* RFF: b (M).  RBF: must be NULL */
  float gamma;             /* RBF width (> 0).  RFF: ignored */
  const float* w;          /* M feature weights */
  float bias;              /* logit bias */
  double lipschitz;        /* 0, or a bound on |Hess c| checked against eta */
} pdmp_field;

/* Static, NUL-terminated description of a status code (never NULL). */
const char* pdmp_status_string(pdmp_status s);

/* Library version, as major * 10000 + minor * 100 + patch. */
int32_t pdmp_version(void);

/* Synchronises `stream`, then reports the first error raised on it since the
 * previous call: a CUDA error (PDMP_ERR_CUDA) or a numerical failure a kernel
 * recorded in the library's device flag (PDMP_ERR_DEVICE_FLAG; the flag is
 * cleared by this call).  *detail (host, may be NULL) receives the CUDA error
 * code or the flag value. */
pdmp_status pdmp_stream_status(void* stream, int32_t* detail);

/* Host-side watchdog: waits for the work queued on `stream` so far, polling
 * an event, for at most timeout_ms milliseconds (>= 0).  PDMP_ERR_TIMEOUT if
 * the work has not finished by then (it keeps running; call again to keep
 * waiting); otherwise as pdmp_stream_status. */
pdmp_status pdmp_stream_wait(void* stream, int32_t timeout_ms, int32_t* detail);

/* Self-test of the kernels' bounded wait for a shared-memory stage copy (the
 * bulk copies that stage the random Fourier tables).  One block initialises
 * a stage barrier; with with_copy != 0 it copies the 16 floats at src
 * (device, 16-byte aligned) into shared memory by the staging path and then
 * to dst (device, 16 floats); one thread waits for the barrier at most
 * limit_clocks (1 .. 2^31) SM clocks.  Without the copy nothing completes
 * the barrier, the wait runs out and the kernel raises
 * PDMP_FLAG_STAGE_TIMEOUT, which pdmp_stream_status then reports; nothing
 * hangs and nothing is left in flight. */
pdmp_status pdmp_selftest_stage_wait(const float* src, float* dst, int64_t limit_clocks, int32_t with_copy,
                                     void* stream);

/* ---------------------------------------------------------------------- */
/* Sec. 3.2 (Eq. 1, "Drawing Samples"): morph a batch of base samples.      */
/* ---------------------------------------------------------------------- */
/* x0: N x d base samples.  xT: N x d output; may alias x0 exactly (in place).
 * T >= 0 Euler steps of size eta > 0.  N = 0 or T = 0 are valid (T = 0
 * copies x0 to xT).
 * ckpt: NULL, or a (T/k) x N x d buffer that receives x_{k}, x_{2k}, ..., x_T
 * (checkpoints for pdmp_morph_vjp); then k >= 1 must divide T.
 * ws: NULL, or ws_bytes >= pdmp_morph_workspace(f, N) bytes of caller-owned
 * device scratch.  With a workspace, RBF fields in d = 2 or 3 take the fast
 * path: samples are ordered spatially (a deterministic counting sort on
 * Hilbert-ordered cells) so that each tile of 320 samples (128 when N is too
 * small to fill the GPU with 320-sample tiles) is compact, and features are
 * evaluated in an expanded form about the tile's centre with packed f32x2
 * arithmetic (2d + 1 FP32 operations and one ex2 per feature); RFF fields
 * with d <= 7 put both contractions of a step, theta = omega . x + b and
 * sum_m w_m sin(theta_m) omega_m, on the tensor cores (TF32 with hi/lo
 * splits) and d = 8 takes a packed-pair path.  The RBF fast
 * path needs N < 2^31 (PDMP_ERR_INVALID_ARG otherwise).  Without a
 * workspace every feature is evaluated directly from x - mu (RBF) or
 * omega . x + b (RFF).  With PDMP_RBF_TC05=1 in the environment the RBF
 * fast path (d = 2, 3) takes a variant whose exponent a_m + b_m . u runs on
 * the fifth-generation tensor cores (tcgen05.mma, TF32 hi/lo pieces, FP32
 * accumulators in tensor memory) for groups of 256 samples; it is slower
 * than the default on the measured workloads and kept for comparison.
 * Sample state stays on chip (registers or shared memory) for all T steps;
 * features are evaluated in
 * FP32 with exp2 / sin / cos on the special-function unit.  Calls that share
 * a workspace must not overlap on the GPU. */
size_t pdmp_morph_workspace(const pdmp_field* f, int64_t N);
pdmp_status pdmp_morph(const pdmp_field* f, const float* x0, int64_t N, int32_t T, float eta,
                       float* xT, float* ckpt, int32_t k, void* ws, size_t ws_bytes, void* stream);

/* Diagnostic twin of pdmp_morph with the same kernel arithmetic (the same
 * path is chosen for the same f, N and ws): traj ((T+1) x N x d) receives
 * x_0 .. x_T and steps (T x N x d) the FP32 increment -eta sigma'(s)
 * grad s(x_t) of every step as computed, before it is added to x_t (so that
 * the accuracy of a step can be checked apart from the rounding of the
 * float32 state).  steps may be NULL only when T = 0. */
pdmp_status pdmp_morph_trace(const pdmp_field* f, const float* x0, int64_t N, int32_t T, float eta, float* traj,
                             float* steps, void* ws, size_t ws_bytes, void* stream);

/* The fast RBF morph for callers that cannot allocate device memory (no
 * counterpart in the paper).  Same arguments and results as pdmp_morph with
 * ws = NULL replaced by scratch built into the library: a 12 MiB device array
 * that every GPU loading the library holds until the process exits.  Limits:
 * RBF fields with d = 2 or 3 (others give PDMP_ERR_UNSUPPORTED), N <= 2^20
 * and M <= 16384 (larger requests give PDMP_ERR_WORKSPACE_TOO_SMALL before
 * anything is launched).  No checkpoints.  The first call on a device looks up
 * the scratch's device address; make it before any stream capture.  That
 * address is cached per device and does not survive cudaDeviceReset (or any
 * other teardown of the device's primary context).  All calls share the
 * scratch: calls that overlap on the GPU race and must be serialised by the
 * caller.  Calls no cudaMalloc / cudaFree. */
pdmp_status pdmp_morph_noalloc(const pdmp_field* f, const float* x0, int64_t N, int32_t T, float eta, float* xT,
                               void* stream);

/* ---------------------------------------------------------------------- */
/* Many environments in one persistent launch (no counterpart in the paper: */
/* the paper morphs one scene's samples).                                   */
/* ---------------------------------------------------------------------- */
/* One environment: an RBF field with d = 2 or 3, its own N samples (x0, N x d,
 * device), output xT (N x d, device; may alias x0), step size and step count.
 * Environments may differ in d, M, N, eta and T. */
typedef struct {
  pdmp_field field;
  const float* x0;
  float* xT;
  int64_t N;
  float eta;
  int32_t T;
} pdmp_env;

/* What pdmp_batch_prepare planned (host struct, filled by the library). */
typedef struct {
  int32_t n_envs;
  int32_t variant;        /* tile shape, 0 .. pdmp_batch_variants() - 1 */
  int32_t grid, block;    /* persistent blocks and threads per block */
  size_t smem_bytes;
  int64_t n_units;        /* (environment, 256-or-128-sample tile) work units */
  int64_t total_N, total_M, total_cells, nchunks;
  size_t ws_bytes;        /* workspace bytes the plan uses */
  double work;            /* sum over environments of N * M * T feature evaluations */
  size_t off[12];         /* byte offsets of the workspace regions */
} pdmp_batch_plan;

/* Number of tile shapes the batched kernel is built with. */
int32_t pdmp_batch_variants(void);

/* Workspace bytes for these environments (host array) and tile shape. */
size_t pdmp_batch_workspace(const pdmp_env* envs, int32_t n_envs, int32_t variant);

/* Validates the environments (host array of n_envs >= 1), writes the device
 * environment table and the work list -- (environment, tile) units ordered
 * by decreasing M * T -- into ws, and fills *plan.  Copies host to device and
 * synchronises `stream`: call it outside stream capture, once per set of
 * environments (their buffers' addresses are baked into the plan). */
pdmp_status pdmp_batch_prepare(const pdmp_env* envs, int32_t n_envs, int32_t variant, void* ws, size_t ws_bytes,
                               pdmp_batch_plan* plan, void* stream);

/* Runs a prepared batch: every environment's centre table, one spatial sort
 * over all samples, and one persistent morph kernel whose blocks claim work
 * units from an atomic counter.  Launches and memsets only (no host copies,
 * no allocation), so it can be captured into a CUDA graph; calls sharing a
 * workspace must not overlap on the GPU. */
pdmp_status pdmp_morph_batched(const pdmp_batch_plan* plan, void* ws, void* stream);

/* Autotuner: prepares and times every tile shape on these environments
 * (one warm-up and `reps` timed runs each, CUDA events on `stream`), leaves
 * ws prepared for the fastest, and returns it in *best and its plan in *plan.
 * times_ms (host, may be NULL) receives pdmp_batch_variants() best times.
 * ws must hold the largest pdmp_batch_workspace over the variants.
 * Synchronises `stream`. */
pdmp_status pdmp_batch_autotune(const pdmp_env* envs, int32_t n_envs, int32_t reps, void* ws, size_t ws_bytes,
                                int32_t* best, float* times_ms, pdmp_batch_plan* plan, void* stream);

/* Captures pdmp_morph_batched(plan, ws) into a CUDA graph and instantiates
 * it; *graph_exec receives an opaque cudaGraphExec_t.  `stream` must not be
 * the legacy default stream (capture needs a created stream). */
pdmp_status pdmp_batch_graph_create(const pdmp_batch_plan* plan, void* ws, void* stream, void** graph_exec);
pdmp_status pdmp_graph_launch(void* graph_exec, void* stream);
pdmp_status pdmp_graph_destroy(void* graph_exec);

/* ---------------------------------------------------------------------- */
/* Learned surrogate of the T-step map (no counterpart in the paper): an MLP */
/* predicts x_T - x_0; the plain morph checks it and replaces it when it    */
/* fails.                                                                   */
/* ---------------------------------------------------------------------- */
/* Network 39 -> 128 -> 128 -> 128 -> 3, SiLU between the linear layers, on
 * normalised coordinates: u = (x_0 - lo) * in_scale - 1 is encoded as
 * enc(u) = [u_0..u_2, then for k = 0..5: sin(2^k pi u_0..u_2),
 * cos(2^k pi u_0..u_2)] (39 values), output f = (x_T - x_0) / out_scale.
 * Device buffers, caller-owned:
 *   W        FP32 master weights, PDMP_MLP_NW floats: W1 (128 x 39), W2 (128 x
 *            128), W3 (128 x 128), W4 (3 x 128), each [out][in] row-major;
 *   b        FP32 biases, PDMP_MLP_NB floats: b1, b2, b3 (128 each), b4 (3);
 *   W_bf16   BF16 copy of W (same layout), the weights the kernels use;
 *   Wt_bf16  BF16 transposes of W2 and W3 (2 x 128 x 128), for the backward;
 *   adam     Adam moments: m_W, v_W (PDMP_MLP_NW each), m_b, v_b (PDMP_MLP_NB
 *            each); zero before the first step.
 * Matrix products run on the tensor cores in BF16 with FP32 accumulation,
 * the weight gradient too ([dW | db] = dZ^T [a | 1] per layer). */
#define PDMP_MLP_NW 38144
#define PDMP_MLP_NB 387
typedef struct {
  float* W;
  float* b;
  uint16_t* W_bf16;
  uint16_t* Wt_bf16;
  float* adam;
  float lo[3], in_scale[3], out_scale[3];
} pdmp_mlp;

/* rms (device, d floats) = root mean square over the N rows of xT - x0, per
 * coordinate: the output scale of the network, from training pairs. */
pdmp_status pdmp_displacement_rms(const float* x0, const float* xT, int64_t N, int32_t d, float* rms, void* stream);

/* Rewrites W_bf16 and Wt_bf16 from W (after initialising or loading W). */
pdmp_status pdmp_mlp_refresh(const pdmp_mlp* net, void* stream);

/* xT_hat (N x 3) = x0 + out_scale * f(u(x0)). */
pdmp_status pdmp_mlp_forward(const pdmp_mlp* net, const float* x0, int64_t N, float* xT_hat, void* stream);

/* pdmp_mlp_forward in the FP32-activation mode (diagnostic): the same kernel
 * and fragment layouts, with every activation fed to the tensor cores as the
 * sum of three BF16 pieces (at least 24 bits of the FP32 value), so that the
 * products are those of FP32 activations with the BF16 weights. */
pdmp_status pdmp_mlp_forward_fp32act(const pdmp_mlp* net, const float* x0, int64_t N, float* xT_hat, void* stream);

/* The loss and gradient of one training batch without an update (diagnostic):
 * gW (PDMP_MLP_NW floats, device, the layout of W) and gb (PDMP_MLP_NB, the
 * layout of b) receive d loss / d(W, b) with respect to the BF16 weights the
 * kernels use; loss (device, may be NULL) the batch loss.  fp32_act = 0: the
 * training step's own arithmetic (BF16 activations and backward signals, FP32
 * accumulation); fp32_act = 1: the same kernels with activations and backward
 * signals carried as three BF16 pieces each (FP32-activation mode), so that
 * the result matches an FP64 evaluation of the same BF16 weights to FP32
 * rounding.  ws: pdmp_mlp_train_workspace(B) bytes. */
pdmp_status pdmp_mlp_gradient(const pdmp_mlp* net, const float* x0, const float* xT, int32_t B, int32_t fp32_act,
                              float* loss, float* gW, float* gb, void* ws, size_t ws_bytes, void* stream);

/* One Adam step (step = 1, 2, ...) on the mean squared error between f(u(x0))
 * and (xT - x0) / out_scale over a batch of B pairs (x0, xT: B x 3 device).
 * loss (device, one float, may be NULL) receives the batch loss before the
 * update.  ws: pdmp_mlp_train_workspace(B) bytes. */
size_t pdmp_mlp_train_workspace(int32_t B);
pdmp_status pdmp_mlp_train_step(const pdmp_mlp* net, const float* x0, const float* xT, int32_t B, float lr,
                                float beta1, float beta2, float eps, int32_t step, float* loss, void* ws,
                                size_t ws_bytes, void* stream);

/* Surrogate morph with the plain morph as fallback and judge: xT (N x 3)
 * first receives the network's prediction; then one plain Euler step is
 * evaluated at every prediction, and a sample fails the residual check when
 * the prediction lies in predicted-occupied space (s >= 0, i.e. c >= 1/2),
 * when that step's length exceeds tau_r, or when it is not finite.  Failed
 * samples are morphed by the plain T-step kernel from their x0 and written
 * back.  *n_fallback (host) receives the number of failed samples (this call
 * synchronises `stream` once, to learn it).  xT must not alias x0.  f: RBF with d = 3 (the network's
 * input and output size).  ws: pdmp_surrogate_workspace(f, N) bytes. */
size_t pdmp_surrogate_workspace(const pdmp_field* f, int64_t N);
pdmp_status pdmp_surrogate_infer(const pdmp_mlp* net, const pdmp_field* f, const float* x0, int64_t N, int32_t T,
                                 float eta, float tau_r, float* xT, int64_t* n_fallback, void* ws, size_t ws_bytes,
                                 void* stream);

/* pdmp_surrogate_infer on the spatially culled kernel (pdmp_morph_culled's
 * features within r_cut of a tile; r_cut > 0 and finite, else
 * PDMP_ERR_INVALID_ARG), for the residual check and for the fallback.  With
 * r_cut from pdmp_cull_radius(f, eps), the checked logit and |grad s| are
 * within eps of the dense check's, so only samples within that margin of the
 * thresholds (s = 0, step length = tau_r) can be decided differently; the
 * step is taken as -eta grad c at the prediction.  Failed samples are morphed
 * by pdmp_morph_culled with the same r_cut.  Same workspace. */
pdmp_status pdmp_surrogate_infer_culled(const pdmp_mlp* net, const pdmp_field* f, const float* x0, int64_t N,
                                        int32_t T, float eta, float tau_r, float r_cut, float* xT,
                                        int64_t* n_fallback, void* ws, size_t ws_bytes, void* stream);

/* The residual threshold tau_r of pdmp_surrogate_infer from training
 * samples: the q-quantile (nearest rank: the ceil(q N)-th smallest, 0 < q <= 1)
 * of the length |FP32 increment| of the plain morph's last step, T steps of
 * eta from each of the N samples x0 (N x d device; RBF fields, d = 2 or 3).
 * *tau_r (host) receives it (this call synchronises `stream` once); xT (device,
 * N x d, may be NULL) receives x_T, the training targets.  The selection is
 * exact (a radix select on the length's bits; NaN lengths rank last).
 * ws: pdmp_residual_threshold_workspace(f, N) bytes. */
size_t pdmp_residual_threshold_workspace(const pdmp_field* f, int64_t N);
pdmp_status pdmp_residual_threshold(const pdmp_field* f, const float* x0, int64_t N, int32_t T, float eta, float q,
                                    float* tau_r, float* xT, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------- */
/* The diffeomorphic sampler (Sec. 3.3).                                    */
/* ---------------------------------------------------------------------- */
/* A bounded concurrent bucket of d-dimensional float samples on the host
 * (FIFO).  push copies up to n samples in, waiting up to timeout_ms for room
 * (*pushed receives how many went in; fewer after a timeout or close); pop
 * copies out up to n of the oldest without waiting (*popped: how many).
 * Thread-safe; close wakes waiting pushers and makes later pushes push
 * nothing.  Host memory only: usable without a GPU. */
typedef struct pdmp_queue pdmp_queue;
pdmp_status pdmp_queue_create(int32_t d, int64_t capacity, pdmp_queue** out);
pdmp_status pdmp_queue_push(pdmp_queue* q, const float* x, int64_t n, int32_t timeout_ms, int64_t* pushed);
pdmp_status pdmp_queue_pop(pdmp_queue* q, float* out, int64_t n, int64_t* popped);
pdmp_status pdmp_queue_size(pdmp_queue* q, int64_t* n);
pdmp_status pdmp_queue_close(pdmp_queue* q);
pdmp_status pdmp_queue_destroy(pdmp_queue* q);

/* The sampler keeps such a bucket filled from a background thread: batch
 * base samples uniform on [lo, hi] drawn on the current device by a
 * counter-based generator (Philox4x32-10; coordinate j of sample i of batch
 * b is word (i d + j) mod 4 of block (i d + j) / 4 under counter (block, b)
 * and key seed, the coordinate fmaf(top 24 bits * 2^-24, hi - lo, lo)),
 * morphed by pdmp_morph (T, eta) and copied to pinned host memory.  Batches
 * enter the bucket in order, so the k-th morphed sample drawn is sample
 * k mod batch of batch k / batch.  draw never waits for the GPU: it takes up
 * to n morphed samples from the bucket (*n_morphed receives how many; they
 * come first in out) and fills the rest from the prior (the same generator,
 * another key, on the host).  The field's device arrays must outlive the
 * sampler.  A producer failure stops production and is reported by stats;
 * draws then come from the prior. */
typedef struct {
  int32_t d;
  float lo[8];
  float hi[8];
  int32_t batch;       /* samples per device batch */
  int64_t capacity;    /* bucket size in samples (>= batch) */
  int32_t T;
  float eta;
  uint64_t seed;
} pdmp_sampler_config;

typedef struct {
  int64_t produced;      /* morphed samples pushed into the bucket */
  int64_t batches;
  int64_t drawn_morphed;
  int64_t drawn_prior;
  int64_t queued;        /* samples in the bucket now */
  int32_t error;         /* 0, or the producer's failing status */
} pdmp_sampler_stats_t;

typedef struct pdmp_sampler pdmp_sampler;
pdmp_status pdmp_sampler_create(const pdmp_field* f, const pdmp_sampler_config* cfg, pdmp_sampler** out);
pdmp_status pdmp_sampler_draw(pdmp_sampler* s, float* out, int64_t n, int64_t* n_morphed);
pdmp_status pdmp_sampler_stats(pdmp_sampler* s, pdmp_sampler_stats_t* stats);
pdmp_status pdmp_sampler_destroy(pdmp_sampler* s);

/* ---------------------------------------------------------------------- */
/* Configuration space (Sec. 3.2, Eq. (3)).                                 */
/* ---------------------------------------------------------------------- */
/* A planar serial chain: n revolute joints (1..16) at base, link lengths
 * (host values, the first n used), p body points per link (1..8) at
 * fractions r/p of each link, r = 1..p.  Joint angles q (N x n, device,
 * row-major); absolute link angles are the prefix sums of q. */
typedef struct {
  int32_t n;
  int32_t p;
  float base[2];
  float lengths[16];
} pdmp_chain;

/* The T Euler steps of Eq. (1) in joint space with the cost
 * f_c(q) = sum_i c(psi_i(q)) over the b = n p body points and its gradient
 * by Eq. (3): grad_q f_c = sum_i J_i^T grad_x c(psi_i(q)).  The field is the
 * 2-D workspace occupancy (RBF or RFF, d = 2).  q0 may alias qT.  ws:
 * pdmp_cspace_workspace bytes (body points, their gradients and the fast
 * kernel's workspace for N b points), 16-byte aligned. */
size_t pdmp_cspace_workspace(const pdmp_field* f, const pdmp_chain* chain, int64_t N);
pdmp_status pdmp_cspace_morph(const pdmp_field* f, const pdmp_chain* chain, const float* q0, int64_t N, int32_t T,
                              float eta, float* qT, void* ws, size_t ws_bytes, void* stream);
/* Certified bound *Lq >= sup |Hess_q f_c|_2 from task-space bounds
 * Lx >= sup |Hess c|_2 and Gx >= sup |grad c| (host arithmetic):
 * sum over body points of |J_i|^2 Lx + Gx |Hess_q psi_i|, both from the chain
 * lengths between the joints and the point. */
pdmp_status pdmp_cspace_lipschitz(const pdmp_chain* chain, double Lx, double Gx, double* Lq);

/* ---------------------------------------------------------------------- */
/* The paper's own occupancy model as the cost (Sec. 3.1).                  */
/* ---------------------------------------------------------------------- */
/* A fully connected network with tanh between its hidden layers and a
 * sigmoid output:  s(x) = w3 . tanh(W2 tanh(W1 x + b1) + b2) + b3,
 * c = sigma(s).  Device float32 arrays, row-major with rows = output units:
 * W1 H x d, b1 H, W2 H x H, b2 H, w3 H.  Supported: d in {2, 3},
 * H in {32, 64} (else PDMP_ERR_UNSUPPORTED).  lipschitz as in pdmp_field. */
typedef struct {
  int32_t d;
  int32_t H;
  const float* W1;
  const float* b1;
  const float* W2;
  const float* b2;
  const float* w3;
  float b3;
  double lipschitz;
} pdmp_tanh_net;

/* The T Euler steps of Eq. (1) with c the network's occupancy; x0, xT, ckpt,
 * k as in pdmp_morph (x0 may alias xT). */
pdmp_status pdmp_tanh_net_morph(const pdmp_tanh_net* net, const float* x0, int64_t N, int32_t T, float eta,
                                float* xT, float* ckpt, int32_t k, void* stream);
/* c, s (N each) and grad c (N x d) at N points; any output may be NULL. */
pdmp_status pdmp_tanh_net_query(const pdmp_tanh_net* net, const float* x, int64_t N, float* c, float* s,
                                float* grad, void* stream);
/* Certified bounds over all of R^d, in FP64 on the host (the weights are
 * copied from the device; synchronises the stream): *G >= sup |grad s| and
 * *L >= sup |Hess c|_2, from the spectral norms of W1 and W2 and the maxima
 * |tanh'| <= 1, |tanh''| <= 4 / (3 sqrt 3), sigma' <= 1/4,
 * |sigma''| <= 1 / (6 sqrt 3). */
pdmp_status pdmp_tanh_net_lipschitz(const pdmp_tanh_net* net, double* L, double* G, void* stream);

/* ---------------------------------------------------------------------- */
/* Spatially culled morph (RBF, d = 2 or 3).                                */
/* ---------------------------------------------------------------------- */
/* The T Euler steps of pdmp_morph, but every sample tile sums, at every
 * step, only over the centres that can lie within r_cut of one of its
 * samples (the centres are sorted into a uniform grid each call).  Features
 * farther than r_cut are dropped: with W = sum |w_m| and r_cut >=
 * 1/sqrt(2 gamma), each gradient evaluation loses at most
 * W exp(-gamma r_cut^2) of s and W 2 gamma r_cut exp(-gamma r_cut^2) of
 * |grad s|.  ws: pdmp_morph_culled_workspace bytes, 16-byte aligned, required.
 * work (device, 8-byte aligned, may be NULL) is incremented by the number of
 * feature evaluations performed (sum over tiles and steps of the visited
 * centres times the tile's samples).  x0 may alias xT; checkpoints as in
 * pdmp_morph.  N < 2^31.  PDMP_ERR_UNSUPPORTED for RFF fields or d = 1. */
size_t pdmp_morph_culled_workspace(const pdmp_field* f, int64_t N);
pdmp_status pdmp_morph_culled(const pdmp_field* f, const float* x0, int64_t N, int32_t T, float eta, float r_cut,
                              float* xT, float* ckpt, int32_t k, void* ws, size_t ws_bytes,
                              unsigned long long* work, void* stream);

/* The smallest r_cut >= 1/sqrt(2 gamma) for which both dropped parts above
 * are at most eps (W computed on the device in FP64; synchronises the
 * stream; calls from several host threads are serialised).  *r_cut
 * receives it (host float, rounded up); *w_abs (may be NULL) receives W. */
pdmp_status pdmp_cull_radius(const pdmp_field* f, float eps, float* r_cut, double* w_abs, void* stream);

/* ---------------------------------------------------------------------- */
/* Eq. (2): the inverse map.                                                */
/* ---------------------------------------------------------------------- */
/* y[n] = phi^{-1}(z[n]): the T Euler steps of pdmp_morph are undone last
 * first, each by the fixed point y = z + eta grad c(y) (a contraction when
 * eta L < 1), iterated until every sample of a block moves by at most
 * tol * (1 + |y|) per coordinate, or maxit times.  iters (N, may be NULL)
 * receives, per sample, the largest number of iterations any step of its
 * block used; a block that stops at maxit without reaching the tolerance
 * raises PDMP_FLAG_NOT_CONVERGED in the device flag.  y may alias z.
 * ws: NULL, or ws_bytes >= pdmp_morph_workspace(f, N) bytes of device
 * scratch.  With a workspace, RBF fields in d = 2 or 3 run on the forward's
 * spatially sorted tiles (blocks of 320 samples in Hilbert order, the
 * expanded exponent about the tile's current centre; N < 2^31) and RFF
 * fields with d <= 7 on the tensor cores (blocks of 128 samples, each
 * iteration one pass of the morph's tensor-core sweep); other fields and
 * ws = NULL use blocks of 256 samples in input order, every feature
 * evaluated directly.  work (device, 8-byte aligned, may be NULL) is
 * incremented by the feature evaluations performed (per block, its
 * iterations summed over the steps times its samples times M). */
pdmp_status pdmp_morph_inverse(const pdmp_field* f, const float* z, int64_t N, int32_t T, float eta, float tol,
                               int32_t maxit, float* y, int32_t* iters, void* ws, size_t ws_bytes,
                               unsigned long long* work, void* stream);

/* Density of the morphed samples (Sec. 3.2, "Drawing Samples", by the
 * change of variables through the T-step map) for a base density uniform on
 * the box [lo, hi] (host arrays of d doubles):
 *   log_p[n] = -log vol(box) - log det J(y[n])   if y[n] lies in the box,
 *            = -inf                                otherwise,
 * with y = phi^{-1}(z) from pdmp_morph_inverse (tol, maxit, ws, ws_bytes as
 * there) written to y (N x d, must not alias z) and log det J as pdmp_logdet
 * computes it (with the same workspace).  With a workspace, RBF fields in
 * d = 2, 3 take one kernel on sorted tiles (256 samples for d = 2, 192 for
 * d = 3): every fixed-point sweep of the inverse also sums the Hessian
 * moments, and step t's log det (I - eta Hess c) is taken at the iterate of
 * the sweep that stopped, a point within the stopping tolerance of x_t,
 * instead of on a second forward pass from y. */
pdmp_status pdmp_log_density(const pdmp_field* f, const float* z, int64_t N, int32_t T, float eta, const double* lo,
                             const double* hi, float tol, int32_t maxit, float* y, float* log_p, void* ws,
                             size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------- */
/* Chain rule through Eq. (1): vector-Jacobian product of the T-step map.   */
/* ---------------------------------------------------------------------- */
/* g0[n] = (d x_T / d x_0)^T gT[n] for every sample, computed backwards as
 * g_t = (I - eta Hess c(x_t)) g_{t+1} with Hessian-vector products.
 * Intermediate states are recomputed segment by segment from checkpoints:
 * ckpt is the buffer pdmp_morph filled with the same (f, x0, T, eta, k), or
 * NULL to recompute each segment from x0.  k >= 1 must divide T.
 * gw: NULL, or an M vector that receives d/dw of sum_n <gT[n], x_T[n]>
 * (overwritten, not accumulated); gbias: NULL or one float, likewise for the
 * bias.  Both need the workspace (16-byte aligned): at least the per-block
 * rows of the sums, the size pdmp_morph_vjp_workspace(..., want_param_grad =
 * 2) returns (else PDMP_ERR_WORKSPACE_TOO_SMALL); with the
 * pdmp_morph_vjp_workspace(..., want_param_grad = 1) bytes and k <= 16, RFF
 * fields with d <= 7 also run on the tensor cores (the weight terms in a
 * further MMA pass per step) and RBF fields in d = 2, 3 on the sorted tiles
 * (a transposed pass per step: each lane sums its own features over the
 * tile's samples); the query gives the rows alone otherwise.
 * Without them ws is optional: NULL, or at least
 * pdmp_morph_vjp_workspace(..., 0) bytes; with it (k <= 16), RFF fields with
 * d <= 7 run on the tensor cores (theta, grad s, omega . g and the
 * Hessian-vector sum as TF32 MMAs with hi/lo splits) and RBF fields in
 * d = 2, 3 on the morph's sorted tiles (expanded exponent; N < 2^31), the
 * segment's states in shared memory.  gT may alias g0. */
size_t pdmp_morph_vjp_workspace(const pdmp_field* f, int64_t N, int32_t T, int32_t k, int32_t want_param_grad);
pdmp_status pdmp_morph_vjp(const pdmp_field* f, const float* x0, int64_t N, int32_t T, float eta, int32_t k,
                           const float* ckpt, const float* gT, float* g0, float* gw, float* gbias,
                           void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------- */
/* Sec. 3.2 ("Drawing Samples"): log-determinant of the map's Jacobian.     */
/* ---------------------------------------------------------------------- */
/* logdet[n] = sum_t log det(I - eta Hess c(x_t)) for sample n; xT (N x d, may
 * be NULL) receives x_T.  I - eta Hess c is symmetric positive definite when
 * eta L < 1; a step where it is not records a device flag (read with
 * pdmp_stream_status) and that sample's logdet is NaN.  ws: NULL, or
 * ws_bytes >= pdmp_morph_workspace(f, N) bytes; with it, RFF fields with
 * d <= 7 run on the tensor cores (theta, grad s and the d(d+1)/2 Hessian
 * entries as TF32 MMAs with hi/lo splits; a d x d Cholesky per sample), and
 * RBF fields in d = 2, 3 on the morph's sorted tiles (expanded exponent, the
 * Hessian from the moments sum e' c c^T; N < 2^31). */
pdmp_status pdmp_logdet(const pdmp_field* f, const float* x0, int64_t N, int32_t T, float eta,
                        float* logdet, float* xT, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------- */
/* Sec. 3.1: occupancy queries and ground-truth labels.                     */
/* ---------------------------------------------------------------------- */
/* c (N, may be NULL) = sigmoid(s(x)); s (N, may be NULL) = s(x);
 * grad (N x d, may be NULL) = grad c(x). */
pdmp_status pdmp_occupancy_query(const pdmp_field* f, const float* x, int64_t N, float* c, float* s, float* grad,
                                 void* stream);

/* label[n] = 1 iff x[n] lies in some closed axis-aligned box:
 * lo_j <= x_j <= hi_j on every axis, compared exactly in float32.
 * boxes: nb x 2d (lo_0..lo_{d-1}, hi_0..hi_{d-1}); nb >= 0; 1 <= d <= 8. */
pdmp_status pdmp_box_labels(int32_t d, const float* boxes, int64_t nb, const float* x, int64_t N, uint8_t* label,
                            void* stream);

/* ---------------------------------------------------------------------- */
/* Sec. 3.2: a certified Lipschitz constant of grad c, which sets eta < 1/L. */
/* ---------------------------------------------------------------------- */
/* Computed in FP64 on the device, then copied to the host (this call
 * synchronises `stream`; calls from several host threads are serialised).
 *   |Hess c| <= |Hess s| / 4 + |grad s|^2 / (6 sqrt 3).
 * RBF: |grad phi_m| and |Hess phi_m| are radial functions of r = |x - mu_m|;
 * the box [lo, hi] (host, d doubles each) is cut into cells^d cells, each
 * radial factor is replaced by its maximum over the cell's range of r, and the
 * bound is the maximum over cells.  1 <= cells and cells^d <= 2^24.
 * RFF: |grad phi_m| <= |omega_m|, |Hess phi_m| <= |omega_m|^2 everywhere;
 * lo, hi and cells are ignored.
 * L (host) receives the bound on |Hess c|_2, G (host, may be NULL) a bound
 * on |grad c|_2 over the same region. */
pdmp_status pdmp_lipschitz_bound(const pdmp_field* f, const double* lo, const double* hi, int32_t cells, double* L,
                                 double* G, void* stream);

/* ---------------------------------------------------------------------- */
/* Sec. 3.1: fit the weights to labelled occupancy points (BCE, gradient     */
/* descent).                                                                */
/* ---------------------------------------------------------------------- */
/* Minimises mean_i BCE(sigmoid(s(X_i)), y_i) + (l2 / 2) |w|^2 over w and the
 * bias, starting from zero.  The step is alpha = 1 / (lambda / 4 + l2), where
 * lambda estimates the top eigenvalue of (1/n) [Phi 1]^T [Phi 1] by
 * power_iters power iterations from the normalised all-ones vector; then
 * `iters` Nesterov iterations  v = w_k + (k-1)/(k+2) (w_k - w_{k-1}),
 * w_{k+1} = v - alpha grad(v).
 * f gives kind, d, M, centres, phase and gamma; f->w and f->bias are ignored.
 * X: n x d points, y: n labels in {0, 1}.  w_out: M (device).  bias_out,
 * loss_out (final objective), alpha_out: host, each may be NULL; when any is
 * given the call synchronises `stream`.
 * ws must hold pdmp_fit_workspace(M, n) bytes. */
size_t pdmp_fit_workspace(int64_t M, int64_t n);
pdmp_status pdmp_fit_occupancy(const pdmp_field* f, const float* X, const uint8_t* y, int64_t n, float l2,
                               int32_t power_iters, int32_t iters, float* w_out, float* bias_out, float* loss_out,
                               float* alpha_out, void* ws, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PDMP_H */
