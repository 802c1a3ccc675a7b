// Surrogate inference with the plain morph as fallback and judge (no
// counterpart in the paper; the fallback mirrors the paper's non-blocking
// fall-back to the prior when the morphed samples are not available).
//   1. the MLP predicts x_T for every sample;
//   2. one plain Euler step is evaluated at every prediction (the fast RBF
//      kernel with T = 1, which also reports the logit s), or, with a cut-off
//      radius, the culled kernel's step (features farther than r_cut from a
//      tile dropped, so that s and |grad s| are within the culling bound of
//      the dense ones; it reports s and grad c, and the step is -eta grad c);
//   3. a sample fails when s >= 0 (c >= 1/2: the prediction is in
//      predicted-occupied space), when that step is longer than tau_r, or when
//      either is not finite;
//   4. failed samples are compacted (prefix sum, so in index order), morphed
//      by the plain T-step kernel from their x0, and scattered back.
#include <cstring>

#include "kernels.cuh"
#include "sort.cuh"

namespace pdmp {

__global__ void k_residual_flags(const float* __restrict__ s, const float* __restrict__ steps, int64_t N, int d,
                                 float tau_r2, uint32_t* __restrict__ flags) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float r2 = 0.0f;
  for (int j = 0; j < d; ++j) {
    const float v = steps[n * d + j];
    r2 = fmaf(v, v, r2);
  }
  const float sv = s[n];
  const bool ok = (sv < 0.0f) && (r2 <= tau_r2);     // false for NaN
  flags[n] = ok ? 0u : 1u;
}

// the same from grad c of the checked state (the culled check): the step is -eta grad c
__global__ void k_residual_flags_grad(const float* __restrict__ s, const float* __restrict__ g, int64_t N, int d,
                                      float eta, float tau_r2, uint32_t* __restrict__ flags) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float r2 = 0.0f;
  for (int j = 0; j < d; ++j) {
    const float v = __fmul_rn(eta, g[n * d + j]);
    r2 = fmaf(v, v, r2);
  }
  const float sv = s[n];
  const bool ok = (sv < 0.0f) && (r2 <= tau_r2);     // false for NaN
  flags[n] = ok ? 0u : 1u;
}

__global__ void k_compact(const uint32_t* __restrict__ flags, const uint32_t* __restrict__ offs, int64_t N,
                          int32_t* __restrict__ idx, int64_t* __restrict__ count) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  if (flags[n]) idx[offs[n]] = (int32_t)n;
  if (n == N - 1) *count = (int64_t)offs[n] + flags[n];
}

__global__ void k_gather(const float* __restrict__ x, const int32_t* __restrict__ idx, int64_t n, int d,
                         float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * d) return;
  out[i] = x[(int64_t)idx[i / d] * d + i % d];
}

__global__ void k_scatter_rows(const float* __restrict__ v, const int32_t* __restrict__ idx, int64_t n, int d,
                               float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * d) return;
  out[(int64_t)idx[i / d] * d + i % d] = v[i];
}

struct SurWs {
  float *traj, *steps, *s, *xs, *ys;
  uint32_t *flags, *offs, *chunks;
  int32_t* idx;
  int64_t* count;
  void* fast;
  size_t bytes;
};

static size_t al(size_t b) { return (b + 255) & ~size_t(255); }

static SurWs sur_layout(void* ws, int d, int64_t M, int64_t N) {
  SurWs w;
  char* p = (char*)ws;
  auto take = [&](size_t b) { char* q = p; p += al(b); return q; };
  w.traj = (float*)take(sizeof(float) * 2 * N * d);
  w.steps = (float*)take(sizeof(float) * N * d);
  w.s = (float*)take(sizeof(float) * N);
  w.xs = (float*)take(sizeof(float) * N * d);
  w.ys = (float*)take(sizeof(float) * N * d);
  w.flags = (uint32_t*)take(sizeof(uint32_t) * N);
  w.offs = (uint32_t*)take(sizeof(uint32_t) * N);
  w.chunks = (uint32_t*)take(sizeof(uint32_t) * ((N + kScanChunk - 1) / kScanChunk + 1));
  w.idx = (int32_t*)take(sizeof(int32_t) * N);
  w.count = (int64_t*)take(sizeof(int64_t));
  // the fast kernel's workspace, or the culled kernel's for the check (used one after the other)
  const size_t fb = morph_rbf_fast_workspace(d, M, N), cb = morph_rbf_cull_workspace(d, M, N);
  w.fast = take(fb > cb ? fb : cb);
  w.bytes = (size_t)(p - (char*)ws);
  return w;
}

size_t surrogate_workspace(int d, int64_t M, int64_t N) { return sur_layout(nullptr, d, M, N).bytes; }

// rms[j] = sqrt(mean_n (xT[n][j] - x0[n][j])^2), single block, fixed order
__global__ void __launch_bounds__(1024) k_displacement_rms(const float* __restrict__ x0, const float* __restrict__ xT,
                                                            int64_t N, int d, float* __restrict__ rms) {
  __shared__ double sh[1024];
  for (int j = 0; j < d; ++j) {
    double a = 0.0;
    for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
      const double v = (double)xT[n * d + j] - (double)x0[n * d + j];
      a += v * v;
    }
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) rms[j] = (float)sqrt(sh[0] / (double)N);
    __syncthreads();
  }
}

cudaError_t displacement_rms(const float* x0, const float* xT, int64_t N, int d, float* rms, cudaStream_t st) {
  k_displacement_rms<<<1, 1024, 0, st>>>(x0, xT, N, d, rms);
  return cudaGetLastError();
}

cudaError_t surrogate_infer(const pdmp_mlp* net, int d, const FieldArgs& fa, const float* x0, int64_t N, int T,
                            float eta, float tau_r, float r_cut, float* xT, int64_t* n_fallback, void* ws,
                            cudaStream_t st) {
  *n_fallback = 0;
  if (N == 0) return cudaSuccess;
  SurWs w = sur_layout(ws, d, fa.M, N);
  cudaError_t e;
  if ((e = mlp_forward(net, x0, N, xT, false, st))) return e;
  if (T == 0) return cudaSuccess;
  const unsigned nb = (unsigned)((N + 255) / 256);
  if (r_cut > 0.0f) {
    // one culled step at every prediction: s = its logit, steps = grad c there (the step is -eta grad c)
    if ((e = morph_rbf_cull(d, fa, xT, N, 1, eta, r_cut, w.traj, nullptr, 0, w.fast, nullptr, st, w.s, w.steps)))
      return e;
    k_residual_flags_grad<<<nb, 256, 0, st>>>(w.s, w.steps, N, d, eta, tau_r * tau_r, w.flags);
  } else {
    // one plain step at every prediction: traj[0] = prediction, steps[0] = its increment, s = its logit
    if ((e = morph_rbf_fast(d, fa, xT, N, 1, eta, nullptr, nullptr, 0, w.traj, w.steps, w.fast, st, w.s))) return e;
    k_residual_flags<<<nb, 256, 0, st>>>(w.s, w.steps, N, d, tau_r * tau_r, w.flags);
  }
  if ((e = exclusive_scan_u32(w.flags, N, w.offs, w.chunks, st))) return e;
  k_compact<<<nb, 256, 0, st>>>(w.flags, w.offs, N, w.idx, w.count);
  int64_t cnt = 0;
  if ((e = cudaMemcpyAsync(&cnt, w.count, sizeof(int64_t), cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaStreamSynchronize(st))) return e;
  *n_fallback = cnt;
  if (cnt == 0) return cudaGetLastError();
  const unsigned gb = (unsigned)((cnt * d + 255) / 256);
  k_gather<<<gb, 256, 0, st>>>(x0, w.idx, cnt, d, w.xs);
  // the fallback: the plain morph of the failed samples, culled like the
  // check when r_cut > 0
  if (r_cut > 0.0f)
    e = morph_rbf_cull(d, fa, w.xs, cnt, T, eta, r_cut, w.ys, nullptr, 0, w.fast, nullptr, st);
  else
    e = morph_rbf_fast(d, fa, w.xs, cnt, T, eta, w.ys, nullptr, 0, nullptr, nullptr, w.fast, st);
  if (e) return e;
  k_scatter_rows<<<gb, 256, 0, st>>>(w.ys, w.idx, cnt, d, xT);
  return cudaGetLastError();
}

// ------------------------------------------------------------ threshold
// tau_r: a quantile of the plain morph's last-step length over training
// samples.  The k-th smallest length is found exactly by a two-pass radix
// select on the float bits (non-negative floats order like their bit
// patterns; NaN lengths count as the largest): a histogram of the high 16 bits
// locates the bin holding rank k, a histogram of the low 16 bits within that
// bin the value.  Integer work only, so the result is reproducible.
constexpr int kSelBins = 1 << 16;

__global__ void k_step_length_keys(const float* __restrict__ steps, int64_t N, int d, uint32_t* __restrict__ keys,
                                   uint32_t* __restrict__ hist) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float r2 = 0.0f;
  for (int j = 0; j < d; ++j) {
    const float v = steps[n * d + j];
    r2 = fmaf(v, v, r2);
  }
  const float len = sqrtf(r2);
  const uint32_t key = len == len ? __float_as_uint(len) : 0xffffffffu;
  keys[n] = key;
  atomicAdd(&hist[key >> 16], 1u);
}

__global__ void k_select_low_hist(const uint32_t* __restrict__ keys, int64_t N, const uint32_t* __restrict__ sel,
                                  uint32_t* __restrict__ hist) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const uint32_t key = keys[n];
  if ((key >> 16) == sel[0]) atomicAdd(&hist[key & 0xffffu], 1u);
}

// single block of 1024 threads: the bin of hist (kSelBins counts) holding rank
// k (0-based; pass 0: k0, pass 1: sel[1]); sel[0] <- (pass 0) the bin, or
// (pass 1) sel[0] << 16 | bin; sel[1] <- the rank within the bin
__global__ void __launch_bounds__(1024) k_select_bin(uint32_t* __restrict__ hist, uint32_t* __restrict__ sel,
                                                     int pass, uint32_t k0) {
  __shared__ uint32_t sh[33];
  constexpr int per = kSelBins / 1024;
  const int base = threadIdx.x * per;
  uint32_t local = 0;
  for (int i = 0; i < per; ++i) local += hist[base + i];
  // block exclusive scan of the per-thread totals
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = sh[lane];
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += v;
    }
    sh[lane] = wi - w;
  }
  __syncthreads();
  const uint32_t before = inc - local + sh[warp];
  const uint32_t k = pass == 0 ? k0 : sel[1];
  __syncthreads();
  if (k >= before && k < before + local) {
    uint32_t c = before;
    for (int i = 0; i < per; ++i) {
      const uint32_t h = hist[base + i];
      if (k < c + h) {
        sel[0] = pass == 0 ? (uint32_t)(base + i) : ((sel[0] << 16) | (uint32_t)(base + i));
        sel[1] = k - c;
        break;
      }
      c += h;
    }
  }
}

struct ThrWs {
  float *xprev, *traj, *steps;
  uint32_t *keys, *hist, *sel;
  void* fast;
  size_t bytes;
};

static ThrWs thr_layout(void* ws, int d, int64_t M, int64_t N) {
  ThrWs w;
  char* p = (char*)ws;
  auto take = [&](size_t b) { char* q = p; p += al(b); return q; };
  w.xprev = (float*)take(sizeof(float) * N * d);
  w.traj = (float*)take(sizeof(float) * 2 * N * d);
  w.steps = (float*)take(sizeof(float) * N * d);
  w.keys = (uint32_t*)take(sizeof(uint32_t) * N);
  w.hist = (uint32_t*)take(sizeof(uint32_t) * kSelBins);
  w.sel = (uint32_t*)take(sizeof(uint32_t) * 4);
  w.fast = take(morph_rbf_fast_workspace(d, M, N));
  w.bytes = (size_t)(p - (char*)ws);
  return w;
}

size_t residual_threshold_workspace(int d, int64_t M, int64_t N) { return thr_layout(nullptr, d, M, N).bytes; }

cudaError_t residual_threshold(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, int64_t k,
                               float* tau_r, float* xT, void* ws, cudaStream_t st) {
  ThrWs w = thr_layout(ws, d, fa.M, N);
  cudaError_t e;
  if (T > 1) {
    if ((e = morph_rbf_fast(d, fa, x0, N, T - 1, eta, w.xprev, nullptr, 0, nullptr, nullptr, w.fast, st))) return e;
  } else if ((e = cudaMemcpyAsync(w.xprev, x0, sizeof(float) * N * d, cudaMemcpyDeviceToDevice, st))) {
    return e;
  }
  // the last step, traced: traj[1] = x_T, steps[0] = its FP32 increment
  if ((e = morph_rbf_fast(d, fa, w.xprev, N, 1, eta, nullptr, nullptr, 0, w.traj, w.steps, w.fast, st))) return e;
  if (xT && (e = cudaMemcpyAsync(xT, w.traj + N * d, sizeof(float) * N * d, cudaMemcpyDeviceToDevice, st))) return e;
  if ((e = cudaMemsetAsync(w.hist, 0, sizeof(uint32_t) * kSelBins, st))) return e;
  const unsigned nb = (unsigned)((N + 255) / 256);
  k_step_length_keys<<<nb, 256, 0, st>>>(w.steps, N, d, w.keys, w.hist);
  k_select_bin<<<1, 1024, 0, st>>>(w.hist, w.sel, 0, (uint32_t)k);
  if ((e = cudaMemsetAsync(w.hist, 0, sizeof(uint32_t) * kSelBins, st))) return e;
  k_select_low_hist<<<nb, 256, 0, st>>>(w.keys, N, w.sel, w.hist);
  k_select_bin<<<1, 1024, 0, st>>>(w.hist, w.sel, 1, 0u);
  uint32_t bits = 0;
  if ((e = cudaMemcpyAsync(&bits, w.sel, sizeof(uint32_t), cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaStreamSynchronize(st))) return e;
  memcpy(tau_r, &bits, sizeof(float));
  return cudaGetLastError();
}

}  // namespace pdmp
