// Occupancy fit (Sec. 3.1): binary cross entropy between sigmoid(s(x_i)) and
// the labels y_i, plus (l2/2)|w|^2, minimised by gradient descent -- here a
// power-iteration step size followed by Nesterov-accelerated iterations.
// The bias is handled as a last weight whose feature is the constant 1 and
// which is not regularised.
//
// Every reduction runs in a fixed order (per-block partials, then one block),
// so a fit is bit-reproducible.
#include "field.cuh"
#include "kernels.cuh"

namespace pdmp {

constexpr int kFitThreads = 128;
constexpr int kFitTile = 256;        // centres per smem tile (forward)
constexpr int kFitChunk = 4096;      // samples per block (transposed pass)
constexpr int kFitSampleTile = 512;  // samples per smem tile (transposed pass)

struct FitWs {
  float* logits;   // n
  float* resid;    // n
  float* v;        // M + 1   power-iteration vector / Nesterov extrapolation
  float* av;       // M + 1
  float* w;        // M + 1   iterate
  float* wprev;    // M + 1
  float* partial;  // chunks x (M + 1)
  double* scal;    // [0] lambda, [1] alpha, [2] loss, [3] norm
  double* bpart;   // per-block partials of the sample reductions
  int64_t chunks;
  int64_t nblk;    // blocks of the per-sample kernels
};

static int64_t fit_chunks(int64_t n) { return (n + kFitChunk - 1) / kFitChunk; }
static int64_t fit_nblk(int64_t n) { return (n + kFitThreads - 1) / kFitThreads; }
static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

size_t fit_workspace(int64_t M, int64_t n) {
  size_t b = 0;
  b += align256(sizeof(float) * n) * 2;
  b += align256(sizeof(float) * (M + 1)) * 4;
  b += align256(sizeof(float) * (M + 1) * fit_chunks(n));
  b += align256(sizeof(double) * 8);
  b += align256(sizeof(double) * 2 * fit_nblk(n));
  return b;
}

static FitWs carve(void* ws, int64_t M, int64_t n) {
  FitWs f;
  char* p = (char*)ws;
  auto take = [&](size_t bytes) { char* q = p; p += align256(bytes); return q; };
  f.logits = (float*)take(sizeof(float) * n);
  f.resid = (float*)take(sizeof(float) * n);
  f.v = (float*)take(sizeof(float) * (M + 1));
  f.av = (float*)take(sizeof(float) * (M + 1));
  f.w = (float*)take(sizeof(float) * (M + 1));
  f.wprev = (float*)take(sizeof(float) * (M + 1));
  f.chunks = fit_chunks(n);
  f.partial = (float*)take(sizeof(float) * (M + 1) * f.chunks);
  f.scal = (double*)take(sizeof(double) * 8);
  f.nblk = fit_nblk(n);
  f.bpart = (double*)take(sizeof(double) * 2 * f.nblk);
  return f;
}

// unweighted feature value (RBF: exp(-gamma r^2) = 2^{ngl2e r^2}; RFF: cos(theta))
template <int KIND, int D>
__device__ __forceinline__ float feat(const float* c, float ph, const float* x, float ngl2e) {
  if (KIND == PDMP_KIND_RBF) {
    float r2 = 0.0f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      float dx = x[j] - c[j];
      r2 = fmaf(dx, dx, r2);
    }
    return ex2_approx(r2 * ngl2e);
  } else {
    float th = ph;
#pragma unroll
    for (int j = 0; j < D; ++j) th = fmaf(c[j], x[j], th);
    return cos_approx(reduce_2pi(th));
  }
}

// out[i] = sum_m v[m] phi_m(x_i) + v[M]
template <int KIND, int D>
__global__ void __launch_bounds__(kFitThreads)
k_fit_forward(FieldArgs g, const float* __restrict__ X, int64_t n, const float* __restrict__ v,
              float* __restrict__ out) {
  __shared__ float sc[kFitTile * (D + 2)];
  const float ngl2e = -g.gamma * kLog2e;
  const int64_t i = (int64_t)blockIdx.x * kFitThreads + threadIdx.x;
  float x[D];
#pragma unroll
  for (int j = 0; j < D; ++j) x[j] = i < n ? X[i * D + j] : 0.0f;
  float acc = 0.0f;
  for (int64_t m0 = 0; m0 < g.M; m0 += kFitTile) {
    __syncthreads();
    const int cnt = (int)min64(kFitTile, g.M - m0);
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
#pragma unroll
      for (int j = 0; j < D; ++j) sc[q * (D + 2) + j] = g.centres[(m0 + q) * D + j];
      sc[q * (D + 2) + D] = KIND == PDMP_KIND_RFF ? g.phase[m0 + q] : 0.0f;
      sc[q * (D + 2) + D + 1] = v[m0 + q];
    }
    __syncthreads();
    for (int q = 0; q < cnt; ++q) {
      const float* c = sc + q * (D + 2);
      acc = fmaf(c[D + 1], feat<KIND, D>(c, c[D], x, ngl2e), acc);
    }
  }
  if (i < n) out[i] = acc + v[g.M];
}

// partial[chunk][m] = sum_{i in chunk} r[i] phi_m(x_i); partial[chunk][M] = sum r[i]
template <int KIND, int D>
__global__ void __launch_bounds__(kFitThreads)
k_fit_backward(FieldArgs g, const float* __restrict__ X, int64_t n, const float* __restrict__ r,
               float* __restrict__ partial) {
  __shared__ float sx[kFitSampleTile * (D + 1)];
  const float ngl2e = -g.gamma * kLog2e;
  const int64_t m = (int64_t)blockIdx.x * kFitThreads + threadIdx.x;
  const int64_t chunk = blockIdx.y;
  const int64_t i0 = chunk * kFitChunk, i1 = min64(n, i0 + kFitChunk);
  float c[D], ph = 0.0f;
  const bool is_bias = (m == g.M);
#pragma unroll
  for (int j = 0; j < D; ++j) c[j] = m < g.M ? g.centres[m * D + j] : 0.0f;
  if (KIND == PDMP_KIND_RFF && m < g.M) ph = g.phase[m];
  float acc = 0.0f;
  for (int64_t s0 = i0; s0 < i1; s0 += kFitSampleTile) {
    __syncthreads();
    const int cnt = (int)min64(kFitSampleTile, i1 - s0);
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
#pragma unroll
      for (int j = 0; j < D; ++j) sx[q * (D + 1) + j] = X[(s0 + q) * D + j];
      sx[q * (D + 1) + D] = r[s0 + q];
    }
    __syncthreads();
    if (m < g.M) {
      for (int q = 0; q < cnt; ++q) acc = fmaf(sx[q * (D + 1) + D], feat<KIND, D>(c, ph, sx + q * (D + 1), ngl2e), acc);
    } else if (is_bias) {
      for (int q = 0; q < cnt; ++q) acc += sx[q * (D + 1) + D];
    }
  }
  if (m <= g.M) partial[chunk * (g.M + 1) + m] = acc;
}

// residual r_i = sigmoid(l_i) - y_i (or, in power-iteration mode, r_i = l_i);
// per-block partial sums of the BCE terms softplus(l) - y l.
__global__ void __launch_bounds__(kFitThreads)
k_fit_residual(const float* __restrict__ logits, const uint8_t* __restrict__ y, int64_t n, int power_mode,
               float* __restrict__ r, double* __restrict__ bpart) {
  __shared__ double sred[kFitThreads];
  const int64_t i = (int64_t)blockIdx.x * kFitThreads + threadIdx.x;
  double term = 0.0;
  if (i < n) {
    float l = logits[i];
    if (power_mode) {
      r[i] = l;
    } else {
      float yi = y[i] ? 1.0f : 0.0f;
      r[i] = sigmoid_f(l) - yi;
      double ld = (double)l;
      double sp = ld > 0 ? ld + log1p(exp(-ld)) : log1p(exp(ld));
      term = sp - (double)yi * ld;
    }
  }
  sred[threadIdx.x] = term;
  __syncthreads();
  for (int o = kFitThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sred[threadIdx.x] += sred[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) bpart[blockIdx.x] = sred[0];
}

// out[m] = (sum_chunks partial[.][m]) / n (+ l2 * v[m] for m < M when add_l2)
__global__ void k_fit_reduce(const float* __restrict__ partial, int64_t chunks, int64_t M, double inv_n, float l2,
                             const float* __restrict__ v, int add_l2, float* __restrict__ out) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m > M) return;
  double acc = 0.0;
  for (int64_t c = 0; c < chunks; ++c) acc += (double)partial[c * (M + 1) + m];
  float val = (float)(acc * inv_n);
  if (add_l2 && m < M) val = fmaf(l2, v[m], val);
  out[m] = val;
}

// single block: scal[which] = |a| (which = 3) after normalising v = a / |a|, lambda = |a|
__global__ void __launch_bounds__(1024) k_fit_normalise(float* __restrict__ a, int64_t len, float* __restrict__ v,
                                                         double* __restrict__ scal, float l2) {
  __shared__ double sred[1024];
  double acc = 0.0;
  for (int64_t m = threadIdx.x; m < len; m += blockDim.x) acc += (double)a[m] * (double)a[m];
  sred[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sred[threadIdx.x] += sred[threadIdx.x + o];
    __syncthreads();
  }
  double nrm = sqrt(sred[0]);
  if (nrm > 0.0)
    for (int64_t m = threadIdx.x; m < len; m += blockDim.x) v[m] = (float)((double)a[m] / nrm);
  if (threadIdx.x == 0) {
    scal[0] = nrm;
    scal[1] = 1.0 / (0.25 * nrm + (double)l2);
  }
}

// single block: scal[2] = sum(bpart) / n + (l2/2) |w[0..M)|^2
__global__ void __launch_bounds__(1024) k_fit_loss(const double* __restrict__ bpart, int64_t nblk,
                                                    const float* __restrict__ w, int64_t M, double inv_n, float l2,
                                                    double* __restrict__ scal) {
  __shared__ double s1[1024], s2[1024];
  double a = 0.0, b = 0.0;
  for (int64_t q = threadIdx.x; q < nblk; q += blockDim.x) a += bpart[q];
  for (int64_t m = threadIdx.x; m < M; m += blockDim.x) b += (double)w[m] * (double)w[m];
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double loss = s1[0] * inv_n + 0.5 * (double)l2 * s2[0];
    scal[2] = loss;
    if (!isfinite(loss)) raise_flag(FLAG_FIT_NONFINITE);
  }
}

__global__ void k_fill(float* p, int64_t len, float v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) p[i] = v;
}

// v = w + beta (w - wprev)
__global__ void k_nesterov_extrapolate(const float* __restrict__ w, const float* __restrict__ wprev, int64_t len,
                                       float beta, float* __restrict__ v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) v[i] = fmaf(beta, w[i] - wprev[i], w[i]);
}
// wprev = w; w = v - alpha g
__global__ void k_nesterov_step(float* __restrict__ w, float* __restrict__ wprev, const float* __restrict__ v,
                                const float* __restrict__ g, int64_t len, const double* __restrict__ scal) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) {
    float alpha = (float)scal[1];
    wprev[i] = w[i];
    w[i] = fmaf(-alpha, g[i], v[i]);
  }
}

template <int KIND, int D>
static cudaError_t fit_impl(const FieldArgs& geom, const float* X, const uint8_t* y, int64_t n, float l2,
                            int power_iters, int iters, float* w_out, float* bias_out, float* loss_out,
                            float* alpha_out, void* ws, cudaStream_t st) {
  const int64_t M = geom.M, len = M + 1;
  FitWs f = carve(ws, M, n);
  const double inv_n = 1.0 / (double)n;
  const unsigned eb = (unsigned)((len + 255) / 256);
  const unsigned nb = (unsigned)f.nblk;
  const dim3 bgrid((unsigned)((len + kFitThreads - 1) / kFitThreads), (unsigned)f.chunks);
  cudaError_t e;

  // ---- power iteration on (1/n) [Phi 1]^T [Phi 1]
  k_fill<<<eb, 256, 0, st>>>(f.v, len, (float)(1.0 / sqrt((double)len)));
  for (int it = 0; it < power_iters; ++it) {
    k_fit_forward<KIND, D><<<nb, kFitThreads, 0, st>>>(geom, X, n, f.v, f.logits);
    k_fit_residual<<<nb, kFitThreads, 0, st>>>(f.logits, y, n, 1, f.resid, f.bpart);
    k_fit_backward<KIND, D><<<bgrid, kFitThreads, 0, st>>>(geom, X, n, f.resid, f.partial);
    k_fit_reduce<<<eb, 256, 0, st>>>(f.partial, f.chunks, M, inv_n, 0.0f, f.v, 0, f.av);
    k_fit_normalise<<<1, 1024, 0, st>>>(f.av, len, f.v, f.scal, l2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }

  // ---- Nesterov iterations from zero
  cudaMemsetAsync(f.w, 0, sizeof(float) * len, st);
  cudaMemsetAsync(f.wprev, 0, sizeof(float) * len, st);
  for (int k = 1; k <= iters; ++k) {
    float beta = (float)(k - 1) / (float)(k + 2);
    k_nesterov_extrapolate<<<eb, 256, 0, st>>>(f.w, f.wprev, len, beta, f.v);
    k_fit_forward<KIND, D><<<nb, kFitThreads, 0, st>>>(geom, X, n, f.v, f.logits);
    k_fit_residual<<<nb, kFitThreads, 0, st>>>(f.logits, y, n, 0, f.resid, f.bpart);
    k_fit_backward<KIND, D><<<bgrid, kFitThreads, 0, st>>>(geom, X, n, f.resid, f.partial);
    k_fit_reduce<<<eb, 256, 0, st>>>(f.partial, f.chunks, M, inv_n, l2, f.v, 1, f.av);
    k_nesterov_step<<<eb, 256, 0, st>>>(f.w, f.wprev, f.v, f.av, len, f.scal);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }

  // ---- final objective
  k_fit_forward<KIND, D><<<nb, kFitThreads, 0, st>>>(geom, X, n, f.w, f.logits);
  k_fit_residual<<<nb, kFitThreads, 0, st>>>(f.logits, y, n, 0, f.resid, f.bpart);
  k_fit_loss<<<1, 1024, 0, st>>>(f.bpart, f.nblk, f.w, M, inv_n, l2, f.scal);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(w_out, f.w, sizeof(float) * M, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
  if (bias_out || loss_out || alpha_out) {
    float b;
    double sc[3];
    if ((e = cudaMemcpyAsync(&b, f.w + M, sizeof(float), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(sc, f.scal, sizeof(sc), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    if (bias_out) *bias_out = b;
    if (loss_out) *loss_out = (float)sc[2];
    if (alpha_out) *alpha_out = (float)sc[1];
  }
  return cudaSuccess;
}

cudaError_t fit_occupancy(int kind, int d, const FieldArgs& geom, const float* X, const uint8_t* y, int64_t n,
                          float l2, int power_iters, int iters, float* w_out, float* bias_out, float* loss_out,
                          float* alpha_out, void* ws, cudaStream_t st) {
#define PDMP_CASE(KD, DD)                                                                                    \
  if (kind == KD && d == DD)                                                                                 \
    return fit_impl<KD, DD>(geom, X, y, n, l2, power_iters, iters, w_out, bias_out, loss_out, alpha_out, ws, \
                            st);
  PDMP_CASE(PDMP_KIND_RBF, 1) PDMP_CASE(PDMP_KIND_RBF, 2) PDMP_CASE(PDMP_KIND_RBF, 3)
  PDMP_CASE(PDMP_KIND_RFF, 1) PDMP_CASE(PDMP_KIND_RFF, 2) PDMP_CASE(PDMP_KIND_RFF, 3) PDMP_CASE(PDMP_KIND_RFF, 4)
  PDMP_CASE(PDMP_KIND_RFF, 5) PDMP_CASE(PDMP_KIND_RFF, 6) PDMP_CASE(PDMP_KIND_RFF, 7) PDMP_CASE(PDMP_KIND_RFF, 8)
#undef PDMP_CASE
  return cudaErrorInvalidValue;
}

}  // namespace pdmp
