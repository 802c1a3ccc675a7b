// extern "C" entry points of libpdmp: argument validation on the host, then
// the launchers in the other translation units.  Nothing here computes.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <chrono>
#include <mutex>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kernels.cuh"

namespace pdmp {
__device__ int32_t g_device_flag = 0;
__device__ double g_abs_weight_sum = 0.0;
}

using namespace pdmp_host;

namespace pdmp_host {

pdmp_status check_field(const pdmp_field* f) {
  if (f == nullptr) return PDMP_ERR_INVALID_ARG;
  if (f->M < 1) return PDMP_ERR_INVALID_ARG;
  if (f->kind == PDMP_KIND_RBF) {
    if (f->d < 1 || f->d > 3) return PDMP_ERR_INVALID_ARG;
    if (!(f->gamma > 0.0f) || !std::isfinite(f->gamma)) return PDMP_ERR_INVALID_ARG;
    if (f->phase != nullptr) return PDMP_ERR_INVALID_ARG;
  } else if (f->kind == PDMP_KIND_RFF) {
    if (f->d < 1 || f->d > 8) return PDMP_ERR_INVALID_ARG;
    if (!ok_ptr(f->phase, true)) return PDMP_ERR_INVALID_ARG;
  } else {
    return PDMP_ERR_INVALID_ARG;
  }
  if (!ok_ptr(f->centres, true) || !ok_ptr(f->w, true)) return PDMP_ERR_INVALID_ARG;
  if (!std::isfinite(f->bias)) return PDMP_ERR_INVALID_ARG;
  if (f->lipschitz < 0.0 || std::isnan(f->lipschitz)) return PDMP_ERR_INVALID_ARG;
  return PDMP_OK;
}

pdmp_status check_step(const pdmp_field* f, float eta) {
  if (!(eta > 0.0f) || !std::isfinite(eta)) return PDMP_ERR_INVALID_ARG;
  if (f->lipschitz > 0.0 && (double)eta * f->lipschitz >= 1.0) return PDMP_ERR_STEP_TOO_LARGE;
  return PDMP_OK;
}

}  // namespace pdmp_host

// the bound and radius calls reduce into fixed device slots of the library and
// synchronise before they return; this lock serialises them across host threads
static std::mutex g_slot_lock;

// an NVTX range around a boundary call (visible to ncu's --nvtx filters)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

static pdmp::FieldArgs field_args(const pdmp_field* f) {
  pdmp::FieldArgs a;
  a.centres = f->centres;
  a.phase = f->phase;
  a.w = f->w;
  a.M = f->M;
  a.gamma = f->gamma;
  a.bias = f->bias;
  return a;
}

static inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

extern "C" {

const char* pdmp_status_string(pdmp_status s) {
  switch (s) {
    case PDMP_OK: return "ok";
    case PDMP_ERR_INVALID_ARG: return "invalid argument";
    case PDMP_ERR_STEP_TOO_LARGE: return "step too large: eta * L >= 1 breaks the diffeomorphism";
    case PDMP_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case PDMP_ERR_CUDA: return "CUDA runtime error";
    case PDMP_ERR_NOT_CONVERGED: return "not converged";
    case PDMP_ERR_TIMEOUT: return "timed out";
    case PDMP_ERR_DEVICE_FLAG: return "a kernel recorded a numerical failure";
    case PDMP_ERR_UNSUPPORTED: return "unsupported by this library version";
    default: return "unknown status";
  }
}

int32_t pdmp_version(void) { return 200; }   // 0.2.0: the inverse, log-density and log-det take a workspace

pdmp_status pdmp_stream_status(void* stream, int32_t* detail) {
  cudaStream_t st = as_stream(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    if (detail) *detail = (int32_t)e;
    return PDMP_ERR_CUDA;
  }
  int32_t flag = 0, zero = 0;
  e = cudaMemcpyFromSymbolAsync(&flag, pdmp::g_device_flag, sizeof(flag), 0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(pdmp::g_device_flag, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    if (detail) *detail = (int32_t)e;
    return PDMP_ERR_CUDA;
  }
  if (detail) *detail = flag;
  return flag ? PDMP_ERR_DEVICE_FLAG : PDMP_OK;
}

pdmp_status pdmp_selftest_stage_wait(const float* src, float* dst, int64_t limit_clocks, int32_t with_copy,
                                     void* stream) {
  if (limit_clocks < 1 || limit_clocks > (int64_t(1) << 31)) return PDMP_ERR_INVALID_ARG;
  if (with_copy && (!ok_ptr(src, true) || !ok_ptr(dst, true) || !aligned16(src))) return PDMP_ERR_INVALID_ARG;
  return cuda_status(pdmp::stage_wait_selftest(with_copy ? src : nullptr, with_copy ? dst : nullptr,
                                               (long long)limit_clocks, with_copy ? 1 : 0, as_stream(stream)));
}

pdmp_status pdmp_stream_wait(void* stream, int32_t timeout_ms, int32_t* detail) {
  if (timeout_ms < 0) return PDMP_ERR_INVALID_ARG;
  cudaStream_t st = as_stream(stream);
  cudaEvent_t ev = nullptr;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev, st);
  if (e != cudaSuccess) {
    if (ev) cudaEventDestroy(ev);
    if (detail) *detail = (int32_t)e;
    return PDMP_ERR_CUDA;
  }
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  for (;;) {
    e = cudaEventQuery(ev);
    if (e != cudaErrorNotReady) break;
    if (std::chrono::steady_clock::now() >= deadline) {
      cudaEventDestroy(ev);
      if (detail) *detail = 0;
      return PDMP_ERR_TIMEOUT;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  cudaEventDestroy(ev);
  if (e != cudaSuccess) {
    if (detail) *detail = (int32_t)e;
    return PDMP_ERR_CUDA;
  }
  return pdmp_stream_status(stream, detail);   // the work is done: read and clear the device flag
}

size_t pdmp_morph_workspace(const pdmp_field* f, int64_t N) {
  if (f == nullptr || check_field(f) != PDMP_OK || N <= 0) return 0;
  return pdmp::morph_workspace(f->kind, f->d, f->M, N);
}

static pdmp_status check_ws(const pdmp_field* f, int64_t N, void* ws, size_t ws_bytes) {
  if (ws == nullptr) return PDMP_OK;
  if (!aligned16(ws)) return PDMP_ERR_INVALID_ARG;
  // the fast paths index samples through an int32 permutation
  if (N > (int64_t)INT32_MAX && f->kind == PDMP_KIND_RBF && pdmp::morph_workspace(f->kind, f->d, f->M, 1) > 0)
    return PDMP_ERR_INVALID_ARG;
  if (ws_bytes < pdmp::morph_workspace(f->kind, f->d, f->M, N)) return PDMP_ERR_WORKSPACE_TOO_SMALL;
  return PDMP_OK;
}

pdmp_status pdmp_morph(const pdmp_field* f, const float* x0, int64_t N, int32_t T, float eta, float* xT,
                       float* ckpt, int32_t k, void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("pdmp_morph");
  pdmp_status s = check_field(f);
  if (s != PDMP_OK) return s;
  if ((s = check_step(f, eta)) != PDMP_OK) return s;
  if (N < 0 || T < 0) return PDMP_ERR_INVALID_ARG;
  if (ckpt != nullptr && (k < 1 || T % k != 0)) return PDMP_ERR_INVALID_ARG;
  if (N == 0) return PDMP_OK;
  if (!ok_ptr(x0, true) || !ok_ptr(xT, true) || !ok_ptr(ckpt, false)) return PDMP_ERR_INVALID_ARG;
  if ((s = check_ws(f, N, ws, ws_bytes)) != PDMP_OK) return s;
  cudaStream_t st = as_stream(stream);
  if (T == 0) {
    if (xT != x0) return cuda_status(cudaMemcpyAsync(xT, x0, sizeof(float) * N * f->d, cudaMemcpyDeviceToDevice, st));
    return PDMP_OK;
  }
  return cuda_status(pdmp::morph_dispatch(f->kind, f->d, field_args(f), x0, N, T, eta, xT, ckpt, k, nullptr,
                                          nullptr, ws, st));
}

static pdmp_status check_chain(const pdmp_chain* c) {
  if (c == nullptr || c->n < 1 || c->n > pdmp::kChainMax || c->p < 1 || c->p > 8) return PDMP_ERR_INVALID_ARG;
  if (!std::isfinite(c->base[0]) || !std::isfinite(c->base[1])) return PDMP_ERR_INVALID_ARG;
  for (int k = 0; k < c->n; ++k)
    if (!(c->lengths[k] >= 0.0f) || !std::isfinite(c->lengths[k])) return PDMP_ERR_INVALID_ARG;
  return PDMP_OK;
}

size_t pdmp_cspace_workspace(const pdmp_field* f, const pdmp_chain* chain, int64_t N) {
  if (check_field(f) != PDMP_OK || check_chain(chain) != PDMP_OK || f->d != 2 || N <= 0) return 0;
  return pdmp::cspace_workspace(f->d, f->M, chain->n, chain->p, N);
}

pdmp_status pdmp_cspace_morph(const pdmp_field* f, const pdmp_chain* chain, const float* q0, int64_t N, int32_t T,
                              float eta, float* qT, void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("pdmp_cspace_morph");
  pdmp_status s = check_field(f);
  if (s != PDMP_OK) return s;
  if ((s = check_chain(chain)) != PDMP_OK) return s;
  if (f->d != 2) return PDMP_ERR_UNSUPPORTED;
  if (!(eta > 0.0f) || !std::isfinite(eta) || N < 0 || T < 0) return PDMP_ERR_INVALID_ARG;
  if (N == 0) return PDMP_OK;
  if (N > (int64_t)INT32_MAX / (chain->n * chain->p)) return PDMP_ERR_INVALID_ARG;   // body points index the sort
  if (!ok_ptr(q0, true) || !ok_ptr(qT, true) || !ok_ptr(ws, true)) return PDMP_ERR_INVALID_ARG;
  if (ws_bytes < pdmp::cspace_workspace(f->d, f->M, chain->n, chain->p, N)) return PDMP_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = as_stream(stream);
  if (T == 0) {
    if (qT != q0) return cuda_status(cudaMemcpyAsync(qT, q0, sizeof(float) * N * chain->n, cudaMemcpyDeviceToDevice, st));
    return PDMP_OK;
  }
  return cuda_status(pdmp::cspace_morph(field_args(f), f->kind, chain->n, chain->p, chain->base, chain->lengths, q0, N,
                                        T, eta, qT, ws, st));
}

pdmp_status pdmp_cspace_lipschitz(const pdmp_chain* chain, double Lx, double Gx, double* Lq) {
  pdmp_status s = check_chain(chain);
  if (s != PDMP_OK) return s;
  if (Lq == nullptr || !(Lx >= 0.0) || !(Gx >= 0.0) || !std::isfinite(Lx) || !std::isfinite(Gx))
    return PDMP_ERR_INVALID_ARG;
  const int n = chain->n, p = chain->p;
  double total = 0.0;
  for (int k = 0; k < n; ++k) {
    for (int r = 1; r <= p; ++r) {
      // reach[j]: chain length from joint j to this body point
      double reach[pdmp::kChainMax];
      double acc = (double)r / p * chain->lengths[k];
      for (int j = k; j >= 0; --j) {
        reach[j] = acc;
        if (j > 0) acc += chain->lengths[j - 1];
      }
      double jac2 = 0.0, hess2 = 0.0;
      for (int j = 0; j <= k; ++j) {
        jac2 += reach[j] * reach[j];
        for (int m = 0; m <= k; ++m) {
          const double rr = reach[std::max(j, m)];
          hess2 += rr * rr;
        }
      }
      total += jac2 * Lx + Gx * std::sqrt(hess2);
    }
  }
  *Lq = total;
  return PDMP_OK;
}

static pdmp_status check_net(const pdmp_tanh_net* n) {
  if (n == nullptr) return PDMP_ERR_INVALID_ARG;
  if (n->d < 1 || n->d > 8 || n->H < 1 || n->H > 1024) return PDMP_ERR_INVALID_ARG;
  if (!ok_ptr(n->W1, true) || !ok_ptr(n->b1, true) || !ok_ptr(n->W2, true) || !ok_ptr(n->b2, true) ||
      !ok_ptr(n->w3, true))
    return PDMP_ERR_INVALID_ARG;
  if (!std::isfinite(n->b3) || n->lipschitz < 0.0 || std::isnan(n->lipschitz)) return PDMP_ERR_INVALID_ARG;
  if (!((n->d == 2 || n->d == 3) && (n->H == 32 || n->H == 64))) return PDMP_ERR_UNSUPPORTED;
  return PDMP_OK;
}

static pdmp::TanhNetArgs net_args(const pdmp_tanh_net* n) {
  pdmp::TanhNetArgs a;
  a.d = n->d;
  a.H = n->H;
  a.W1 = n->W1;
  a.b1 = n->b1;
  a.W2 = n->W2;
  a.b2 = n->b2;
  a.w3 = n->w3;
  a.b3 = n->b3;
  return a;
}

pdmp_status pdmp_tanh_net_morph(const pdmp_tanh_net* net, const float* x0, int64_t N, int32_t T, float eta,
                                float* xT, float* ckpt, int32_t k, void* stream) {
  NvtxRange nvtx_range("pdmp_tanh_net_morph");
  pdmp_status s = check_net(net);
  if (s != PDMP_OK) return s;
  if (!(eta > 0.0f) || !std::isfinite(eta)) return PDMP_ERR_INVALID_ARG;
  if (net->lipschitz > 0.0 && (double)eta * net->lipschitz >= 1.0) return PDMP_ERR_STEP_TOO_LARGE;
  if (N < 0 || T < 0) return PDMP_ERR_INVALID_ARG;
  if (ckpt != nullptr && (k < 1 || T % k != 0)) return PDMP_ERR_INVALID_ARG;
  if (N == 0) return PDMP_OK;
  if (!ok_ptr(x0, true) || !ok_ptr(xT, true) || !ok_ptr(ckpt, false)) return PDMP_ERR_INVALID_ARG;
  cudaStream_t st = as_stream(stream);
  if (T == 0) {
    if (xT != x0) return cuda_status(cudaMemcpyAsync(xT, x0, sizeof(float) * N * net->d, cudaMemcpyDeviceToDevice, st));
    return PDMP_OK;
  }
  return cuda_status(pdmp::tanh_net_morph(net_args(net), x0, N, T, eta, xT, ckpt, k, st));
}

pdmp_status pdmp_tanh_net_query(const pdmp_tanh_net* net, const float* x, int64_t N, float* c, float* s_out,
                                float* grad, void* stream) {
  pdmp_status s = check_net(net);
  if (s != PDMP_OK) return s;
  if (N < 0) return PDMP_ERR_INVALID_ARG;
  if (N == 0) return PDMP_OK;
  if (!ok_ptr(x, true) || !ok_ptr(c, false) || !ok_ptr(s_out, false) || !ok_ptr(grad, false))
    return PDMP_ERR_INVALID_ARG;
  return cuda_status(pdmp::tanh_net_query(net_args(net), x, N, c, s_out, grad, as_stream(stream)));
}

// largest eigenvalue of the symmetric n x n matrix a (overwritten) by Jacobi
// rotations, each annihilating the largest off-diagonal entry
static double largest_eigenvalue(std::vector<double>& a, int n) {
  for (int it = 0; it < 50 * n * n; ++it) {
    int p = 0, q = 1;
    double big = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i) {
      diag = std::fmax(diag, std::fabs(a[i * n + i]));
      for (int j = i + 1; j < n; ++j)
        if (std::fabs(a[i * n + j]) > big) {
          big = std::fabs(a[i * n + j]);
          p = i;
          q = j;
        }
    }
    if (n < 2 || big <= 1e-17 * std::fmax(diag, 1e-300)) break;
    const double app = a[p * n + p], aqq = a[q * n + q], apq = a[p * n + q];
    const double phi = 0.5 * std::atan2(2.0 * apq, aqq - app);
    const double c = std::cos(phi), s = std::sin(phi);
    for (int k = 0; k < n; ++k) {
      const double akp = a[k * n + p], akq = a[k * n + q];
      a[k * n + p] = c * akp - s * akq;
      a[k * n + q] = s * akp + c * akq;
    }
    for (int k = 0; k < n; ++k) {
      const double apk = a[p * n + k], aqk = a[q * n + k];
      a[p * n + k] = c * apk - s * aqk;
      a[q * n + k] = s * apk + c * aqk;
    }
  }
  double m = a[0];
  for (int i = 1; i < n; ++i) m = std::fmax(m, a[i * n + i]);
  return m;
}

// |W|_2 of the rows x cols matrix W (row-major), from W^T W, rounded up
static double spectral(const std::vector<float>& W, int rows, int cols) {
  std::vector<double> g((size_t)cols * cols, 0.0);
  for (int r = 0; r < rows; ++r)
    for (int a = 0; a < cols; ++a)
      for (int b = 0; b < cols; ++b) g[a * cols + b] += (double)W[r * cols + a] * (double)W[r * cols + b];
  return std::sqrt(std::fmax(largest_eigenvalue(g, cols), 0.0) * (1.0 + 1e-12));
}

pdmp_status pdmp_tanh_net_lipschitz(const pdmp_tanh_net* net, double* L, double* G, void* stream) {
  pdmp_status s = check_net(net);
  if (s != PDMP_OK && s != PDMP_ERR_UNSUPPORTED) return s;
  if (L == nullptr) return PDMP_ERR_INVALID_ARG;
  const int d = net->d, H = net->H;
  std::vector<float> W1((size_t)H * d), W2((size_t)H * H), w3(H);
  cudaStream_t st = as_stream(stream);
  cudaError_t e = cudaMemcpyAsync(W1.data(), net->W1, sizeof(float) * W1.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(W2.data(), net->W2, sizeof(float) * W2.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w3.data(), net->w3, sizeof(float) * w3.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  const double n1 = spectral(W1, H, d), n2 = spectral(W2, H, H);
  double w3sq = 0.0, w3inf = 0.0, col = 0.0;
  for (int i = 0; i < H; ++i) {
    w3sq += (double)w3[i] * w3[i];
    w3inf = std::fmax(w3inf, std::fabs((double)w3[i]));
  }
  for (int j = 0; j < H; ++j) {
    double c = 0.0;
    for (int i = 0; i < H; ++i) c += std::fabs((double)W2[i * H + j]) * std::fabs((double)w3[i]);
    col = std::fmax(col, c);
  }
  const double tanh2_max = 4.0 / (3.0 * std::sqrt(3.0));
  const double grad_bound = n1 * n2 * std::sqrt(w3sq);
  const double hess_s = n1 * n1 * tanh2_max * (col + n2 * n2 * w3inf);
  if (G) *G = grad_bound;
  *L = 0.25 * hess_s + grad_bound * grad_bound / (6.0 * std::sqrt(3.0));
  return PDMP_OK;
}

static bool cull_field(const pdmp_field* f) { return f->kind == PDMP_KIND_RBF && (f->d == 2 || f->d == 3); }

size_t pdmp_morph_culled_workspace(const pdmp_field* f, int64_t N) {
  if (f == nullptr || check_field(f) != PDMP_OK || !cull_field(f) || N <= 0) return 0;
  return pdmp::morph_rbf_cull_workspace(f->d, f->M, N);
}

pdmp_status pdmp_morph_culled(const pdmp_field* f, const float* x0, int64_t N, int32_t T, float eta, float r_cut,
                              float* xT, float* ckpt, int32_t k, void* ws, size_t ws_bytes,
                              unsigned long long* work, void* stream) {
  NvtxRange nvtx_range("pdmp_morph_culled");
  pdmp_status s = check_field(f);
  if (s != PDMP_OK) return s;
  if (!cull_field(f)) return PDMP_ERR_UNSUPPORTED;
  if ((s = check_step(f, eta)) != PDMP_OK) return s;
  if (N < 0 || N > (int64_t)INT32_MAX || T < 0 || !(r_cut > 0.0f) || !std::isfinite(r_cut)) return PDMP_ERR_INVALID_ARG;
  if (f->M > (int64_t)INT32_MAX) return PDMP_ERR_INVALID_ARG;
  if (ckpt != nullptr && (k < 1 || T % k != 0)) return PDMP_ERR_INVALID_ARG;
  if (N == 0) return PDMP_OK;
  if (!ok_ptr(x0, true) || !ok_ptr(xT, true) || !ok_ptr(ckpt, false) || !ok_ptr(ws, true) ||
      (reinterpret_cast<uintptr_t>(work) & 7u) != 0)
    return PDMP_ERR_INVALID_ARG;
  if (ws_bytes < pdmp::morph_rbf_cull_workspace(f->d, f->M, N)) return PDMP_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = as_stream(stream);
  if (T == 0) {
    if (xT != x0) return cuda_status(cudaMemcpyAsync(xT, x0, sizeof(float) * N * f->d, cudaMemcpyDeviceToDevice, st));
    return PDMP_OK;
  }
  return cuda_status(pdmp::morph_rbf_cull(f->d, field_args(f), x0, N, T, eta, r_cut, xT, ckpt, k, ws, work, st));
}

pdmp_status pdmp_cull_radius(const pdmp_field* f, float eps, float* r_cut, double* w_abs, void* stream) {
  pdmp_status s = check_field(f);
  if (s != PDMP_OK) return s;
  if (f->kind != PDMP_KIND_RBF) return PDMP_ERR_UNSUPPORTED;
  if (!(eps > 0.0f) || !std::isfinite(eps) || r_cut == nullptr) return PDMP_ERR_INVALID_ARG;
  cudaStream_t st = as_stream(stream);
  std::lock_guard<std::mutex> slot(g_slot_lock);
  double* dsum = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void**)&dsum, pdmp::g_abs_weight_sum);
  if (e == cudaSuccess) e = pdmp::abs_weight_sum(f->w, f->M, dsum, st);
  double W = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&W, dsum, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  if (w_abs) *w_abs = W;
  // smallest r >= 1/sqrt(2 gamma) with W max(1, 2 gamma r) exp(-gamma r^2) <= eps (decreasing there)
  const double g = f->gamma;
  auto bound = [&](double r) { return W * std::fmax(1.0, 2.0 * g * r) * std::exp(-g * r * r); };
  double lo = 1.0 / std::sqrt(2.0 * g), hi = lo;
  if (bound(lo) > (double)eps) {
    while (bound(hi) > (double)eps) hi *= 2.0;
    for (int i = 0; i < 200 && hi - lo > 1e-12 * hi; ++i) {
      const double mid = 0.5 * (lo + hi);
      if (bound(mid) > (double)eps) lo = mid; else hi = mid;
    }
  }
  float r = (float)hi;
  if ((double)r < hi) r = std::nextafter(r, INFINITY);
  *r_cut = r;
  return PDMP_OK;
}

pdmp_status pdmp_morph_trace(const pdmp_field* f, const float* x0, int64_t N, int32_t T, float eta, float* traj,
                             float* steps, void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("pdmp_morph_trace");
  pdmp_status s = check_field(f);
  if (s != PDMP_OK) return s;
  if ((s = check_step(f, eta)) != PDMP_OK) return s;
  if (N < 0 || T < 0) return PDMP_ERR_INVALID_ARG;
  if (N == 0) return PDMP_OK;
  if (!ok_ptr(x0, true) || !ok_ptr(traj, true) || !ok_ptr(steps, T > 0)) return PDMP_ERR_INVALID_ARG;
  if ((s = check_ws(f, N, ws, ws_bytes)) != PDMP_OK) return s;
  cudaStream_t st = as_stream(stream);
  if (T == 0) return cuda_status(cudaMemcpyAsync(traj, x0, sizeof(float) * N * f->d, cudaMemcpyDeviceToDevice, st));
  return cuda_status(pdmp::morph_dispatch(f->kind, f->d, field_args(f), x0, N, T, eta, nullptr, nullptr, 0, traj,
                                          steps, ws, st));
}

pdmp_status pdmp_morph_inverse(const pdmp_field* f, const float* z, int64_t N, int32_t T, float eta, float tol,
                               int32_t maxit, float* y, int32_t* iters, void* ws, size_t ws_bytes,
                               unsigned long long* work, void* stream) {
  NvtxRange nvtx_range("pdmp_morph_inverse");
  pdmp_status s = check_field(f);
  if (s != PDMP_OK) return s;
  if ((s = check_step(f, eta)) != PDMP_OK) return s;
  if (N < 0 || T < 0 || maxit < 1 || !(tol >= 0.0f) || !std::isfinite(tol)) return PDMP_ERR_INVALID_ARG;
  if (N == 0) return PDMP_OK;
  if (!ok_ptr(z, true) || !ok_ptr(y, true) || !ok_ptr(iters, false) || (reinterpret_cast<uintptr_t>(work) & 7u) != 0)
    return PDMP_ERR_INVALID_ARG;
  if ((s = check_ws(f, N, ws, ws_bytes)) != PDMP_OK) return s;
  cudaStream_t st = as_stream(stream);
  if (T == 0) {
    if (y != z) return cuda_status(cudaMemcpyAsync(y, z, sizeof(float) * N * f->d, cudaMemcpyDeviceToDevice, st));
    return PDMP_OK;
  }
  return cuda_status(
      pdmp::morph_inverse(f->kind, f->d, field_args(f), z, N, T, eta, tol, maxit, y, iters, ws, work, st));
}

pdmp_status pdmp_log_density(const pdmp_field* f, const float* z, int64_t N, int32_t T, float eta, const double* lo,
                             const double* hi, float tol, int32_t maxit, float* y, float* log_p, void* ws,
                             size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("pdmp_log_density");
  pdmp_status s = check_field(f);
  if (s != PDMP_OK) return s;
  if ((s = check_step(f, eta)) != PDMP_OK) return s;
  if (N < 0 || T < 0 || maxit < 1 || !(tol >= 0.0f) || !std::isfinite(tol) || !lo || !hi) return PDMP_ERR_INVALID_ARG;
  for (int j = 0; j < f->d; ++j)
    if (!(hi[j] > lo[j]) || !std::isfinite(lo[j]) || !std::isfinite(hi[j])) return PDMP_ERR_INVALID_ARG;
  if (N == 0) return PDMP_OK;
  if (!ok_ptr(z, true) || !ok_ptr(y, true) || !ok_ptr(log_p, true) || y == z) return PDMP_ERR_INVALID_ARG;
  cudaStream_t st = as_stream(stream);
  if ((s = check_ws(f, N, ws, ws_bytes)) != PDMP_OK) return s;
  if (T > 0 && ws != nullptr && f->kind == PDMP_KIND_RBF && (f->d == 2 || f->d == 3)) {
    // one kernel: each step's log-det from the inverse's last fixed-point sweep
    if ((s = cuda_status(pdmp::log_density_rbf_fast(f->d, field_args(f), z, N, T, eta, tol, maxit, y, log_p, nullptr,
                                                    nullptr, ws, st))) != PDMP_OK)
      return s;
    return cuda_status(pdmp::uniform_log_density(y, N, f->d, lo, hi, log_p, st));
  }
  if ((s = pdmp_morph_inverse(f, z, N, T, eta, tol, maxit, y, nullptr, ws, ws_bytes, nullptr, stream)) != PDMP_OK)
    return s;
  if ((s = cuda_status(pdmp::logdet(f->kind, f->d, field_args(f), y, N, T, eta, log_p, nullptr, ws, st))) != PDMP_OK)
    return s;
  return cuda_status(pdmp::uniform_log_density(y, N, f->d, lo, hi, log_p, st));
}

// the tensor-core VJP: RFF fields with d <= 7, segments of at most 16 steps
static bool vjp_mma_eligible(const pdmp_field* f, int32_t k) {
  return f->kind == PDMP_KIND_RFF && f->d <= 7 && k >= 1 && k <= pdmp::kVjpMmaMaxSegment;
}

// the sorted-tile VJP: RBF fields in d = 2, 3, segments of at most 16 steps
static bool vjp_tiles_eligible(const pdmp_field* f, int64_t N, int32_t k) {
  return f->kind == PDMP_KIND_RBF && (f->d == 2 || f->d == 3) && k >= 1 && k <= pdmp::kVjpMmaMaxSegment &&
         N <= (int64_t)INT32_MAX;
}

// the per-block rows of the parameter gradient (any VJP kernel's blocks), rounded to 256 bytes
static size_t vjp_rows_bytes(const pdmp_field* f, int64_t N) {
  int64_t blocks = std::max(pdmp::vjp_blocks(N), pdmp::vjp_rff_mma_blocks(N));
  if (f->kind == PDMP_KIND_RBF && (f->d == 2 || f->d == 3)) blocks = std::max(blocks, pdmp::vjp_rbf_fast_blocks(f->d, N));
  return (sizeof(float) * (size_t)blocks * (size_t)(f->M + 1) + 255) & ~size_t(255);
}

size_t pdmp_morph_vjp_workspace(const pdmp_field* f, int64_t N, int32_t T, int32_t k, int32_t want_param_grad) {
  (void)T;
  if (f == nullptr || N <= 0 || f->M < 1) return 0;
  if (want_param_grad) {
    if (want_param_grad == 1 && vjp_mma_eligible(f, k)) return vjp_rows_bytes(f, N) + pdmp::morph_rff_mma_workspace(f->M);
    if (want_param_grad == 1 && vjp_tiles_eligible(f, N, k))
      return vjp_rows_bytes(f, N) + pdmp::morph_rbf_fast_workspace(f->d, f->M, N);
    return vjp_rows_bytes(f, N);
  }
  if (vjp_mma_eligible(f, k)) return pdmp::morph_rff_mma_workspace(f->M);
  if (vjp_tiles_eligible(f, N, k)) return pdmp::morph_rbf_fast_workspace(f->d, f->M, N);
  return 0;
}

pdmp_status pdmp_morph_vjp(const pdmp_field* f, const float* x0, int64_t N, int32_t T, float eta, int32_t k,
                           const float* ckpt, const float* gT, float* g0, float* gw, float* gbias, void* ws,
                           size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("pdmp_morph_vjp");
  pdmp_status s = check_field(f);
  if (s != PDMP_OK) return s;
  if ((s = check_step(f, eta)) != PDMP_OK) return s;
  if (N < 0 || T < 0 || k < 1 || k > pdmp::kMaxSegment || T % k != 0) return PDMP_ERR_INVALID_ARG;
  if (!ok_ptr(ckpt, false) || !ok_ptr(gw, false) || !ok_ptr(gbias, false)) return PDMP_ERR_INVALID_ARG;
  const bool want = gw != nullptr || gbias != nullptr;
  if (want) {
    // the rows are required; the tensor-core kernel also wants its table after them
    size_t need = N > 0 && f->M >= 1 ? vjp_rows_bytes(f, N) : 0;
    if (need > 0 && (ws == nullptr || !aligned16(ws))) return PDMP_ERR_INVALID_ARG;
    if (ws_bytes < need) return PDMP_ERR_WORKSPACE_TOO_SMALL;
  } else if (ws != nullptr) {
    if (!aligned16(ws)) return PDMP_ERR_INVALID_ARG;
    if (ws_bytes < pdmp_morph_vjp_workspace(f, N, T, k, 0)) return PDMP_ERR_WORKSPACE_TOO_SMALL;
  }
  cudaStream_t st = as_stream(stream);
  if (N > 0) {
    if (!ok_ptr(x0, true) || !ok_ptr(gT, true) || !ok_ptr(g0, true)) return PDMP_ERR_INVALID_ARG;
  }
  if (T == 0) {
    if (N > 0 && g0 != gT) {
      cudaError_t e = cudaMemcpyAsync(g0, gT, sizeof(float) * N * f->d, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return PDMP_ERR_CUDA;
    }
    if (gw) cudaMemsetAsync(gw, 0, sizeof(float) * f->M, st);
    if (gbias) cudaMemsetAsync(gbias, 0, sizeof(float), st);
    return launch_status();
  }
  if (!want && ws != nullptr && N > 0 && vjp_mma_eligible(f, k))
    return cuda_status(pdmp::vjp_rff_mma(f->d, field_args(f), x0, N, T, eta, k, ckpt, gT, g0, nullptr, nullptr,
                                         nullptr, ws, st));
  if (want && N > 0 && vjp_mma_eligible(f, k) && ws_bytes >= pdmp_morph_vjp_workspace(f, N, T, k, 1)) {
    const size_t rows_bytes = vjp_rows_bytes(f, N);
    return cuda_status(pdmp::vjp_rff_mma(f->d, field_args(f), x0, N, T, eta, k, ckpt, gT, g0, (float*)ws, gw, gbias,
                                         (char*)ws + rows_bytes, st));
  }
  if (!want && ws != nullptr && N > 0 && vjp_tiles_eligible(f, N, k))
    return cuda_status(pdmp::vjp_rbf_fast(f->d, field_args(f), x0, N, T, eta, k, ckpt, gT, g0, nullptr, nullptr,
                                          nullptr, ws, st));
  if (want && N > 0 && vjp_tiles_eligible(f, N, k) && ws_bytes >= pdmp_morph_vjp_workspace(f, N, T, k, 1)) {
    const size_t rows_bytes = vjp_rows_bytes(f, N);
    return cuda_status(pdmp::vjp_rbf_fast(f->d, field_args(f), x0, N, T, eta, k, ckpt, gT, g0, (float*)ws, gw, gbias,
                                          (char*)ws + rows_bytes, st));
  }
  return cuda_status(pdmp::morph_vjp(f->kind, f->d, field_args(f), x0, N, T, eta, k, ckpt, gT, g0,
                                     want ? (float*)ws : nullptr, gw, gbias, st));
}

pdmp_status pdmp_logdet(const pdmp_field* f, const float* x0, int64_t N, int32_t T, float eta, float* logdet,
                        float* xT, void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("pdmp_logdet");
  pdmp_status s = check_field(f);
  if (s != PDMP_OK) return s;
  if ((s = check_step(f, eta)) != PDMP_OK) return s;
  if (N < 0 || T < 0) return PDMP_ERR_INVALID_ARG;
  if (N == 0) return PDMP_OK;
  if (!ok_ptr(x0, true) || !ok_ptr(logdet, true) || !ok_ptr(xT, false)) return PDMP_ERR_INVALID_ARG;
  if ((s = check_ws(f, N, ws, ws_bytes)) != PDMP_OK) return s;
  return cuda_status(
      pdmp::logdet(f->kind, f->d, field_args(f), x0, N, T, eta, logdet, xT, ws, as_stream(stream)));
}

pdmp_status pdmp_occupancy_query(const pdmp_field* f, const float* x, int64_t N, float* c, float* s_out, float* grad,
                                 void* stream) {
  NvtxRange nvtx_range("pdmp_occupancy_query");
  pdmp_status s = check_field(f);
  if (s != PDMP_OK) return s;
  if (N < 0) return PDMP_ERR_INVALID_ARG;
  if (N == 0) return PDMP_OK;
  if (!ok_ptr(x, true) || !ok_ptr(c, false) || !ok_ptr(s_out, false) || !ok_ptr(grad, false))
    return PDMP_ERR_INVALID_ARG;
  return cuda_status(pdmp::occupancy_query(f->kind, f->d, field_args(f), x, N, c, s_out, grad, as_stream(stream)));
}

pdmp_status pdmp_box_labels(int32_t d, const float* boxes, int64_t nb, const float* x, int64_t N, uint8_t* label,
                            void* stream) {
  if (d < 1 || d > 8 || nb < 0 || N < 0) return PDMP_ERR_INVALID_ARG;
  if (N == 0) return PDMP_OK;
  if (!ok_ptr(x, true) || !ok_ptr(label, true) || !ok_ptr(boxes, nb > 0)) return PDMP_ERR_INVALID_ARG;
  return cuda_status(pdmp::box_labels(d, boxes, nb, x, N, label, as_stream(stream)));
}

pdmp_status pdmp_lipschitz_bound(const pdmp_field* f, const double* lo, const double* hi, int32_t cells, double* L,
                                 double* G, void* stream) {
  NvtxRange nvtx_range("pdmp_lipschitz_bound");
  pdmp_status s = check_field(f);
  if (s != PDMP_OK) return s;
  if (L == nullptr) return PDMP_ERR_INVALID_ARG;
  if (f->kind == PDMP_KIND_RBF) {
    if (lo == nullptr || hi == nullptr || cells < 1) return PDMP_ERR_INVALID_ARG;
    double ncells = 1.0;
    for (int j = 0; j < f->d; ++j) {
      if (!(hi[j] > lo[j]) || !std::isfinite(lo[j]) || !std::isfinite(hi[j])) return PDMP_ERR_INVALID_ARG;
      ncells *= cells;
    }
    if (ncells > (double)(1 << 24)) return PDMP_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> slot(g_slot_lock);
  return cuda_status(pdmp::lipschitz_bound(f->kind, f->d, field_args(f), lo, hi, cells, L, G, as_stream(stream)));
}

int32_t pdmp_batch_variants(void) { return pdmp::batch_variants(); }

static pdmp_status check_envs(const pdmp_env* envs, int32_t n) {
  if (envs == nullptr || n < 1) return PDMP_ERR_INVALID_ARG;
  int64_t total = 0;
  for (int32_t e = 0; e < n; ++e) {
    const pdmp_env& E = envs[e];
    pdmp_status s = check_field(&E.field);
    if (s != PDMP_OK) return s;
    if (E.field.kind != PDMP_KIND_RBF || (E.field.d != 2 && E.field.d != 3)) return PDMP_ERR_UNSUPPORTED;
    if ((s = check_step(&E.field, E.eta)) != PDMP_OK) return s;
    if (E.N < 0 || E.T < 0) return PDMP_ERR_INVALID_ARG;
    if (E.N > 0 && (!ok_ptr(E.x0, true) || !ok_ptr(E.xT, true))) return PDMP_ERR_INVALID_ARG;
    total += E.N;
  }
  if (total >= ((int64_t)1 << 31)) return PDMP_ERR_INVALID_ARG;
  return PDMP_OK;
}

size_t pdmp_batch_workspace(const pdmp_env* envs, int32_t n_envs, int32_t variant) {
  if (check_envs(envs, n_envs) != PDMP_OK || variant < 0 || variant >= pdmp::batch_variants()) return 0;
  return pdmp::batch_workspace(envs, n_envs, variant);
}

pdmp_status pdmp_batch_prepare(const pdmp_env* envs, int32_t n_envs, int32_t variant, void* ws, size_t ws_bytes,
                               pdmp_batch_plan* plan, void* stream) {
  pdmp_status s = check_envs(envs, n_envs);
  if (s != PDMP_OK) return s;
  if (variant < 0 || variant >= pdmp::batch_variants() || plan == nullptr) return PDMP_ERR_INVALID_ARG;
  if (ws == nullptr || !aligned16(ws)) return PDMP_ERR_INVALID_ARG;
  if (ws_bytes < pdmp::batch_workspace(envs, n_envs, variant)) return PDMP_ERR_WORKSPACE_TOO_SMALL;
  if (pdmp::batch_workspace(envs, n_envs, variant) == 0) return PDMP_ERR_INVALID_ARG;
  return cuda_status(pdmp::batch_prepare(envs, n_envs, variant, ws, plan, as_stream(stream)));
}

pdmp_status pdmp_morph_batched(const pdmp_batch_plan* plan, void* ws, void* stream) {
  NvtxRange nvtx_range("pdmp_morph_batched");
  if (plan == nullptr || ws == nullptr || !aligned16(ws) || plan->n_envs < 1) return PDMP_ERR_INVALID_ARG;
  if (plan->variant < 0 || plan->variant >= pdmp::batch_variants()) return PDMP_ERR_INVALID_ARG;
  return cuda_status(pdmp::batch_run(plan, ws, as_stream(stream)));
}

pdmp_status pdmp_batch_autotune(const pdmp_env* envs, int32_t n_envs, int32_t reps, void* ws, size_t ws_bytes,
                                int32_t* best, float* times_ms, pdmp_batch_plan* plan, void* stream) {
  pdmp_status s = check_envs(envs, n_envs);
  if (s != PDMP_OK) return s;
  if (best == nullptr || plan == nullptr || reps < 1 || ws == nullptr || !aligned16(ws)) return PDMP_ERR_INVALID_ARG;
  const int nv = pdmp::batch_variants();
  for (int v = 0; v < nv; ++v)
    if (ws_bytes < pdmp::batch_workspace(envs, n_envs, v)) return PDMP_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = as_stream(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return PDMP_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PDMP_ERR_CUDA;
  }
  int bestv = -1;
  float bestt = 0.0f;
  pdmp_status out = PDMP_OK;
  for (int v = 0; v < nv && out == PDMP_OK; ++v) {
    pdmp_batch_plan p;
    if (pdmp::batch_prepare(envs, n_envs, v, ws, &p, st) != cudaSuccess) { out = PDMP_ERR_CUDA; break; }
    if (pdmp::batch_run(&p, ws, st) != cudaSuccess) { out = PDMP_ERR_CUDA; break; }
    float tmin = 0.0f;
    for (int r = 0; r < reps; ++r) {
      float ms = 0.0f;
      if (cudaEventRecord(e0, st) != cudaSuccess || pdmp::batch_run(&p, ws, st) != cudaSuccess ||
          cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        out = PDMP_ERR_CUDA;
        break;
      }
      if (r == 0 || ms < tmin) tmin = ms;
    }
    if (times_ms) times_ms[v] = tmin;
    if (bestv < 0 || tmin < bestt) {
      bestv = v;
      bestt = tmin;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (out != PDMP_OK) return out;
  *best = bestv;
  return cuda_status(pdmp::batch_prepare(envs, n_envs, bestv, ws, plan, st));
}

pdmp_status pdmp_batch_graph_create(const pdmp_batch_plan* plan, void* ws, void* stream, void** graph_exec) {
  if (plan == nullptr || ws == nullptr || graph_exec == nullptr || stream == nullptr) return PDMP_ERR_INVALID_ARG;
  cudaStream_t st = as_stream(stream);
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PDMP_ERR_CUDA;
  cudaError_t run = pdmp::batch_run(plan, ws, st);
  cudaGraph_t g = nullptr;
  cudaError_t end = cudaStreamEndCapture(st, &g);
  if (run != cudaSuccess || end != cudaSuccess || g == nullptr) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return PDMP_ERR_CUDA;
  }
  cudaGraphExec_t ex = nullptr;
  cudaError_t inst = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (inst != cudaSuccess) return PDMP_ERR_CUDA;
  *graph_exec = (void*)ex;
  return PDMP_OK;
}

pdmp_status pdmp_graph_launch(void* graph_exec, void* stream) {
  if (graph_exec == nullptr) return PDMP_ERR_INVALID_ARG;
  return cuda_status(cudaGraphLaunch((cudaGraphExec_t)graph_exec, as_stream(stream)));
}

pdmp_status pdmp_graph_destroy(void* graph_exec) {
  if (graph_exec == nullptr) return PDMP_ERR_INVALID_ARG;
  return cuda_status(cudaGraphExecDestroy((cudaGraphExec_t)graph_exec));
}

static pdmp_status check_mlp(const pdmp_mlp* net, bool training) {
  if (net == nullptr) return PDMP_ERR_INVALID_ARG;
  if (!ok_ptr(net->W_bf16, true) || !ok_ptr(net->b, true) || !ok_ptr(net->Wt_bf16, training)) return PDMP_ERR_INVALID_ARG;
  if (training && (!ok_ptr(net->W, true) || !ok_ptr(net->adam, true))) return PDMP_ERR_INVALID_ARG;
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(net->lo[i]) || !std::isfinite(net->in_scale[i]) || !(net->out_scale[i] != 0.0f) ||
        !std::isfinite(net->out_scale[i]))
      return PDMP_ERR_INVALID_ARG;
  return PDMP_OK;
}

pdmp_status pdmp_mlp_refresh(const pdmp_mlp* net, void* stream) {
  if (net == nullptr || !ok_ptr(net->W, true) || !ok_ptr(net->W_bf16, true) || !ok_ptr(net->Wt_bf16, true))
    return PDMP_ERR_INVALID_ARG;
  return cuda_status(pdmp::mlp_refresh(net, as_stream(stream)));
}

pdmp_status pdmp_mlp_forward(const pdmp_mlp* net, const float* x0, int64_t N, float* xT_hat, void* stream) {
  pdmp_status s = check_mlp(net, false);
  if (s != PDMP_OK) return s;
  if (N < 0) return PDMP_ERR_INVALID_ARG;
  if (N == 0) return PDMP_OK;
  if (!ok_ptr(x0, true) || !ok_ptr(xT_hat, true)) return PDMP_ERR_INVALID_ARG;
  return cuda_status(pdmp::mlp_forward(net, x0, N, xT_hat, false, as_stream(stream)));
}

pdmp_status pdmp_mlp_forward_fp32act(const pdmp_mlp* net, const float* x0, int64_t N, float* xT_hat, void* stream) {
  pdmp_status s = check_mlp(net, false);
  if (s != PDMP_OK) return s;
  if (N < 0) return PDMP_ERR_INVALID_ARG;
  if (N == 0) return PDMP_OK;
  if (!ok_ptr(x0, true) || !ok_ptr(xT_hat, true)) return PDMP_ERR_INVALID_ARG;
  return cuda_status(pdmp::mlp_forward(net, x0, N, xT_hat, true, as_stream(stream)));
}

size_t pdmp_mlp_train_workspace(int32_t B) { return B < 1 ? 0 : pdmp::mlp_train_workspace(B); }

pdmp_status pdmp_mlp_train_step(const pdmp_mlp* net, const float* x0, const float* xT, int32_t B, float lr,
                                float beta1, float beta2, float eps, int32_t step, float* loss, void* ws,
                                size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("pdmp_mlp_train_step");
  pdmp_status s = check_mlp(net, true);
  if (s != PDMP_OK) return s;
  if (B < 1 || step < 1 || !(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) ||
      !(eps > 0.0f))
    return PDMP_ERR_INVALID_ARG;
  if (!ok_ptr(x0, true) || !ok_ptr(xT, true) || !ok_ptr(loss, false) || ws == nullptr || !aligned16(ws))
    return PDMP_ERR_INVALID_ARG;
  if (ws_bytes < pdmp::mlp_train_workspace(B)) return PDMP_ERR_WORKSPACE_TOO_SMALL;
  return cuda_status(pdmp::mlp_train_step(net, x0, xT, B, lr, beta1, beta2, eps, step, loss, ws, as_stream(stream)));
}

pdmp_status pdmp_mlp_gradient(const pdmp_mlp* net, const float* x0, const float* xT, int32_t B, int32_t fp32_act,
                              float* loss, float* gW, float* gb, void* ws, size_t ws_bytes, void* stream) {
  pdmp_status s = check_mlp(net, false);
  if (s != PDMP_OK) return s;
  if (B < 1 || (fp32_act != 0 && fp32_act != 1)) return PDMP_ERR_INVALID_ARG;
  if (!ok_ptr(x0, true) || !ok_ptr(xT, true) || !ok_ptr(loss, false) || !ok_ptr(gW, true) || !ok_ptr(gb, true) ||
      ws == nullptr || !aligned16(ws))
    return PDMP_ERR_INVALID_ARG;
  if (ws_bytes < pdmp::mlp_train_workspace(B)) return PDMP_ERR_WORKSPACE_TOO_SMALL;
  return cuda_status(pdmp::mlp_gradient(net, x0, xT, B, fp32_act != 0, loss, gW, gb, ws, as_stream(stream)));
}

pdmp_status pdmp_displacement_rms(const float* x0, const float* xT, int64_t N, int32_t d, float* rms, void* stream) {
  if (N < 1 || d < 1 || d > 8 || !ok_ptr(x0, true) || !ok_ptr(xT, true) || rms == nullptr) return PDMP_ERR_INVALID_ARG;
  return cuda_status(pdmp::displacement_rms(x0, xT, N, d, rms, as_stream(stream)));
}

size_t pdmp_surrogate_workspace(const pdmp_field* f, int64_t N) {
  if (check_field(f) != PDMP_OK || f->kind != PDMP_KIND_RBF || f->d != 3 || N < 1) return 0;
  return pdmp::surrogate_workspace(f->d, f->M, N);
}

pdmp_status pdmp_surrogate_infer(const pdmp_mlp* net, const pdmp_field* f, const float* x0, int64_t N, int32_t T,
                                 float eta, float tau_r, float* xT, int64_t* n_fallback, void* ws, size_t ws_bytes,
                                 void* stream) {
  NvtxRange nvtx_range("pdmp_surrogate_infer");
  pdmp_status s = check_mlp(net, false);
  if (s != PDMP_OK) return s;
  if ((s = check_field(f)) != PDMP_OK) return s;
  if (f->kind != PDMP_KIND_RBF || f->d != 3) return PDMP_ERR_UNSUPPORTED;
  if ((s = check_step(f, eta)) != PDMP_OK) return s;
  if (N < 0 || T < 0 || n_fallback == nullptr || !(tau_r >= 0.0f)) return PDMP_ERR_INVALID_ARG;
  if (N >= ((int64_t)1 << 31)) return PDMP_ERR_INVALID_ARG;
  *n_fallback = 0;
  if (N == 0) return PDMP_OK;
  if (!ok_ptr(x0, true) || !ok_ptr(xT, true) || ws == nullptr || !aligned16(ws)) return PDMP_ERR_INVALID_ARG;
  if (xT == x0) return PDMP_ERR_INVALID_ARG;   // the fallback re-reads x0 after xT is written
  if (ws_bytes < pdmp::surrogate_workspace(f->d, f->M, N)) return PDMP_ERR_WORKSPACE_TOO_SMALL;
  return cuda_status(pdmp::surrogate_infer(net, f->d, field_args(f), x0, N, T, eta, tau_r, 0.0f, xT, n_fallback,
                                           ws, as_stream(stream)));
}

pdmp_status pdmp_surrogate_infer_culled(const pdmp_mlp* net, const pdmp_field* f, const float* x0, int64_t N,
                                        int32_t T, float eta, float tau_r, float r_cut, float* xT,
                                        int64_t* n_fallback, void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("pdmp_surrogate_infer_culled");
  pdmp_status s = check_mlp(net, false);
  if (s != PDMP_OK) return s;
  if ((s = check_field(f)) != PDMP_OK) return s;
  if (f->kind != PDMP_KIND_RBF || f->d != 3) return PDMP_ERR_UNSUPPORTED;
  if ((s = check_step(f, eta)) != PDMP_OK) return s;
  if (N < 0 || T < 0 || n_fallback == nullptr || !(tau_r >= 0.0f)) return PDMP_ERR_INVALID_ARG;
  if (!(r_cut > 0.0f) || !std::isfinite(r_cut)) return PDMP_ERR_INVALID_ARG;
  if (N >= ((int64_t)1 << 31)) return PDMP_ERR_INVALID_ARG;
  *n_fallback = 0;
  if (N == 0) return PDMP_OK;
  if (!ok_ptr(x0, true) || !ok_ptr(xT, true) || ws == nullptr || !aligned16(ws)) return PDMP_ERR_INVALID_ARG;
  if (xT == x0) return PDMP_ERR_INVALID_ARG;
  if (ws_bytes < pdmp::surrogate_workspace(f->d, f->M, N)) return PDMP_ERR_WORKSPACE_TOO_SMALL;
  return cuda_status(pdmp::surrogate_infer(net, f->d, field_args(f), x0, N, T, eta, tau_r, r_cut, xT, n_fallback,
                                           ws, as_stream(stream)));
}

size_t pdmp_residual_threshold_workspace(const pdmp_field* f, int64_t N) {
  if (check_field(f) != PDMP_OK || f->kind != PDMP_KIND_RBF || (f->d != 2 && f->d != 3) || N < 1) return 0;
  return pdmp::residual_threshold_workspace(f->d, f->M, N);
}

pdmp_status pdmp_residual_threshold(const pdmp_field* f, const float* x0, int64_t N, int32_t T, float eta, float q,
                                    float* tau_r, float* xT, void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("pdmp_residual_threshold");
  pdmp_status s = check_field(f);
  if (s != PDMP_OK) return s;
  if (f->kind != PDMP_KIND_RBF || (f->d != 2 && f->d != 3)) return PDMP_ERR_UNSUPPORTED;
  if ((s = check_step(f, eta)) != PDMP_OK) return s;
  if (N < 1 || N >= ((int64_t)1 << 31) || T < 1 || !(q > 0.0f && q <= 1.0f) || tau_r == nullptr)
    return PDMP_ERR_INVALID_ARG;
  if (!ok_ptr(x0, true) || !ok_ptr(xT, false) || ws == nullptr || !aligned16(ws)) return PDMP_ERR_INVALID_ARG;
  if (ws_bytes < pdmp::residual_threshold_workspace(f->d, f->M, N)) return PDMP_ERR_WORKSPACE_TOO_SMALL;
  // nearest rank: the ceil(q N)-th smallest length
  int64_t k = (int64_t)std::ceil((double)q * (double)N) - 1;
  if (k < 0) k = 0;
  if (k > N - 1) k = N - 1;
  return cuda_status(pdmp::residual_threshold(f->d, field_args(f), x0, N, T, eta, k, tau_r, xT, ws, as_stream(stream)));
}

size_t pdmp_fit_workspace(int64_t M, int64_t n) {
  if (M < 1 || n < 1) return 0;
  return pdmp::fit_workspace(M, n);
}

pdmp_status pdmp_fit_occupancy(const pdmp_field* f, const float* X, const uint8_t* y, int64_t n, float l2,
                               int32_t power_iters, int32_t iters, float* w_out, float* bias_out, float* loss_out,
                               float* alpha_out, void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("pdmp_fit_occupancy");
  if (f == nullptr) return PDMP_ERR_INVALID_ARG;
  pdmp_field g = *f;
  g.w = w_out;  // the fit ignores f->w; validate the geometry with the output in its place
  g.bias = 0.0f;
  g.lipschitz = 0.0;
  pdmp_status s = check_field(&g);
  if (s != PDMP_OK) return s;
  if (n < 1 || power_iters < 1 || iters < 0 || !(l2 >= 0.0f) || !std::isfinite(l2)) return PDMP_ERR_INVALID_ARG;
  if (!ok_ptr(X, true) || !ok_ptr(y, true) || !ok_ptr(w_out, true)) return PDMP_ERR_INVALID_ARG;
  if (ws == nullptr || !aligned16(ws)) return PDMP_ERR_INVALID_ARG;
  if (ws_bytes < pdmp::fit_workspace(g.M, n)) return PDMP_ERR_WORKSPACE_TOO_SMALL;
  return cuda_status(pdmp::fit_occupancy(g.kind, g.d, field_args(&g), X, y, n, l2, power_iters, iters, w_out,
                                         bias_out, loss_out, alpha_out, ws, as_stream(stream)));
}

}  // extern "C"
