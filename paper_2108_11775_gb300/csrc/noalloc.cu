// pdmp_morph_noalloc: the fast RBF morph with its scratch memory built into
// the library, for callers that cannot allocate device memory themselves --
// for example code that runs where cudaMalloc is not allowed or not wanted
// (inside a real-time planning loop that must not touch the allocator, or a
// host that hands the library only the buffers it owns).
//
// The scratch (centre table + spatial-sort arrays) is a file-scope device
// array of kNoallocScratchBytes.  Every GPU that loads the library holds it
// until the process exits.  Host code cannot use the array's name as a device
// address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it; that first
// call should come before any stream capture.  The cached address belongs to
// the device's primary context: after cudaDeviceReset (or any teardown of the
// primary context) on that device it is stale, so a process that resets a
// device must not call this entry point on it again.  All calls share the array and
// it keeps the previous call's contents; the sort clears what must start at
// zero on every call.  Calls that overlap on the GPU (different streams, or
// different host threads) race on the array and must be serialised by the
// caller.
#include <mutex>

#include "kernels.cuh"

namespace pdmp {

constexpr int64_t kNoallocMaxN = int64_t(1) << 20;
constexpr int64_t kNoallocMaxM = 16384;
constexpr size_t kNoallocScratchBytes = size_t(12) << 20;   // 12 MiB >= worst case for the limits above

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[64] = {nullptr};

// device address of the scratch for the current device (looked up once per device)
static cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace pdmp

using namespace pdmp_host;

extern "C" pdmp_status pdmp_morph_noalloc(const pdmp_field* f, const float* x0, int64_t N, int32_t T, float eta,
                                          float* xT, void* stream) {
  pdmp_status s = check_field(f);
  if (s != PDMP_OK) return s;
  if (f->kind != PDMP_KIND_RBF || (f->d != 2 && f->d != 3)) return PDMP_ERR_UNSUPPORTED;
  if ((s = check_step(f, eta)) != PDMP_OK) return s;
  if (N < 0 || T < 0) return PDMP_ERR_INVALID_ARG;
  if (N > pdmp::kNoallocMaxN || f->M > pdmp::kNoallocMaxM) return PDMP_ERR_WORKSPACE_TOO_SMALL;
  if (pdmp::morph_rbf_fast_workspace(f->d, f->M, N) > pdmp::kNoallocScratchBytes) return PDMP_ERR_WORKSPACE_TOO_SMALL;
  if (N == 0) return PDMP_OK;
  if (!ok_ptr(x0, true) || !ok_ptr(xT, true)) return PDMP_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (T == 0) {
    if (xT != x0) return cuda_status(cudaMemcpyAsync(xT, x0, sizeof(float) * N * f->d, cudaMemcpyDeviceToDevice, st));
    return PDMP_OK;
  }
  void* scratch = nullptr;
  cudaError_t e = pdmp::noalloc_scratch(&scratch);
  if (e != cudaSuccess) return PDMP_ERR_CUDA;
  pdmp::FieldArgs fa;
  fa.centres = f->centres;
  fa.phase = f->phase;
  fa.w = f->w;
  fa.M = f->M;
  fa.gamma = f->gamma;
  fa.bias = f->bias;
  return cuda_status(pdmp::morph_rbf_fast(f->d, fa, x0, N, T, eta, xT, nullptr, 0, nullptr, nullptr, scratch, st));
}
