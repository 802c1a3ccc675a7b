// Shared device helpers and host-side checks for libpdmp (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include "pdmp.h"

namespace pdmp {

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

// ---------------------------------------------------------------- device flag
// Numerical failures seen by a kernel (for example a non-positive pivot in the
// log-det Cholesky) are OR-ed into this word; pdmp_stream_status reads and
// clears it.
enum : int32_t {
  FLAG_NONPOSITIVE_PIVOT = PDMP_FLAG_NONPOSITIVE_PIVOT,
  FLAG_FIT_NONFINITE = PDMP_FLAG_FIT_NONFINITE,
  FLAG_NOT_CONVERGED = PDMP_FLAG_NOT_CONVERGED,
  FLAG_STAGE_TIMEOUT = PDMP_FLAG_STAGE_TIMEOUT,
  FLAG_MMA_TIMEOUT = PDMP_FLAG_MMA_TIMEOUT,
};
extern __device__ int32_t g_device_flag;

__device__ __forceinline__ void raise_flag(int32_t bits) { atomicOr(&g_device_flag, bits); }

// ------------------------------------------------------------- fast maths
// 2^x on the special-function unit (flush-to-zero: results below 2^-126 are 0).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sin_approx(float x) {
  float y;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float cos_approx(float x) {
  float y;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Cody-Waite reduction of theta to [-pi, pi]: theta - 2 pi rint(theta / 2 pi)
// with 2 pi split into a float head and tail, so that the special-function
// unit's sin / cos (accurate on [-pi, pi]) see a reduced argument.
constexpr float kInv2Pi = 0.159154943091895336f;
constexpr float k2PiHi = 6.28318548202514648f;       // float(2 pi)
constexpr float k2PiLo = -1.7484556e-07f;             // 2 pi - float(2 pi)
__device__ __forceinline__ float reduce_2pi(float theta) {
  float k = rintf(theta * kInv2Pi);
  float r = fmaf(-k, k2PiHi, theta);
  return fmaf(-k, k2PiLo, r);
}

constexpr float kLog2e = 1.44269504088896341f;

// sigmoid'(s) = e / (1 + e)^2 and sigmoid''(s) = sigmoid' * (1 - 2 sigmoid),
// both from e = exp(-|s|) so that nothing overflows and sigmoid' keeps its
// relative accuracy in the tails.
__device__ __forceinline__ void sigmoid_d12(float s, float& d1, float& d2) {
  float e = expf(-fabsf(s));
  float inv = 1.0f / (1.0f + e);
  d1 = e * inv * inv;
  // 1 - 2 sigmoid(s) = (1 - e^{s}) / (1 + e^{s}) = sign(-s) (1 - e) / (1 + e)
  float t = (1.0f - e) * inv;
  d2 = d1 * (s >= 0.0f ? -t : t);
}
__device__ __forceinline__ float sigmoid_f(float s) {
  float e = expf(-fabsf(s));
  float inv = 1.0f / (1.0f + e);
  return s >= 0.0f ? inv : e * inv;
}

}  // namespace pdmp

// ------------------------------------------------------------------ host side
namespace pdmp_host {

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
inline bool ok_ptr(const void* p, bool needed) { return needed ? (p != nullptr && aligned16(p)) : (p == nullptr || aligned16(p)); }

// validates a field; returns PDMP_OK or PDMP_ERR_INVALID_ARG
pdmp_status check_field(const pdmp_field* f);
// additionally checks eta > 0 (finite) and eta * L < 1 when the field carries L
pdmp_status check_step(const pdmp_field* f, float eta);

inline pdmp_status cuda_status(cudaError_t e) { return e == cudaSuccess ? PDMP_OK : PDMP_ERR_CUDA; }
inline pdmp_status launch_status() { return cuda_status(cudaGetLastError()); }

inline int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

}  // namespace pdmp_host
