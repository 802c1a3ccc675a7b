// Fast random-Fourier-feature morph: T Euler steps of Eq. (1) with
// phi_m = cos(omega_m . x + b_m), for d = 1 .. 8.
//
// The records do not depend on the samples, so a table of packed pairs
// [omega_0 omega_0] .. [omega_{d-1} ..] [b b] [w w] [-w -w] is built once per
// call; each warp of a block owns a contiguous slice of it and streams the
// slice through its own double-buffered shared-memory stages (cp.async, warp
// synchronisation only).  Every warp holds all the block's samples (K per
// lane, in f32x2 pairs), so a feature costs per sample pair d + 1 + 2 + 1 + 1
// + d packed FP32 instructions (theta, its reduction by 2 pi, s, -w sin, the
// gradient) and four MUFU sin/cos; the warps' partial sums are added in a
// fixed order once per step.
#include "fast_tile.cuh"
#include "kernels.cuh"

namespace pdmp {

constexpr int kRffWarps = 4;
constexpr int kRffK = 4;                         // samples per lane (two pairs)
constexpr int kRffTile = 32 * kRffK;             // samples per block
constexpr int kRffStage = 64;                    // records per warp per stage

template <int D>
struct RffRec {
  static constexpr int kPairs = D + 3;           // u64 pairs per record
  static constexpr int kChunks = (kPairs * 8 + 15) / 16;   // 16-byte copies per record
  static constexpr int kWords = kChunks * 2;     // u64 words per record (padded)
};

template <int D>
__host__ __device__ constexpr size_t rff_stage_bytes() {
  return (size_t)kRffStage * RffRec<D>::kWords * 8;
}
template <int D>
__host__ __device__ constexpr size_t rff_red_bytes() {
  return (size_t)kRffWarps * kRffTile * (D + 1) * 4;
}
template <int D>
__host__ __device__ constexpr size_t rff_smem_bytes() {
  return kRffWarps * 2 * rff_stage_bytes<D>() > rff_red_bytes<D>() ? kRffWarps * 2 * rff_stage_bytes<D>()
                                                                    : rff_red_bytes<D>();
}

template <int D>
__global__ void k_rff_table(FieldArgs fa, u64* __restrict__ tab) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= fa.M) return;
  u64* r = tab + m * RffRec<D>::kWords;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const float o = fa.centres[m * D + j];
    r[j] = ((u64)__float_as_uint(o) << 32) | __float_as_uint(o);
  }
  const float b = fa.phase[m], w = fa.w[m];
  r[D] = ((u64)__float_as_uint(b) << 32) | __float_as_uint(b);
  r[D + 1] = ((u64)__float_as_uint(w) << 32) | __float_as_uint(w);
  r[D + 2] = ((u64)__float_as_uint(-w) << 32) | __float_as_uint(-w);
#pragma unroll
  for (int j = D + 3; j < RffRec<D>::kWords; ++j) r[j] = 0ull;
}

// copies records [m0, m0 + kRffStage) of the table into the warp's stage
// (records past M are zero: w = 0 contributes nothing)
template <int D>
__device__ __forceinline__ void rff_prefetch(const u64* __restrict__ tab, int64_t M, int64_t m0, int64_t mend,
                                             u64* dst, int lane) {
  constexpr int C = RffRec<D>::kChunks;
  for (int i = lane; i < kRffStage * C; i += 32) {
    const int rec = i / C, q = i % C;
    const int64_t m = m0 + rec;
    if (m < mend && m < M) cp_async16(dst + rec * RffRec<D>::kWords + 2 * q, tab + m * RffRec<D>::kWords + 2 * q);
    else {
      ulonglong2 z = make_ulonglong2(0ull, 0ull);
      *reinterpret_cast<ulonglong2*>(dst + rec * RffRec<D>::kWords + 2 * q) = z;
    }
  }
  cp_async_commit();
}

template <int D, bool TRACE>
__global__ void __launch_bounds__(kRffWarps * 32, 3)
k_morph_rff_fast(const u64* __restrict__ tab, int64_t M, float bias, const float* __restrict__ x0, int64_t N, int T,
                 float eta, float* __restrict__ xT, float* __restrict__ ckpt, int kck, float* __restrict__ traj,
                 float* __restrict__ steps) {
  constexpr int P = kRffK / 2;
  constexpr int RW = RffRec<D>::kWords;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64* wbuf = reinterpret_cast<u64*>(smem) + (size_t)warp * 2 * kRffStage * RW;
  float* red = reinterpret_cast<float*>(smem);   // aliases the stages after a step's last stage
  const int64_t n0 = (int64_t)blockIdx.x * kRffTile;
  const int64_t Mw = ((M + kRffWarps - 1) / kRffWarps + kRffStage - 1) / kRffStage * kRffStage;
  const int64_t mbase = (int64_t)warp * Mw, mend = mbase + Mw;
  const int nstage = (int)(Mw / kRffStage);
  const u64 inv2pi = pk(kInv2Pi, kInv2Pi);
  const u64 n2pi_hi = pk(-k2PiHi, -k2PiHi);     // the same head / tail split as reduce_2pi
  const u64 n2pi_lo = pk(-k2PiLo, -k2PiLo);

  float x[kRffK][D];
  bool act[kRffK];
#pragma unroll
  for (int k = 0; k < kRffK; ++k) {
    const int64_t n = n0 + k * 32 + lane;
    act[k] = n < N;
#pragma unroll
    for (int j = 0; j < D; ++j) x[k][j] = act[k] ? x0[n * D + j] : 0.0f;
  }

  for (int t = 0; t < T; ++t) {
    u64 X[P][D], S[P], G[P][D];
#pragma unroll
    for (int i = 0; i < P; ++i) {
#pragma unroll
      for (int j = 0; j < D; ++j) {
        X[i][j] = pk(x[2 * i][j], x[2 * i + 1][j]);
        G[i][j] = 0ull;
      }
      S[i] = 0ull;
    }
    if (nstage > 0) rff_prefetch<D>(tab, M, mbase, mend, wbuf, lane);
    for (int st = 0; st < nstage; ++st) {
      cp_async_wait_all();
      __syncwarp();
      if (st + 1 < nstage)
        rff_prefetch<D>(tab, M, mbase + (int64_t)(st + 1) * kRffStage, mend,
                        wbuf + (size_t)((st + 1) & 1) * kRffStage * RW, lane);
      const u64* rb = wbuf + (size_t)(st & 1) * kRffStage * RW;
#pragma unroll 2
      for (int c = 0; c < kRffStage; ++c) {
        const u64* r = rb + (size_t)c * RW;
        u64 rec[D + 3];
#pragma unroll
        for (int j = 0; j < (D + 3) / 2; ++j) {
          const ulonglong2 v = reinterpret_cast<const ulonglong2*>(r)[j];
          rec[2 * j] = v.x;
          rec[2 * j + 1] = v.y;
        }
        if ((D + 3) & 1) rec[D + 2] = r[D + 2];
#pragma unroll
        for (int i = 0; i < P; ++i) {
          u64 th = rec[D];
#pragma unroll
          for (int j = 0; j < D; ++j) th = fma2(rec[j], X[i][j], th);
          // theta - 2 pi rint(theta / 2 pi), 2 pi split into head and tail
          float k0, k1;
          upk(mul2(th, inv2pi), k0, k1);
          const u64 kk = pk(rintf(k0), rintf(k1));
          th = fma2(kk, n2pi_hi, th);
          th = fma2(kk, n2pi_lo, th);
          float t0, t1;
          upk(th, t0, t1);
          const u64 cs = pk(cos_approx(t0), cos_approx(t1));
          const u64 sn = pk(sin_approx(t0), sin_approx(t1));
          S[i] = fma2(rec[D + 1], cs, S[i]);
          const u64 nws = mul2(rec[D + 2], sn);
#pragma unroll
          for (int j = 0; j < D; ++j) G[i][j] = fma2(nws, rec[j], G[i][j]);
        }
      }
      __syncwarp();   // the stage is read before the next prefetch overwrites it
    }
    __syncthreads();  // every warp is done with its stages before they become the reduction buffer
#pragma unroll
    for (int i = 0; i < P; ++i) {
      float s0, s1;
      upk(S[i], s0, s1);
      red[(warp * kRffTile + (2 * i) * 32 + lane) * (D + 1)] = s0;
      red[(warp * kRffTile + (2 * i + 1) * 32 + lane) * (D + 1)] = s1;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        float g0, g1;
        upk(G[i][j], g0, g1);
        red[(warp * kRffTile + (2 * i) * 32 + lane) * (D + 1) + 1 + j] = g0;
        red[(warp * kRffTile + (2 * i + 1) * 32 + lane) * (D + 1) + 1 + j] = g1;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kRffK; ++k) {
      const int row = k * 32 + lane;
      float acc[D + 1];
#pragma unroll
      for (int j = 0; j <= D; ++j) acc[j] = red[row * (D + 1) + j];
#pragma unroll
      for (int w = 1; w < kRffWarps; ++w)
#pragma unroll
        for (int j = 0; j <= D; ++j) acc[j] += red[(w * kRffTile + row) * (D + 1) + j];
      float d1, d2;
      sigmoid_d12(acc[0] + bias, d1, d2);
      const float c = -eta * d1;
      const int64_t n = n0 + row;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const float inc = __fmul_rn(c, acc[1 + j]);
        if (TRACE && act[k] && warp == 0) {
          traj[((int64_t)t * N + n) * D + j] = x[k][j];
          steps[((int64_t)t * N + n) * D + j] = inc;
        }
        x[k][j] = __fadd_rn(x[k][j], inc);
      }
    }
    __syncthreads();  // the reduction buffer is read before the next step's stages overwrite it
    if (ckpt != nullptr && (t + 1) % kck == 0 && warp == 0) {
      float* dst = ckpt + (int64_t)((t + 1) / kck - 1) * N * D;
#pragma unroll
      for (int k = 0; k < kRffK; ++k)
        if (act[k])
#pragma unroll
          for (int j = 0; j < D; ++j) dst[(n0 + k * 32 + lane) * D + j] = x[k][j];
    }
  }
  if (warp == 0)
#pragma unroll
    for (int k = 0; k < kRffK; ++k)
      if (act[k]) {
        const int64_t n = n0 + k * 32 + lane;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          if (xT) xT[n * D + j] = x[k][j];
          if (TRACE) traj[((int64_t)T * N + n) * D + j] = x[k][j];
        }
      }
}

size_t morph_rff_fast_workspace(int d, int64_t M) { return ((size_t)M * 8 * (size_t)(((d + 3) * 8 + 15) / 16 * 2) + 255) & ~size_t(255); }

template <int D>
static cudaError_t launch_rff(const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* xT,
                              float* ckpt, int k, float* traj, float* steps, void* ws, cudaStream_t st) {
  u64* tab = reinterpret_cast<u64*>(ws);
  k_rff_table<D><<<(unsigned)((fa.M + 255) / 256), 256, 0, st>>>(fa, tab);
  constexpr size_t smem = rff_smem_bytes<D>();
  const unsigned blocks = (unsigned)((N + kRffTile - 1) / kRffTile);
  if (traj != nullptr) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_morph_rff_fast<D, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_morph_rff_fast<D, true><<<blocks, kRffWarps * 32, smem, st>>>(tab, fa.M, fa.bias, x0, N, T, eta, xT, ckpt, k,
                                                                    traj, steps);
  } else {
    const cudaError_t e =
        cudaFuncSetAttribute(k_morph_rff_fast<D, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_morph_rff_fast<D, false><<<blocks, kRffWarps * 32, smem, st>>>(tab, fa.M, fa.bias, x0, N, T, eta, xT, ckpt,
                                                                     k, nullptr, nullptr);
  }
  return cudaGetLastError();
}

cudaError_t morph_rff_fast(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* xT,
                           float* ckpt, int k, float* traj, float* steps, void* ws, cudaStream_t st) {
  switch (d) {
    case 1: return launch_rff<1>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
    case 2: return launch_rff<2>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
    case 3: return launch_rff<3>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
    case 4: return launch_rff<4>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
    case 5: return launch_rff<5>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
    case 6: return launch_rff<6>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
    case 7: return launch_rff<7>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
    case 8: return launch_rff<8>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace pdmp
