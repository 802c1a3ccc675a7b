// Fast RBF morph for d = 2 and d = 3: T Euler steps of Eq. (1) on spatially
// sorted sample tiles.
//
// Expanded exponent.  For a tile with origin o (the centre of its current
// bounding box), u = x - o and c_m = mu_m - o:
//   log2(|w_m| phi_m(x)) = lw_m - g' |u - c_m|^2
//                        = (lw_m - g' |c_m|^2) + 2 g' c_m . u  -  g' |u|^2,
// with g' = gamma log2(e) and lw_m = log2|w_m|.  The last term is the same for
// every feature, so with e'_m = 2^(a_m + b_m . u), a_m = lw_m - g'|c_m|^2 and
// b_m = 2 g' c_m (per tile and step, staged in shared memory):
//   s - bias              = f S,              S = sum_m sg_m e'_m,   f = 2^(-g'|u|^2)
//   sum_m w_m phi_m (x - mu_m) = f (u S - G),  G = sum_m sg_m e'_m c_m
// and grad s = -2 gamma f (u S - G).  A feature then costs 2d + 1 FP32
// operations and one ex2; they run as packed f32x2 instructions over pairs of
// samples.  The rounding error grows with g'|u|^2, so a tile uses the expanded
// form only while g' R^2 <= 4 (R the tile's half-diagonal) and otherwise the
// direct form x - mu_m for that step.
//
// Work split.  A block of 4 warps owns a tile of 256 samples; every warp holds
// all 256 (8 per lane) and sums over its own quarter of each 256-centre stage;
// the four partial sums are added in a fixed order once per step.
#include "field.cuh"
#include "kernels.cuh"
#include "sort.cuh"

namespace pdmp {

typedef unsigned long long u64;

__device__ __forceinline__ u64 pk(float lo, float hi) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk(u64 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
  u64 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 ex2x2(u64 a) {
  float lo, hi;
  upk(a, lo, hi);
  return pk(ex2_approx(lo), ex2_approx(hi));
}

// Tile shape (compile-time; the defaults are the tuned configuration).
#ifndef PDMP_FAST_WARPS
#define PDMP_FAST_WARPS 4      // warps per block, each summing over its share of M
#endif
#ifndef PDMP_FAST_K
#define PDMP_FAST_K 8          // samples per lane (even)
#endif
#ifndef PDMP_FAST_MINB
#define PDMP_FAST_MINB 4       // blocks per SM the register budget is sized for
#endif
#ifndef PDMP_FAST_UNROLL
#define PDMP_FAST_UNROLL 2     // centres per unrolled inner iteration
#endif
#ifndef PDMP_FAST_STAGE
#define PDMP_FAST_STAGE 256    // centres per shared-memory stage
#endif
constexpr int kFastWarps = PDMP_FAST_WARPS;
constexpr int kFastThreads = 32 * kFastWarps;
constexpr int kFastK = PDMP_FAST_K;
constexpr int kFastPairs = kFastK / 2;
constexpr int kFastTile = 32 * kFastK;         // samples per block
constexpr int kFastStage = PDMP_FAST_STAGE;
constexpr int kFastSlice = kFastStage / kFastWarps;
constexpr int kFastUnroll = PDMP_FAST_UNROLL;
static_assert(kFastK % 2 == 0, "samples per lane must be even (f32x2 pairs)");
static_assert(kFastStage % kFastWarps == 0, "stage must split evenly across warps");

template <int D>
struct FastRec {
  static constexpr int kPairs = 2 * D + 2;     // u64 pairs per staged centre
  static constexpr int kTab = D == 2 ? 1 : 2;  // float4s per centre in the table
};

template <int D>
constexpr size_t fast_smem_bytes() {
  return 2 * kFastStage * FastRec<D>::kPairs * sizeof(u64) + kFastWarps * kFastTile * sizeof(float4);
}

// table: RBF centre records {mu_0 .. mu_{d-1}, lw = log2|w|, sg = sign(w)}
template <int D>
__global__ void k_rbf_table(const float* __restrict__ centres, const float* __restrict__ w, int64_t M,
                            float4* __restrict__ tab) {
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  float wm = w[m];
  float lw = wm != 0.0f ? log2f(fabsf(wm)) : -INFINITY;
  float sg = wm > 0.0f ? 1.0f : (wm < 0.0f ? -1.0f : 0.0f);
  if (D == 2) {
    tab[m] = make_float4(centres[m * 2], centres[m * 2 + 1], lw, sg);
  } else {
    tab[2 * m] = make_float4(centres[m * 3], centres[m * 3 + 1], centres[m * 3 + 2], lw);
    tab[2 * m + 1] = make_float4(sg, 0.0f, 0.0f, 0.0f);
  }
}

// Stages centres [m0, m0 + kFastStage) into rec (kFastStage x kPairs u64).
//   expanded: [a a][b_0 b_0]..[b_{d-1} ..][sg sg][c~_0 c~_0]..  (c~ = sg (mu - o))
//   direct:   [-mu_0 -mu_0]..[-mu_{d-1} ..][lw lw][sg sg]
template <int D>
__device__ __forceinline__ void fast_stage(const float4* __restrict__ tab, int64_t M, int64_t m0, bool expanded,
                                           const float* o, float gl2e, u64* rec) {
  constexpr int RP = FastRec<D>::kPairs;
  for (int i = threadIdx.x; i < kFastStage; i += kFastThreads) {
    int64_t m = m0 + i;
    float mu[D], lw = -INFINITY, sg = 0.0f;
    if (m < M) {
      float4 t0 = tab[FastRec<D>::kTab * m];
      mu[0] = t0.x;
      mu[1] = t0.y;
      if (D == 2) {
        lw = t0.z;
        sg = t0.w;
      } else {
        mu[2] = t0.z;
        lw = t0.w;
        sg = tab[2 * m + 1].x;
      }
    } else {
#pragma unroll
      for (int j = 0; j < D; ++j) mu[j] = 0.0f;
    }
    u64 r[RP];
    if (expanded) {
      float c[D], r2 = 0.0f;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        c[j] = mu[j] - o[j];
        r2 = fmaf(c[j], c[j], r2);
      }
      float a = fmaf(-gl2e, r2, lw);
      r[0] = pk(a, a);
#pragma unroll
      for (int j = 0; j < D; ++j) {
        float b = 2.0f * gl2e * c[j];
        r[1 + j] = pk(b, b);
        float ct = sg * c[j];
        r[D + 2 + j] = pk(ct, ct);
      }
      r[D + 1] = pk(sg, sg);
    } else {
#pragma unroll
      for (int j = 0; j < D; ++j) r[j] = pk(-mu[j], -mu[j]);
      r[D] = pk(lw, lw);
      r[D + 1] = pk(sg, sg);
#pragma unroll
      for (int j = D + 2; j < RP; ++j) r[j] = 0ull;
    }
    ulonglong2* dst = reinterpret_cast<ulonglong2*>(rec + (size_t)i * RP);
#pragma unroll
    for (int j = 0; j < RP / 2; ++j) dst[j] = make_ulonglong2(r[2 * j], r[2 * j + 1]);
  }
}

template <int D, bool TRACE>
__global__ void __launch_bounds__(kFastThreads, PDMP_FAST_MINB)
k_morph_rbf_fast(const float4* __restrict__ tab, int64_t M, float gamma, float bias, const float* x0,
                 const int32_t* __restrict__ perm, int64_t N, int T, float eta, float* xT, float* __restrict__ ckpt,
                 int kck, float* __restrict__ traj, float* __restrict__ steps) {
  constexpr int RP = FastRec<D>::kPairs;
  constexpr int K = kFastK, P = kFastPairs;
  extern __shared__ __align__(16) unsigned char smem[];
  u64* bufs = reinterpret_cast<u64*>(smem);
  float4* red = reinterpret_cast<float4*>(smem + 2 * kFastStage * RP * sizeof(u64));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tile0 = (int64_t)blockIdx.x * kFastTile;
  const float gl2e = gamma * kLog2e;
  const int nstage = (int)((M + kFastStage - 1) / kFastStage);

  float x[K][D];
  bool act[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int64_t p = tile0 + k * 32 + lane;
    act[k] = p < N;
    const int64_t n = act[k] ? (int64_t)perm[p] : 0;
#pragma unroll
    for (int j = 0; j < D; ++j) x[k][j] = act[k] ? x0[n * D + j] : 0.0f;
  }

  for (int t = 0; t < T; ++t) {
    // tile origin and half-diagonal (identical in every warp)
    float lo[D], hi[D];
#pragma unroll
    for (int j = 0; j < D; ++j) { lo[j] = INFINITY; hi[j] = -INFINITY; }
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (act[k])
#pragma unroll
        for (int j = 0; j < D; ++j) { lo[j] = fminf(lo[j], x[k][j]); hi[j] = fmaxf(hi[j], x[k][j]); }
    float o[D], R2 = 0.0f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) {
        lo[j] = fminf(lo[j], __shfl_xor_sync(0xffffffffu, lo[j], s));
        hi[j] = fmaxf(hi[j], __shfl_xor_sync(0xffffffffu, hi[j], s));
      }
      o[j] = 0.5f * (lo[j] + hi[j]);
      float h = 0.5f * (hi[j] - lo[j]);
      R2 = fmaf(h, h, R2);
    }
    const bool expanded = (gl2e * R2 <= 4.0f) && (o[0] == o[0]);
    if (!expanded)
#pragma unroll
      for (int j = 0; j < D; ++j) o[j] = 0.0f;

    u64 U[P][D], S[P], G[P][D];
#pragma unroll
    for (int i = 0; i < P; ++i) {
#pragma unroll
      for (int j = 0; j < D; ++j) {
        U[i][j] = pk(x[2 * i][j] - o[j], x[2 * i + 1][j] - o[j]);
        G[i][j] = 0ull;
      }
      S[i] = 0ull;
    }

    fast_stage<D>(tab, M, 0, expanded, o, gl2e, bufs);
    __syncthreads();
    for (int st = 0; st < nstage; ++st) {
      const u64* rec = bufs + (size_t)(st & 1) * kFastStage * RP + (size_t)warp * kFastSlice * RP;
      if (expanded) {
#pragma unroll kFastUnroll
        for (int c = 0; c < kFastSlice; ++c) {
          const ulonglong2* q = reinterpret_cast<const ulonglong2*>(rec + (size_t)c * RP);
          u64 r[RP];
#pragma unroll
          for (int j = 0; j < RP / 2; ++j) {
            ulonglong2 v = q[j];
            r[2 * j] = v.x;
            r[2 * j + 1] = v.y;
          }
#pragma unroll
          for (int i = 0; i < P; ++i) {
            u64 arg = fma2(r[1], U[i][0], r[0]);
#pragma unroll
            for (int j = 1; j < D; ++j) arg = fma2(r[1 + j], U[i][j], arg);
            const u64 e = ex2x2(arg);
            S[i] = fma2(r[D + 1], e, S[i]);
#pragma unroll
            for (int j = 0; j < D; ++j) G[i][j] = fma2(e, r[D + 2 + j], G[i][j]);
          }
        }
      } else {
        const u64 ng = pk(-gl2e, -gl2e);
        for (int c = 0; c < kFastSlice; ++c) {
          const u64* r = rec + (size_t)c * RP;
#pragma unroll
          for (int i = 0; i < P; ++i) {
            u64 dx[D];
#pragma unroll
            for (int j = 0; j < D; ++j) dx[j] = add2(U[i][j], r[j]);
            u64 r2 = mul2(dx[0], dx[0]);
#pragma unroll
            for (int j = 1; j < D; ++j) r2 = fma2(dx[j], dx[j], r2);
            const u64 we = mul2(r[D + 1], ex2x2(fma2(r2, ng, r[D])));
            S[i] = add2(S[i], we);
#pragma unroll
            for (int j = 0; j < D; ++j) G[i][j] = fma2(we, dx[j], G[i][j]);
          }
        }
      }
      if (st + 1 < nstage)
        fast_stage<D>(tab, M, (int64_t)(st + 1) * kFastStage, expanded, o, gl2e,
                      bufs + (size_t)((st + 1) & 1) * kFastStage * RP);
      __syncthreads();
    }

    // partial sums -> shared memory, then the same fixed-order total in every warp
#pragma unroll
    for (int i = 0; i < P; ++i) {
      float s0, s1, g0[D], g1[D];
      upk(S[i], s0, s1);
#pragma unroll
      for (int j = 0; j < D; ++j) upk(G[i][j], g0[j], g1[j]);
      red[warp * kFastTile + (2 * i) * 32 + lane] = make_float4(s0, g0[0], g0[1], D == 3 ? g0[D - 1] : 0.0f);
      red[warp * kFastTile + (2 * i + 1) * 32 + lane] = make_float4(s1, g1[0], g1[1], D == 3 ? g1[D - 1] : 0.0f);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float4 a = red[k * 32 + lane];
#pragma unroll
      for (int w = 1; w < kFastWarps; ++w) {
        float4 b = red[w * kFastTile + k * 32 + lane];
        a.x += b.x;
        a.y += b.y;
        a.z += b.z;
        a.w += b.w;
      }
      const float Ssum = a.x, Gs[3] = {a.y, a.z, a.w};
      float shat, ghat[D];
      if (expanded) {
        float u[D], u2 = 0.0f;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          u[j] = x[k][j] - o[j];
          u2 = fmaf(u[j], u[j], u2);
        }
        const float f = ex2_approx(-gl2e * u2);
        shat = f * Ssum;
#pragma unroll
        for (int j = 0; j < D; ++j) ghat[j] = f * fmaf(u[j], Ssum, -Gs[j]);
      } else {
        shat = Ssum;
#pragma unroll
        for (int j = 0; j < D; ++j) ghat[j] = Gs[j];
      }
      float d1, d2;
      sigmoid_d12(shat + bias, d1, d2);
      const float c = -eta * d1;
      const int64_t p = tile0 + k * 32 + lane;
      const int64_t n = (TRACE && act[k] && warp == 0) ? (int64_t)perm[p] : 0;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const float inc = __fmul_rn(c, -2.0f * gamma * ghat[j]);
        if (TRACE && act[k] && warp == 0) {
          traj[((int64_t)t * N + n) * D + j] = x[k][j];
          steps[((int64_t)t * N + n) * D + j] = inc;
        }
        x[k][j] = __fadd_rn(x[k][j], inc);
      }
    }
    if (ckpt != nullptr && (t + 1) % kck == 0 && warp == 0) {
      float* dst = ckpt + (int64_t)((t + 1) / kck - 1) * N * D;
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (act[k]) {
          const int64_t n = perm[tile0 + k * 32 + lane];
#pragma unroll
          for (int j = 0; j < D; ++j) dst[n * D + j] = x[k][j];
        }
    }
  }
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (act[k]) {
        const int64_t n = perm[tile0 + k * 32 + lane];
#pragma unroll
        for (int j = 0; j < D; ++j) {
          if (xT) xT[n * D + j] = x[k][j];
          if (TRACE) traj[((int64_t)T * N + n) * D + j] = x[k][j];
        }
      }
  }
}

// ------------------------------------------------------------------ host
static size_t table_bytes(int d, int64_t M) {
  return (((size_t)M * 16 * (d == 2 ? 1 : 2)) + 255) & ~size_t(255);
}

size_t morph_rbf_fast_workspace(int d, int64_t M, int64_t N) {
  return table_bytes(d, M) + sort_workspace(d, N);
}

template <int D>
static cudaError_t launch_fast(const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* xT,
                               float* ckpt, int k, float* traj, float* steps, void* ws, cudaStream_t st) {
  float4* tab = reinterpret_cast<float4*>(ws);
  SortWs sw = sort_layout((char*)ws + table_bytes(D, fa.M), D, N);
  k_rbf_table<D><<<(unsigned)((fa.M + 255) / 256), 256, 0, st>>>(fa.centres, fa.w, fa.M, tab);
  cudaError_t e = spatial_sort(D, x0, N, sw, st);
  if (e != cudaSuccess) return e;
  constexpr size_t smem = fast_smem_bytes<D>();
  const unsigned blocks = (unsigned)((N + kFastTile - 1) / kFastTile);
  if (traj != nullptr) {
    cudaFuncSetAttribute(k_morph_rbf_fast<D, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_morph_rbf_fast<D, true><<<blocks, kFastThreads, smem, st>>>(tab, fa.M, fa.gamma, fa.bias, x0, sw.perm, N, T,
                                                                  eta, xT, ckpt, k, traj, steps);
  } else {
    cudaFuncSetAttribute(k_morph_rbf_fast<D, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_morph_rbf_fast<D, false><<<blocks, kFastThreads, smem, st>>>(tab, fa.M, fa.gamma, fa.bias, x0, sw.perm, N, T,
                                                                   eta, xT, ckpt, k, nullptr, nullptr);
  }
  return cudaGetLastError();
}

cudaError_t morph_rbf_fast(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* xT,
                           float* ckpt, int k, float* traj, float* steps, void* ws, cudaStream_t st) {
  if (d == 2) return launch_fast<2>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
  if (d == 3) return launch_fast<3>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
  return cudaErrorInvalidValue;
}

}  // namespace pdmp
