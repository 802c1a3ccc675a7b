// VJP of the T-step map (g_t = (I - eta Hess c(x_t)) g_{t+1}) for RBF fields
// in d = 2, 3 on the forward's spatially sorted tiles.
//
// Segment by segment (last first), the tile's states are recomputed from the
// checkpoint with the forward's tile step and kept in shared memory; each
// step back is one pass over the features at x_t with v = g.  With the
// tile's origin o, u = x - o, c_m = mu_m - o and e'_m = sg_m 2^(a_m + b_m . u)
// (w_m phi_m = f e'_m, f = 2^(-g' |u|^2)), the pass sums
//   S = sum e',  G = sum e' c,  K = sum e' (c . v),  Kc = sum e' (c . v) c,
// which give grad s = -2 gamma f (u S - G) and
//   (Hess s) v = 4 gamma^2 f ((u . v)(u S - G) - (u K - Kc)) - 2 gamma f S v:
// 4d + 3 packed FP32 operations and one ex2 per sample pair and feature.
// Tiles too wide for the expanded form take the direct form.
#include "fast_tile.cuh"
#include "kernels.cuh"
#include "sort.cuh"

namespace pdmp {

template <int D>
struct VjRbf {
  static constexpr int kUsed = 3 * D + 2;              // u64 pairs: a, b, sg, c~ = sg c, c
  // whole 16-byte chunks, an odd number of them: the lanes of a quarter warp
  // building consecutive records then write to distinct banks
  static constexpr int kChunks = (kUsed + 1) / 2 % 2 == 1 ? (kUsed + 1) / 2 : (kUsed + 1) / 2 + 1;
  static constexpr int kPairs = 2 * kChunks;
  static constexpr int kSums = 2 * D + 2;              // S, G, K, Kc (direct: S, G, -, P)
  static constexpr int kK = D == 2 ? 8 : 6;
  static constexpr int kW = 4;
  static constexpr int kTile = 32 * kK;
};

template <int D>
__host__ __device__ constexpr size_t vj_rbf_region0() {
  constexpr size_t bufs = (size_t)VjRbf<D>::kW * 2 * kWarpStage * VjRbf<D>::kPairs * 8;
  constexpr size_t red = (size_t)VjRbf<D>::kW * VjRbf<D>::kSums * VjRbf<D>::kTile * 4;
  return bufs > red ? bufs : red;
}
// region 0 (stages / reduction), the raw table entries, the segment's states
template <int D>
__host__ __device__ constexpr size_t vj_rbf_smem(int kseg) {
  return vj_rbf_region0<D>() + (size_t)VjRbf<D>::kW * kWarpStage * FastRec<D>::kTab * sizeof(float4) +
         (size_t)kseg * VjRbf<D>::kTile * D * sizeof(float);
}

//   expanded: [a][b_0 ..][sg][c~_0 ..][c_0 ..]     direct: [-mu_0 ..][lw][sg] (rest zero)
template <int D>
__device__ __forceinline__ void vj_stage_build(int64_t M, int64_t m0, bool expanded, const float* o, float gl2e,
                                               const float4* raw, u64* rec, int lane) {
  constexpr int RP = VjRbf<D>::kPairs;
  constexpr int KT = FastRec<D>::kTab;
  cp_async_wait_all();
  for (int i = lane; i < kWarpStage; i += 32) {
    const int64_t m = m0 + i;
    float mu[D], lw = -INFINITY, sg = 0.0f;
    if (m < M) {
      const float4 t0 = raw[i * KT];
      mu[0] = t0.x;
      mu[1] = t0.y;
      if (D == 2) {
        lw = t0.z;
        sg = t0.w;
      } else {
        mu[2] = t0.z;
        lw = t0.w;
        sg = raw[i * KT + 1].x;
      }
    } else {
#pragma unroll
      for (int j = 0; j < D; ++j) mu[j] = 0.0f;
    }
    u64 r[RP];
#pragma unroll
    for (int j = 0; j < RP; ++j) r[j] = 0ull;
    if (expanded) {
      float c[D], r2 = 0.0f;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        c[j] = mu[j] - o[j];
        r2 = fmaf(c[j], c[j], r2);
      }
      const float a = fmaf(-gl2e, r2, lw);
      r[0] = pk(a, a);
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const float b = 2.0f * gl2e * c[j], ct = sg * c[j];
        r[1 + j] = pk(b, b);
        r[D + 2 + j] = pk(ct, ct);
        r[2 * D + 2 + j] = pk(c[j], c[j]);
      }
      r[D + 1] = pk(sg, sg);
    } else {
#pragma unroll
      for (int j = 0; j < D; ++j) r[j] = pk(-mu[j], -mu[j]);
      r[D] = pk(lw, lw);
      r[D + 1] = pk(sg, sg);
    }
    ulonglong2* dst = reinterpret_cast<ulonglong2*>(rec + (size_t)i * RP);
#pragma unroll
    for (int j = 0; j < RP / 2; ++j) dst[j] = make_ulonglong2(r[2 * j], r[2 * j + 1]);
  }
}

// sums of one pass at u (U) with v (V); Z = K (expanded) or unused (direct), Y = Kc or P
template <int D, int P>
__device__ __forceinline__ void vj_stage_accumulate(const u64* rec, bool expanded, float gl2e, const u64 (&U)[P][D],
                                                    const u64 (&V)[P][D], u64 (&S)[P], u64 (&G)[P][D], u64 (&Z)[P],
                                                    u64 (&Y)[P][D]) {
  constexpr int RP = VjRbf<D>::kPairs;
  if (expanded) {
#pragma unroll 2
    for (int c = 0; c < kWarpStage; ++c) {
      const ulonglong2* q = reinterpret_cast<const ulonglong2*>(rec + (size_t)c * RP);
      u64 r[RP];
#pragma unroll
      for (int j = 0; j < RP / 2; ++j) {
        const ulonglong2 v = q[j];
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
        u64 cv = mul2(r[D + 2], V[i][0]);                       // c~ . v
#pragma unroll
        for (int j = 1; j < D; ++j) cv = fma2(r[D + 2 + j], V[i][j], cv);
        const u64 p = mul2(e, cv);                               // e' (c . v)
        Z[i] = add2(Z[i], p);
#pragma unroll
        for (int j = 0; j < D; ++j) Y[i][j] = fma2(p, r[2 * D + 2 + j], Y[i][j]);
      }
    }
  } else {
    const u64 ng = pk(-gl2e, -gl2e);
    for (int c = 0; c < kWarpStage; ++c) {
      const u64* r = rec + (size_t)c * RP;
#pragma unroll
      for (int i = 0; i < P; ++i) {
        u64 dx[D];
#pragma unroll
        for (int j = 0; j < D; ++j) dx[j] = add2(U[i][j], r[j]);
        u64 r2 = mul2(dx[0], dx[0]);
        u64 rv = mul2(dx[0], V[i][0]);
#pragma unroll
        for (int j = 1; j < D; ++j) {
          r2 = fma2(dx[j], dx[j], r2);
          rv = fma2(dx[j], V[i][j], rv);
        }
        const u64 we = mul2(r[D + 1], ex2x2(fma2(r2, ng, r[D])));   // w phi
        S[i] = add2(S[i], we);
        const u64 wrv = mul2(we, rv);
#pragma unroll
        for (int j = 0; j < D; ++j) {
          G[i][j] = fma2(we, dx[j], G[i][j]);
          Y[i][j] = fma2(wrv, dx[j], Y[i][j]);                 // sum w phi ((x - mu) . v)(x - mu)
        }
      }
    }
  }
}

template <int D>
__global__ void __launch_bounds__(VjRbf<D>::kW * 32, 3)
k_vjp_rbf_fast(TileArgs a, int kseg, const float* __restrict__ ckpt, const float* __restrict__ gT,
               float* __restrict__ g0) {
  constexpr int W = VjRbf<D>::kW, K = VjRbf<D>::kK, P = K / 2, RP = VjRbf<D>::kPairs;
  constexpr int NS = VjRbf<D>::kSums, kTile = VjRbf<D>::kTile, KT = FastRec<D>::kTab;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64* wbuf = reinterpret_cast<u64*>(smem) + (size_t)warp * 2 * kWarpStage * RP;
  float* red = reinterpret_cast<float*>(smem);   // [W][NS][kTile], aliases the stages after a pass's last stage
  float4* wraw = reinterpret_cast<float4*>(smem + vj_rbf_region0<D>()) + (size_t)warp * kWarpStage * KT;
  float* seg = reinterpret_cast<float*>(smem + vj_rbf_region0<D>() +
                                        (size_t)W * kWarpStage * KT * sizeof(float4));   // [kseg][kTile][D]
  const int64_t p0 = (int64_t)blockIdx.x * kTile;
  const int64_t N = a.N, M = a.M;
  const float gamma = a.gamma, gl2e = gamma * kLog2e, eta = a.eta;
  const int64_t Mw = ((M + W - 1) / W + kWarpStage - 1) / kWarpStage * kWarpStage;
  const int64_t mbase = (int64_t)warp * Mw;
  const int nstage = (int)(Mw / kWarpStage);

  bool act[K];
  int64_t idx[K];
  float g[K][D], x[K][D];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int64_t p = p0 + k * 32 + lane;
    act[k] = p < N;
    idx[k] = act[k] ? (int64_t)a.perm[p] - a.perm_base : 0;
#pragma unroll
    for (int j = 0; j < D; ++j) g[k][j] = act[k] ? gT[idx[k] * D + j] : 0.0f;
  }

  const int nseg = a.T / kseg;
  for (int sgi = nseg - 1; sgi >= 0; --sgi) {
    const float* src = (sgi == 0 || ckpt == nullptr) ? a.x0 : ckpt + (int64_t)(sgi - 1) * N * D;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int j = 0; j < D; ++j) x[k][j] = act[k] ? src[idx[k] * D + j] : 0.0f;
    const int pre = (sgi > 0 && ckpt == nullptr) ? sgi * kseg : 0;   // no checkpoints: recompute from x0
    for (int i = 0; i < pre + kseg; ++i) {
      if (i >= pre) {
        if (warp == 0)
#pragma unroll
          for (int k = 0; k < K; ++k)
#pragma unroll
            for (int j = 0; j < D; ++j) seg[((i - pre) * kTile + k * 32 + lane) * D + j] = x[k][j];
        if (i == pre + kseg - 1) break;
      }
      // one forward step of the tile (every warp holds all its samples)
      float lo[D], hi[D], o[D];
      const bool expanded = tile_frame<D, K>(x, act, gl2e, lo, hi, o);
      u64 U[P][D], S[P], G[P][D];
#pragma unroll
      for (int q = 0; q < P; ++q) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
          U[q][j] = pk(x[2 * q][j] - o[j], x[2 * q + 1][j] - o[j]);
          G[q][j] = 0ull;
        }
        S[q] = 0ull;
      }
      stage_prefetch<D>(a.tab, M, mbase, wraw, lane);
      stage_build<D>(M, mbase, expanded, o, gl2e, wraw, wbuf, lane);
      __syncwarp();
      for (int st = 0; st < nstage; ++st) {
        if (st + 1 < nstage) stage_prefetch<D>(a.tab, M, mbase + (int64_t)(st + 1) * kWarpStage, wraw, lane);
        stage_accumulate<D, P>(wbuf + (size_t)(st & 1) * kWarpStage * RP, expanded, gl2e, U, S, G);
        if (st + 1 < nstage)
          stage_build<D>(M, mbase + (int64_t)(st + 1) * kWarpStage, expanded, o, gl2e, wraw,
                         wbuf + (size_t)((st + 1) & 1) * kWarpStage * RP, lane);
        __syncwarp();
      }
      tile_finish_step<D, W, K, false>(a, 0, p0, act, x, o, expanded, S, G, reinterpret_cast<float4*>(red), warp,
                                       lane);
    }
    __syncthreads();   // the segment's states are visible to every warp
    for (int i = kseg - 1; i >= 0; --i) {
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int j = 0; j < D; ++j) x[k][j] = seg[(i * kTile + k * 32 + lane) * D + j];
      float lo[D], hi[D], o[D];
      const bool expanded = tile_frame<D, K>(x, act, gl2e, lo, hi, o);
      u64 U[P][D], V[P][D], S[P], G[P][D], Z[P], Y[P][D];
#pragma unroll
      for (int q = 0; q < P; ++q) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
          U[q][j] = pk(x[2 * q][j] - o[j], x[2 * q + 1][j] - o[j]);
          V[q][j] = pk(g[2 * q][j], g[2 * q + 1][j]);
          G[q][j] = Y[q][j] = 0ull;
        }
        S[q] = Z[q] = 0ull;
      }
      stage_prefetch<D>(a.tab, M, mbase, wraw, lane);
      vj_stage_build<D>(M, mbase, expanded, o, gl2e, wraw, wbuf, lane);
      __syncwarp();
      for (int st = 0; st < nstage; ++st) {
        if (st + 1 < nstage) stage_prefetch<D>(a.tab, M, mbase + (int64_t)(st + 1) * kWarpStage, wraw, lane);
        vj_stage_accumulate<D, P>(wbuf + (size_t)(st & 1) * kWarpStage * RP, expanded, gl2e, U, V, S, G, Z, Y);
        if (st + 1 < nstage)
          vj_stage_build<D>(M, mbase + (int64_t)(st + 1) * kWarpStage, expanded, o, gl2e, wraw,
                            wbuf + (size_t)((st + 1) & 1) * kWarpStage * RP, lane);
        __syncwarp();
      }
      __syncthreads();   // every warp has finished its centres before the reduction buffer overwrites the stages
      float* rw = red + (size_t)warp * NS * kTile;
#pragma unroll
      for (int q = 0; q < P; ++q) {
        float v0, v1;
        upk(S[q], v0, v1);
        rw[(2 * q) * 32 + lane] = v0;
        rw[(2 * q + 1) * 32 + lane] = v1;
        upk(Z[q], v0, v1);
        rw[(1 + D) * kTile + (2 * q) * 32 + lane] = v0;
        rw[(1 + D) * kTile + (2 * q + 1) * 32 + lane] = v1;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          upk(G[q][j], v0, v1);
          rw[(1 + j) * kTile + (2 * q) * 32 + lane] = v0;
          rw[(1 + j) * kTile + (2 * q + 1) * 32 + lane] = v1;
          upk(Y[q][j], v0, v1);
          rw[(2 + D + j) * kTile + (2 * q) * 32 + lane] = v0;
          rw[(2 + D + j) * kTile + (2 * q + 1) * 32 + lane] = v1;
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < K; ++k) {
        float sum[NS];
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          float v = red[q * kTile + k * 32 + lane];
#pragma unroll
          for (int w = 1; w < W; ++w) v += red[((size_t)w * NS + q) * kTile + k * 32 + lane];
          sum[q] = v;
        }
        const float Ss = sum[0];
        float shat, gs[D], hv[D];
        if (expanded) {
          float u[D], u2 = 0.0f, uv = 0.0f;
#pragma unroll
          for (int j = 0; j < D; ++j) {
            u[j] = x[k][j] - o[j];
            u2 = fmaf(u[j], u[j], u2);
            uv = fmaf(u[j], g[k][j], uv);
          }
          const float f = ex2_approx(-gl2e * u2);
          shat = f * Ss;
#pragma unroll
          for (int j = 0; j < D; ++j) {
            const float usg = fmaf(u[j], Ss, -sum[1 + j]);                  // u S - G
            gs[j] = -2.0f * gamma * (f * usg);
            const float m = fmaf(uv, usg, -fmaf(u[j], sum[1 + D], -sum[2 + D + j]));   // (u.v)(uS-G) - (uK-Kc)
            hv[j] = 4.0f * gamma * gamma * f * m - 2.0f * gamma * f * Ss * g[k][j];
          }
        } else {
          shat = Ss;
#pragma unroll
          for (int j = 0; j < D; ++j) {
            gs[j] = -2.0f * gamma * sum[1 + j];
            hv[j] = 4.0f * gamma * gamma * sum[2 + D + j] - 2.0f * gamma * Ss * g[k][j];
          }
        }
        float d1, d2;
        sigmoid_d12(shat + a.bias, d1, d2);
        float gd = 0.0f;
#pragma unroll
        for (int j = 0; j < D; ++j) gd = fmaf(gs[j], g[k][j], gd);
#pragma unroll
        for (int j = 0; j < D; ++j) g[k][j] = g[k][j] - eta * fmaf(d1, hv[j], d2 * gd * gs[j]);
      }
      __syncthreads();   // every warp has read the reduction buffer before the next pass rebuilds the stages
    }
  }
  if (warp == 0)
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (act[k])
#pragma unroll
        for (int j = 0; j < D; ++j) g0[idx[k] * D + j] = g[k][j];
}

template <int D>
static cudaError_t launch_vjp_rbf_fast(const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, int k,
                                       const float* ckpt, const float* gT, float* g0, void* ws, cudaStream_t st) {
  float4* tab = reinterpret_cast<float4*>(ws);
  SortWs sw = sort_layout((char*)ws + rbf_fast_table_bytes(D, fa.M), D, N);
  k_rbf_table<D><<<(unsigned)((fa.M + 255) / 256), 256, 0, st>>>(fa.centres, fa.w, fa.M, tab);
  cudaError_t e = spatial_sort(D, x0, N, sw, st);
  if (e != cudaSuccess) return e;
  TileArgs a{};
  a.tab = tab;
  a.M = fa.M;
  a.gamma = fa.gamma;
  a.bias = fa.bias;
  a.eta = eta;
  a.T = T;
  a.x0 = x0;
  a.perm = sw.perm;
  a.perm_base = 0;
  a.N = N;
  a.kck = 1;
  const size_t smem = vj_rbf_smem<D>(k);
  e = cudaFuncSetAttribute(k_vjp_rbf_fast<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((N + VjRbf<D>::kTile - 1) / VjRbf<D>::kTile);
  k_vjp_rbf_fast<D><<<blocks, VjRbf<D>::kW * 32, smem, st>>>(a, k, ckpt, gT, g0);
  return cudaGetLastError();
}

cudaError_t vjp_rbf_fast(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, int k,
                         const float* ckpt, const float* gT, float* g0, void* ws, cudaStream_t st) {
  if (d == 2) return launch_vjp_rbf_fast<2>(fa, x0, N, T, eta, k, ckpt, gT, g0, ws, st);
  if (d == 3) return launch_vjp_rbf_fast<3>(fa, x0, N, T, eta, k, ckpt, gT, g0, ws, st);
  return cudaErrorInvalidValue;
}

}  // namespace pdmp
