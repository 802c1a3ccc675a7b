// VJP of the T-step map (g_t = (I - eta Hess c(x_t)) g_{t+1}) for RBF fields
// in d = 2, 3 on the forward's spatially sorted tiles.
//
// Segment by segment (last first), the tile's states are recomputed from the
// checkpoint with the forward's tile step and kept in shared memory; each
// step back is one pass over the features at x_t with v = g.  With the
// tile's origin o, u = x - o, c_m = mu_m - o and e'_m = sg_m 2^(a_m + b_m . u)
// (w_m phi_m = f e'_m, f = 2^(-g' |u|^2)), the pass sums the moments
//   S = sum e',  G = sum e' c,  H = sum e' c c^T,
// which give grad s = -2 gamma f (u S - G) and
//   (Hess s) v = 4 gamma^2 f ((u . v)(u S - G) - (u (v . G) - H v)) - 2 gamma f S v
// (sum e' (c . v) = v . G and sum e' (c . v) c = H v, so v enters only per
// sample): 2d + 1 + d(d + 1)/2 packed FP32 operations and one ex2 per sample
// pair and feature, 8 for d = 2.  Tiles too wide for the expanded form take
// the direct form.
//
// Weight gradient (optional).  Sample n adds to d/dw_m, with g = g_{t+1},
//   cA phi_m + cB grad phi_m . g = phi_m (alpha + beta . c_m),
//   cA = -eta sigma'' (grad s . g),  cB = -eta sigma',
//   alpha = cA - 2 gamma cB (u . g),  beta = 2 gamma cB g
// (grad phi_m = -2 gamma phi_m (u - c_m)).  After each Hessian-vector pass
// warp 0 writes u, f alpha and f beta of the tile's samples to shared memory;
// then the sweep is transposed: each lane owns features and sums over the
// tile's sample pairs (phi_m / f = 2^(b_m . u - g' |c_m|^2), 2d + 1 packed
// FP32 operations and one ex2 per pair, as in the forward), so no feature
// needs a reduction across lanes or warps; the block's sums go to its own
// row of the workspace, summed over blocks in a fixed order.
#include "fast_tile.cuh"
#include "kernels.cuh"
#include "sort.cuh"

namespace pdmp {

template <int D>
struct VjRbf {
  static constexpr int kH = D * (D + 1) / 2;           // lower-triangle entries of H
  static constexpr int kUsed = 2 * D + 2 + kH;         // u64 pairs: a, b, sg, c~ = sg c, h = sg c_a c_b
  // whole 16-byte chunks, an odd number of them: the lanes of a quarter warp
  // building consecutive records then write to distinct banks
  static constexpr int kChunks = (kUsed + 1) / 2 % 2 == 1 ? (kUsed + 1) / 2 : (kUsed + 1) / 2 + 1;
  static constexpr int kPairs = 2 * kChunks;
  static constexpr int kSums = 1 + D + kH;             // S, G, H (direct: S, G, P in the first D of H)
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
// region 0 (stages / reduction), the raw table entries, the segment's states,
// and with the weight gradient the tile's sample terms (u, f alpha, f beta)
// (and with the cache, the forward's S and G at each of the segment's states)
template <int D>
__host__ __device__ constexpr size_t vj_rbf_smem(int kseg, bool want_gw = false, bool cache = false) {
  return vj_rbf_region0<D>() + (size_t)VjRbf<D>::kW * kWarpStage * FastRec<D>::kTab * sizeof(float4) +
         (size_t)kseg * VjRbf<D>::kTile * D * sizeof(float) +
         (cache ? (size_t)kseg * (1 + D) * VjRbf<D>::kTile * sizeof(float) : 0) +
         (want_gw ? (size_t)(2 * D + 2) * VjRbf<D>::kTile * sizeof(float) : 0);
}

constexpr int kGwFeatures = 4;   // features per lane in the weight-gradient sweep

// Sample terms of the weight-gradient sweep, per pair of samples (2p, 2p + 1):
// 2D + 2 packed pairs [u_0 .. u_{D-1}, f alpha, f beta_0 .. f beta_{D-1}, 0],
// so that a pair's terms are D + 1 16-byte loads.
template <int D>
struct GwTerms {
  static constexpr int kPairs = 2 * D + 2;
  __device__ static void put(float* sm, int s, int slot, float v) {
    sm[((s >> 1) * kPairs + slot) * 2 + (s & 1)] = v;
  }
};

// The weight-gradient sweep of one warp over its slice [m_lo, m_hi) of the
// features (sm: the tile's sample terms); adds each feature's sum to row[m].
template <int D, int kTile>
__device__ __forceinline__ void vj_gw_sweep(const float4* __restrict__ tab, int64_t m_lo, int64_t m_hi,
                                            bool expanded, const float* o, float gl2e, const float* sm,
                                            float* __restrict__ row, int lane) {
  constexpr int TP = GwTerms<D>::kPairs;
  constexpr int KT = FastRec<D>::kTab;
  constexpr int F = kGwFeatures;
  for (int64_t m0 = m_lo; m0 < m_hi; m0 += 32 * F) {
    u64 cst[F], bm[F][D], A[F], Q[F][D];
    float c[F][D];
    bool ok[F];
#pragma unroll
    for (int f = 0; f < F; ++f) {
      const int64_t m = m0 + f * 32 + lane;
      ok[f] = m < m_hi;
      float mu[D];
      if (ok[f]) {
        const float4 t0 = tab[KT * m];
        mu[0] = t0.x;
        mu[1] = t0.y;
        if (D == 3) mu[2] = t0.z;
      } else {
#pragma unroll
        for (int j = 0; j < D; ++j) mu[j] = o[j];
      }
      float c2 = 0.0f;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        c[f][j] = mu[j] - o[j];   // direct form: o = 0
        c2 = fmaf(c[f][j], c[f][j], c2);
      }
      if (expanded) {   // log2(phi / f) = -g' |c|^2 + 2 g' c . u
        const float a0 = ok[f] ? -gl2e * c2 : -INFINITY;
        cst[f] = pk(a0, a0);
#pragma unroll
        for (int j = 0; j < D; ++j) bm[f][j] = pk(2.0f * gl2e * c[f][j], 2.0f * gl2e * c[f][j]);
      } else {          // log2 phi = -g' |x - mu|^2
        const float nm = ok[f] ? -gl2e : -INFINITY;
        cst[f] = pk(nm, nm);
#pragma unroll
        for (int j = 0; j < D; ++j) bm[f][j] = pk(-mu[j], -mu[j]);
      }
      A[f] = 0ull;
#pragma unroll
      for (int j = 0; j < D; ++j) Q[f][j] = 0ull;
    }
#pragma unroll 2
    for (int p = 0; p < kTile / 2; ++p) {
      const ulonglong2* q = reinterpret_cast<const ulonglong2*>(sm + (size_t)p * TP * 2);
      u64 t[TP];
#pragma unroll
      for (int h = 0; h < TP / 2; ++h) {
        const ulonglong2 v = q[h];
        t[2 * h] = v.x;
        t[2 * h + 1] = v.y;
      }
      u64 up[D], bp[D];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        up[j] = t[j];
        bp[j] = t[D + 1 + j];
      }
      const u64 al = t[D];
#pragma unroll
      for (int f = 0; f < F; ++f) {
        u64 e;
        if (expanded) {
          e = fma2(bm[f][0], up[0], cst[f]);
#pragma unroll
          for (int j = 1; j < D; ++j) e = fma2(bm[f][j], up[j], e);
        } else {
          u64 r2 = 0ull;
#pragma unroll
          for (int j = 0; j < D; ++j) {
            const u64 dx = add2(up[j], bm[f][j]);
            r2 = fma2(dx, dx, r2);
          }
          e = mul2(r2, cst[f]);
        }
        e = ex2x2(e);
        A[f] = fma2(e, al, A[f]);
#pragma unroll
        for (int j = 0; j < D; ++j) Q[f][j] = fma2(e, bp[j], Q[f][j]);
      }
    }
#pragma unroll
    for (int f = 0; f < F; ++f) {
      if (!ok[f]) continue;
      float lo, hi;
      upk(A[f], lo, hi);
      float v = lo + hi;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        upk(Q[f][j], lo, hi);
        v = fmaf(c[f][j], lo + hi, v);
      }
      row[m0 + f * 32 + lane] += v;
    }
  }
}

//   expanded: [a][b_0 ..][sg][c~_0 ..][h_q ..] (h_q = sg c_a c_b)     direct: [-mu_0 ..][lw][sg] (rest zero)
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
      }
#pragma unroll
      for (int ia = 0; ia < D; ++ia)
#pragma unroll
        for (int ib = 0; ib <= ia; ++ib) {
          const float h = sg * c[ia] * c[ib];
          r[2 * D + 2 + ia * (ia + 1) / 2 + ib] = pk(h, h);
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

// sums of one pass at u (U) with v (V): S, G and H (expanded), or S, G and
// P = sum w phi ((x - mu) . v)(x - mu) in the first D entries of H (direct)
// (without SG, S and G are left alone: the caller has them from the recompute)
template <int D, int P, bool SG>
__device__ __forceinline__ void vj_stage_accumulate(const u64* rec, bool expanded, float gl2e, const u64 (&U)[P][D],
                                                    const u64 (&V)[P][D], u64 (&S)[P], u64 (&G)[P][D],
                                                    u64 (&H)[P][VjRbf<D>::kH]) {
  constexpr int NH = VjRbf<D>::kH;
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
        if (SG) {
          S[i] = fma2(r[D + 1], e, S[i]);
#pragma unroll
          for (int j = 0; j < D; ++j) G[i][j] = fma2(e, r[D + 2 + j], G[i][j]);
        }
#pragma unroll
        for (int q = 0; q < NH; ++q) H[i][q] = fma2(e, r[2 * D + 2 + q], H[i][q]);
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
        if (SG) S[i] = add2(S[i], we);
        const u64 wrv = mul2(we, rv);
#pragma unroll
        for (int j = 0; j < D; ++j) {
          if (SG) G[i][j] = fma2(we, dx[j], G[i][j]);
          H[i][j] = fma2(wrv, dx[j], H[i][j]);                 // sum w phi ((x - mu) . v)(x - mu)
        }
      }
    }
  }
}

template <int D, bool GW>
__global__ void __launch_bounds__(VjRbf<D>::kW * 32, 3)
k_vjp_rbf_fast(TileArgs a, int kseg, const float* __restrict__ ckpt, const float* __restrict__ gT,
               float* __restrict__ g0, float* __restrict__ rows, int use_cache) {
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
  // weight gradient: this block's row of rows[blocks][M + 1] and the sample terms after the segment
  float* row = GW ? rows + (int64_t)blockIdx.x * (M + 1) : nullptr;
  // the forward's S, G (cross-warp totals) at the segment's states: [kseg][1 + D][kTile]
  float* sgc = seg + (size_t)kseg * kTile * D;
  float* sm_gw = sgc + (use_cache ? (size_t)kseg * (1 + D) * kTile : 0);   // [kTile / 2][2D + 2] packed pairs
  if (GW)
    for (int64_t m = threadIdx.x; m <= M; m += blockDim.x) row[m] = 0.0f;
  float gb = 0.0f;   // warp 0: the bias term of this lane's samples

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
      if (use_cache && i >= pre) {
        // the step's totals, added in the finish's order, for the Hessian-vector pass at the same state
        const float4* r4 = reinterpret_cast<const float4*>(red);
        if (warp == 0)
#pragma unroll
          for (int k = 0; k < K; ++k) {
            float4 acc = r4[k * 32 + lane];
#pragma unroll
            for (int w = 1; w < W; ++w) {
              const float4 b = r4[w * kTile + k * 32 + lane];
              acc.x += b.x;
              acc.y += b.y;
              acc.z += b.z;
              acc.w += b.w;
            }
            float* dst = sgc + (size_t)(i - pre) * (1 + D) * kTile + k * 32 + lane;
            dst[0] = acc.x;
            dst[kTile] = acc.y;
            dst[2 * kTile] = acc.z;
            if (D == 3) dst[3 * kTile] = acc.w;
          }
        __syncthreads();   // read before the next step's stages overwrite the buffer
      }
    }
    __syncthreads();   // the segment's states (and totals) are visible to every warp
    for (int i = kseg - 1; i >= 0; --i) {
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int j = 0; j < D; ++j) x[k][j] = seg[(i * kTile + k * 32 + lane) * D + j];
      float lo[D], hi[D], o[D];
      const bool expanded = tile_frame<D, K>(x, act, gl2e, lo, hi, o);
      const bool have = use_cache && i < kseg - 1;   // S and G at this state from the recompute
      constexpr int NH = VjRbf<D>::kH;
      u64 U[P][D], V[P][D], S[P], G[P][D], H[P][NH];
#pragma unroll
      for (int q = 0; q < P; ++q) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
          U[q][j] = pk(x[2 * q][j] - o[j], x[2 * q + 1][j] - o[j]);
          V[q][j] = pk(g[2 * q][j], g[2 * q + 1][j]);
          G[q][j] = 0ull;
        }
#pragma unroll
        for (int h = 0; h < NH; ++h) H[q][h] = 0ull;
        S[q] = 0ull;
      }
      stage_prefetch<D>(a.tab, M, mbase, wraw, lane);
      vj_stage_build<D>(M, mbase, expanded, o, gl2e, wraw, wbuf, lane);
      __syncwarp();
      for (int st = 0; st < nstage; ++st) {
        if (st + 1 < nstage) stage_prefetch<D>(a.tab, M, mbase + (int64_t)(st + 1) * kWarpStage, wraw, lane);
        if (have)
          vj_stage_accumulate<D, P, false>(wbuf + (size_t)(st & 1) * kWarpStage * RP, expanded, gl2e, U, V, S, G, H);
        else
          vj_stage_accumulate<D, P, true>(wbuf + (size_t)(st & 1) * kWarpStage * RP, expanded, gl2e, U, V, S, G, H);
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
        if (!have) {
          upk(S[q], v0, v1);
          rw[(2 * q) * 32 + lane] = v0;
          rw[(2 * q + 1) * 32 + lane] = v1;
#pragma unroll
          for (int j = 0; j < D; ++j) {
            upk(G[q][j], v0, v1);
            rw[(1 + j) * kTile + (2 * q) * 32 + lane] = v0;
            rw[(1 + j) * kTile + (2 * q + 1) * 32 + lane] = v1;
          }
        }
#pragma unroll
        for (int h = 0; h < NH; ++h) {   // H (direct: P in the first D)
          upk(H[q][h], v0, v1);
          rw[(1 + D + h) * kTile + (2 * q) * 32 + lane] = v0;
          rw[(1 + D + h) * kTile + (2 * q + 1) * 32 + lane] = v1;
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < K; ++k) {
        float sum[NS];
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          if (have && q <= D) {   // the recompute's totals at this state
            sum[q] = sgc[((size_t)i * (1 + D) + q) * kTile + k * 32 + lane];
            continue;
          }
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
          float vG = 0.0f;   // K = sum e' (c . v) = v . G
#pragma unroll
          for (int j = 0; j < D; ++j) vG = fmaf(g[k][j], sum[1 + j], vG);
#pragma unroll
          for (int j = 0; j < D; ++j) {
            float Hv = 0.0f;   // Kc_j = (H v)_j, H from its lower triangle
#pragma unroll
            for (int i2 = 0; i2 < D; ++i2) {
              const int q = j >= i2 ? j * (j + 1) / 2 + i2 : i2 * (i2 + 1) / 2 + j;
              Hv = fmaf(sum[1 + D + q], g[k][i2], Hv);
            }
            const float usg = fmaf(u[j], Ss, -sum[1 + j]);                  // u S - G
            gs[j] = -2.0f * gamma * (f * usg);
            const float m = fmaf(uv, usg, -fmaf(u[j], vG, -Hv));            // (u.v)(uS-G) - (u K - Kc)
            hv[j] = 4.0f * gamma * gamma * f * m - 2.0f * gamma * f * Ss * g[k][j];
          }
        } else {
          shat = Ss;
#pragma unroll
          for (int j = 0; j < D; ++j) {
            gs[j] = -2.0f * gamma * sum[1 + j];
            hv[j] = 4.0f * gamma * gamma * sum[1 + D + j] - 2.0f * gamma * Ss * g[k][j];
          }
        }
        float d1, d2;
        sigmoid_d12(shat + a.bias, d1, d2);
        float gd = 0.0f;
#pragma unroll
        for (int j = 0; j < D; ++j) gd = fmaf(gs[j], g[k][j], gd);
        if (GW && warp == 0) {   // the sample's weight-gradient terms, with g_{t+1}
          const int sidx = k * 32 + lane;
          const float cA = act[k] ? -eta * d2 * gd : 0.0f, cB = act[k] ? -eta * d1 : 0.0f;
          float u[D], ug = 0.0f, f = 1.0f, u2 = 0.0f;
#pragma unroll
          for (int j = 0; j < D; ++j) {
            // direct form: o = 0; an empty slot sits at the origin, where phi / f <= 1 stays finite
            u[j] = act[k] ? x[k][j] - o[j] : 0.0f;
            ug = fmaf(u[j], g[k][j], ug);
            u2 = fmaf(u[j], u[j], u2);
          }
          if (expanded) f = ex2_approx(-gl2e * u2);
          gb += cA;
#pragma unroll
          for (int j = 0; j < D; ++j) {
            GwTerms<D>::put(sm_gw, sidx, j, u[j]);
            GwTerms<D>::put(sm_gw, sidx, D + 1 + j, f * (2.0f * gamma * cB * g[k][j]));
          }
          GwTerms<D>::put(sm_gw, sidx, D, f * fmaf(-2.0f * gamma * cB, ug, cA));
          GwTerms<D>::put(sm_gw, sidx, 2 * D + 1, 0.0f);
        }
#pragma unroll
        for (int j = 0; j < D; ++j) g[k][j] = g[k][j] - eta * fmaf(d1, hv[j], d2 * gd * gs[j]);
      }
      __syncthreads();   // every warp has read the reduction buffer before the next pass rebuilds the stages
      if (GW)            // (and the sample terms are visible)
        vj_gw_sweep<D, kTile>(a.tab, mbase, mbase + Mw < M ? mbase + Mw : M, expanded, o, gl2e, sm_gw, row, lane);
    }
  }
  if (GW && warp == 0) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) gb += __shfl_xor_sync(0xffffffffu, gb, off);
    if (lane == 0) row[M] = gb;
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
                                       const float* ckpt, const float* gT, float* g0, float* rows, float* gw,
                                       float* gbias, void* ws, cudaStream_t st) {
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
  const bool want = rows != nullptr;
  const void* fn = want ? reinterpret_cast<const void*>(k_vjp_rbf_fast<D, true>)
                        : reinterpret_cast<const void*>(k_vjp_rbf_fast<D, false>);
  // cache the recompute's S and G when the extra shared memory keeps as many blocks on an SM
  const size_t smem0 = vj_rbf_smem<D>(k, want, false), smem1 = vj_rbf_smem<D>(k, want, true);
  int b0 = 0, b1 = 0;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, fn, VjRbf<D>::kW * 32, smem0);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, fn, VjRbf<D>::kW * 32, smem1);
  if (e != cudaSuccess) return e;
  const int use_cache = b1 >= b0 && b1 > 0 ? 1 : 0;
  const size_t smem = use_cache ? smem1 : smem0;
  const unsigned blocks = (unsigned)vjp_rbf_fast_blocks(D, N);
  if (!want) {
    k_vjp_rbf_fast<D, false><<<blocks, VjRbf<D>::kW * 32, smem, st>>>(a, k, ckpt, gT, g0, nullptr, use_cache);
    return cudaGetLastError();
  }
  k_vjp_rbf_fast<D, true><<<blocks, VjRbf<D>::kW * 32, smem, st>>>(a, k, ckpt, gT, g0, rows, use_cache);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return sum_vjp_rows(rows, (int64_t)blocks, fa.M + 1, gw, gbias, st);
}

int64_t vjp_rbf_fast_blocks(int d, int64_t N) {
  const int64_t tile = d == 2 ? VjRbf<2>::kTile : VjRbf<3>::kTile;
  return (N + tile - 1) / tile;
}

cudaError_t vjp_rbf_fast(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, int k,
                         const float* ckpt, const float* gT, float* g0, float* rows, float* gw, float* gbias,
                         void* ws, cudaStream_t st) {
  if (d == 2) return launch_vjp_rbf_fast<2>(fa, x0, N, T, eta, k, ckpt, gT, g0, rows, gw, gbias, ws, st);
  if (d == 3) return launch_vjp_rbf_fast<3>(fa, x0, N, T, eta, k, ckpt, gT, g0, rows, gw, gbias, ws, st);
  return cudaErrorInvalidValue;
}

}  // namespace pdmp
