// Log-det of the T-step map (Sec. 3.2, "Drawing Samples") for RBF fields in
// d = 2, 3 on the forward's spatially sorted tiles.
//
// With the tile's origin o, u = x - o, c_m = mu_m - o and the forward's
// e'_m = sg_m 2^(a_m + b_m . u) (so that w_m phi_m(x) = f e'_m with
// f = 2^(-g' |u|^2)), the sums
//   S = sum e',  G = sum e' c,  H = sum e' c c^T   (lower triangle)
// give s - bias = f S, grad s = -2 gamma f (u S - G) and
//   Hess s = 4 gamma^2 f (u u^T S - u G^T - G u^T + H) - 2 gamma f S I,
// so a feature costs the forward's 2d + 1 packed FP32 operations and one ex2,
// plus d (d + 1) / 2 for H.  Tiles too wide for the expanded form take the
// direct form (x - mu per feature; H = sum w phi (x - mu)(x - mu)^T).  Per
// sample and step: Hess c = sigma'(s) Hess s + sigma''(s) grad s grad s^T,
// the Cholesky log-det of I - eta Hess c, and the Euler update.
#include "fast_tile.cuh"
#include "kernels.cuh"
#include "sort.cuh"

namespace pdmp {

template <int D, int KK = (D == 2 ? 8 : 6)>
struct LdRbf {
  static constexpr int kH = D * (D + 1) / 2;             // lower-triangle entries
  static constexpr int kUsed = 2 * D + 2 + kH;           // u64 pairs a record uses
  static constexpr int kPairs = (kUsed + 1) / 2 * 2;     // padded to whole 16-byte chunks
  static constexpr int kSums = 1 + D + kH;               // S, G, H per sample
  static constexpr int kK = KK;                          // samples per lane (8 for d = 2, 6 for d = 3)
  static constexpr int kW = 4;                           // warps per tile
  static constexpr int kTile = 32 * kK;
};
template <int D>
constexpr int kLdK = LdRbf<D>::kK;

template <int D, int K = kLdK<D>>
__host__ __device__ constexpr size_t ld_rbf_region0() {
  using L = LdRbf<D, K>;
  return (size_t)L::kW * 2 * kWarpStage * L::kPairs * 8 > (size_t)L::kW * L::kSums * L::kTile * 4
             ? (size_t)L::kW * 2 * kWarpStage * L::kPairs * 8
             : (size_t)L::kW * L::kSums * L::kTile * 4;
}
template <int D, int K = kLdK<D>>
__host__ __device__ constexpr size_t ld_rbf_smem() {
  return ld_rbf_region0<D, K>() + (size_t)LdRbf<D, K>::kW * kWarpStage * FastRec<D>::kTab * sizeof(float4);
}

// lower-triangle entry q <-> (a, b), a >= b
template <int D>
__host__ __device__ constexpr int ld_row(int q) { return q < 1 ? 0 : (q < 3 ? 1 : 2); }
template <int D>
__host__ __device__ constexpr int ld_col(int q) { return q - ld_row<D>(q) * (ld_row<D>(q) + 1) / 2; }

// Records of centres [m0, m0 + kWarpStage) for the log-det sweep:
//   expanded: [a][b_0 ..][sg][c~_0 ..][h_q ..]  with c~ = sg c, h_q = sg c_a c_b
//   direct:   [-mu_0 ..][lw][sg] (rest zero)
template <int D>
__device__ __forceinline__ void ld_stage_build(int64_t M, int64_t m0, bool expanded, const float* o, float gl2e,
                                               const float4* raw, u64* rec, int lane) {
  constexpr int RP = LdRbf<D>::kPairs;
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
      r[D + 1] = pk(sg, sg);
#pragma unroll
      for (int q = 0; q < LdRbf<D>::kH; ++q) {
        const float h = sg * c[ld_row<D>(q)] * c[ld_col<D>(q)];
        r[2 * D + 2 + q] = pk(h, h);
      }
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

template <int D, int P>
__device__ __forceinline__ void ld_stage_accumulate(const u64* rec, bool expanded, float gl2e, const u64 (&U)[P][D],
                                                    u64 (&S)[P], u64 (&G)[P][D], u64 (&H)[P][LdRbf<D>::kH]) {
  constexpr int RP = LdRbf<D>::kPairs;
  constexpr int NH = LdRbf<D>::kH;
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
      // phased as the morph: arguments, ex2, then each sum over the pairs
      u64 e[P];
#pragma unroll
      for (int i = 0; i < P; ++i) e[i] = fma2(r[1], U[i][0], r[0]);
#pragma unroll
      for (int j = 1; j < D; ++j)
#pragma unroll
        for (int i = 0; i < P; ++i) e[i] = fma2(r[1 + j], U[i][j], e[i]);
#pragma unroll
      for (int i = 0; i < P; ++i) e[i] = ex2x2(e[i]);
#pragma unroll
      for (int i = 0; i < P; ++i) S[i] = fma2(r[D + 1], e[i], S[i]);
#pragma unroll
      for (int j = 0; j < D; ++j)
#pragma unroll
        for (int i = 0; i < P; ++i) G[i][j] = fma2(e[i], r[D + 2 + j], G[i][j]);
#pragma unroll
      for (int h = 0; h < NH; ++h)
#pragma unroll
        for (int i = 0; i < P; ++i) H[i][h] = fma2(e[i], r[2 * D + 2 + h], H[i][h]);
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
#pragma unroll
        for (int j = 1; j < D; ++j) r2 = fma2(dx[j], dx[j], r2);
        const u64 we = mul2(r[D + 1], ex2x2(fma2(r2, ng, r[D])));
        S[i] = add2(S[i], we);
#pragma unroll
        for (int j = 0; j < D; ++j) G[i][j] = fma2(we, dx[j], G[i][j]);
#pragma unroll
        for (int h = 0; h < NH; ++h) H[i][h] = fma2(mul2(we, dx[ld_row<D>(h)]), dx[ld_col<D>(h)], H[i][h]);
      }
    }
  }
}

// One sweep over the centres for the tile's samples x (every warp over its
// slice of M, double-buffered stages); the per-warp sums S, G, H land in red
// ([W][NS][kTile] floats, aliasing the stages).  Returns whether the tile took
// the expanded form, with its origin in o.  Ends with a block barrier after
// the sums are written; the caller must pass another barrier before the next
// sweep rebuilds the stages.
template <int D, int K = kLdK<D>>
__device__ __forceinline__ bool ld_sweep(const TileArgs& a, const float (&x)[K][D], const bool (&act)[K],
                                         float (&o)[D], unsigned char* smem, int warp, int lane) {
  using L = LdRbf<D, K>;
  constexpr int W = L::kW, P = K / 2, RP = L::kPairs, NH = L::kH;
  constexpr int NS = L::kSums, kTile = L::kTile, KT = FastRec<D>::kTab;
  u64* wbuf = reinterpret_cast<u64*>(smem) + (size_t)warp * 2 * kWarpStage * RP;
  float* red = reinterpret_cast<float*>(smem);
  float4* wraw = reinterpret_cast<float4*>(smem + ld_rbf_region0<D, K>()) + (size_t)warp * kWarpStage * KT;
  const int64_t M = a.M;
  const float gl2e = a.gamma * kLog2e;
  const int64_t Mw = ((M + W - 1) / W + kWarpStage - 1) / kWarpStage * kWarpStage;
  const int64_t mbase = (int64_t)warp * Mw;
  const int nstage = (int)(Mw / kWarpStage);

  float lo[D], hi[D];
  const bool expanded = tile_frame<D, K>(x, act, gl2e, lo, hi, o);
  u64 U[P][D], S[P], G[P][D], H[P][NH];
#pragma unroll
  for (int i = 0; i < P; ++i) {
#pragma unroll
    for (int j = 0; j < D; ++j) {
      U[i][j] = pk(x[2 * i][j] - o[j], x[2 * i + 1][j] - o[j]);
      G[i][j] = 0ull;
    }
#pragma unroll
    for (int h = 0; h < NH; ++h) H[i][h] = 0ull;
    S[i] = 0ull;
  }
  stage_prefetch<D>(a.tab, M, mbase, wraw, lane);
  ld_stage_build<D>(M, mbase, expanded, o, gl2e, wraw, wbuf, lane);
  __syncwarp();
  for (int st = 0; st < nstage; ++st) {
    if (st + 1 < nstage) stage_prefetch<D>(a.tab, M, mbase + (int64_t)(st + 1) * kWarpStage, wraw, lane);
    ld_stage_accumulate<D, P>(wbuf + (size_t)(st & 1) * kWarpStage * RP, expanded, gl2e, U, S, G, H);
    if (st + 1 < nstage)
      ld_stage_build<D>(M, mbase + (int64_t)(st + 1) * kWarpStage, expanded, o, gl2e, wraw,
                        wbuf + (size_t)((st + 1) & 1) * kWarpStage * RP, lane);
    __syncwarp();
  }
  __syncthreads();   // every warp has finished its centres before the reduction buffer overwrites the stages
#pragma unroll
  for (int i = 0; i < P; ++i) {
    float v0, v1;
    float* rw = red + (size_t)warp * NS * kTile;
    upk(S[i], v0, v1);
    rw[(2 * i) * 32 + lane] = v0;
    rw[(2 * i + 1) * 32 + lane] = v1;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      upk(G[i][j], v0, v1);
      rw[(1 + j) * kTile + (2 * i) * 32 + lane] = v0;
      rw[(1 + j) * kTile + (2 * i + 1) * 32 + lane] = v1;
    }
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      upk(H[i][h], v0, v1);
      rw[(1 + D + h) * kTile + (2 * i) * 32 + lane] = v0;
      rw[(1 + D + h) * kTile + (2 * i + 1) * 32 + lane] = v1;
    }
  }
  __syncthreads();
  return expanded;
}

// Sample k of this lane after ld_sweep: s - bias (shat), grad s (gs) and the
// lower triangle of Hess s (hs) at x.
template <int D, int K = kLdK<D>>
__device__ __forceinline__ void ld_sample_terms(const float* red, int k, int lane, const float (&x)[D],
                                                const float (&o)[D], bool expanded, float gamma, float& shat,
                                                float (&gs)[D], float (&hs)[D][D]) {
  using L = LdRbf<D, K>;
  constexpr int W = L::kW, NH = L::kH, NS = L::kSums, kTile = L::kTile;
  const float gl2e = gamma * kLog2e;
  float sum[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    float v = red[q * kTile + k * 32 + lane];
#pragma unroll
    for (int w = 1; w < W; ++w) v += red[((size_t)w * NS + q) * kTile + k * 32 + lane];
    sum[q] = v;
  }
  const float Ssum = sum[0];
  if (expanded) {
    float u[D], u2 = 0.0f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      u[j] = x[j] - o[j];
      u2 = fmaf(u[j], u[j], u2);
    }
    const float f = ex2_approx(-gl2e * u2);
    shat = f * Ssum;
#pragma unroll
    for (int j = 0; j < D; ++j) gs[j] = -2.0f * gamma * (f * fmaf(u[j], Ssum, -sum[1 + j]));   // as the morph
#pragma unroll
    for (int q = 0; q < NH; ++q) {
      const int ra = ld_row<D>(q), cb = ld_col<D>(q);
      // u_a u_b S - u_a G_b - G_a u_b + H_ab
      const float m2 = fmaf(u[ra] * u[cb], Ssum, -fmaf(u[ra], sum[1 + cb], u[cb] * sum[1 + ra])) + sum[1 + D + q];
      hs[ra][cb] = 4.0f * gamma * gamma * f * m2 - (ra == cb ? 2.0f * gamma * f * Ssum : 0.0f);
    }
  } else {
    shat = Ssum;
#pragma unroll
    for (int j = 0; j < D; ++j) gs[j] = -2.0f * gamma * sum[1 + j];
#pragma unroll
    for (int q = 0; q < NH; ++q) {
      const int ra = ld_row<D>(q), cb = ld_col<D>(q);
      hs[ra][cb] = 4.0f * gamma * gamma * sum[1 + D + q] - (ra == cb ? 2.0f * gamma * Ssum : 0.0f);
    }
  }
}

// log det (I - eta Hess c) with Hess c = sigma'(s) Hess s + sigma''(s) grad s grad s^T
// (d1 = sigma', d2 = sigma''), by Cholesky; NaN when a pivot is not positive
template <int D>
__device__ __forceinline__ float step_logdet(float d1, float d2, const float (&gs)[D], const float (&hs)[D][D],
                                             float eta) {
  float A[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      if (c <= r) {
        const float hc = fmaf(d1, hs[r][c], d2 * gs[r] * gs[c]);
        A[r][c] = (r == c ? 1.0f : 0.0f) - eta * hc;
      } else {
        A[r][c] = 0.0f;
      }
    }
  return chol_logdet<D>(A);
}

template <int D>
__global__ void __launch_bounds__(LdRbf<D>::kW * 32, 3)
k_logdet_rbf_fast(TileArgs a, float* __restrict__ logdet) {
  constexpr int K = LdRbf<D>::kK, kTile = LdRbf<D>::kTile;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float* red = reinterpret_cast<const float*>(smem);
  const int64_t p0 = (int64_t)blockIdx.x * kTile;
  const float eta = a.eta;

  float x[K][D];
  bool act[K];
  tile_load<D, K>(a, p0, a.N, lane, x, act);
  float total[K];
  bool bad[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    total[k] = 0.0f;
    bad[k] = false;
  }

  for (int t = 0; t < a.T; ++t) {
    float o[D];
    const bool expanded = ld_sweep<D>(a, x, act, o, smem, warp, lane);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float shat, gs[D], hs[D][D];
      ld_sample_terms<D>(red, k, lane, x[k], o, expanded, a.gamma, shat, gs, hs);
      float d1, d2;
      sigmoid_d12(shat + a.bias, d1, d2);
      const float ld = step_logdet<D>(d1, d2, gs, hs, eta);
      if (!(ld == ld)) bad[k] = true;
      total[k] += ld;
      const float cst = -eta * d1;
#pragma unroll
      for (int j = 0; j < D; ++j) x[k][j] = __fadd_rn(x[k][j], __fmul_rn(cst, gs[j]));
    }
    __syncthreads();   // every warp has read the reduction buffer before the next step rebuilds the stages
  }
  if (warp == 0) {
    bool any_bad = false;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (act[k]) {
        const int64_t n = (int64_t)a.perm[p0 + k * 32 + lane] - a.perm_base;
        logdet[n] = bad[k] ? nanf("") : total[k];
        any_bad = any_bad || bad[k];
        if (a.xT)
#pragma unroll
          for (int j = 0; j < D; ++j) a.xT[n * D + j] = x[k][j];
      }
    if (any_bad) raise_flag(FLAG_NONPOSITIVE_PIVOT);
  }
}

// ---------------------------------------------------------------- log-density
// The inverse map and the log-det in one sweep per fixed-point iteration: each
// iteration of step t evaluates S, G and H at the iterate y, takes the update
// y <- z + eta sigma'(s) grad s(y) from S and G, and keeps the step's
// log det (I - eta Hess c(y)) from all three.  The iteration that stops (every
// update below tol (1 + |y|)) leaves the log-det at its y, a point within the
// stopping tolerance of x_t, so the separate forward log-det sweep from the
// recovered x_0 is not needed.  Warm start and block-uniform stopping as the
// sorted-tile inverse (z + 2 delta_{t+1} - delta_{t+2} once two corrections
// are known).  a.x0 holds z; a.xT receives y = phi^{-1}(z); logdet receives
// sum_t log det J_t.
template <int D, int K>
__global__ void __launch_bounds__(LdRbf<D, K>::kW * 32, 3)
k_log_density_rbf_fast(TileArgs a, float tol, int maxit, float* __restrict__ logdet, int32_t* __restrict__ iters,
                       unsigned long long* __restrict__ work) {
  constexpr int kTile = LdRbf<D, K>::kTile;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float* red = reinterpret_cast<const float*>(smem);
  const int64_t p0 = (int64_t)blockIdx.x * kTile;
  const float eta = a.eta;
  float* zs = reinterpret_cast<float*>(smem + ld_rbf_smem<D, K>());   // kTile x D: the step's target z
  float* ds = zs + kTile * D;    // the corrections of the two steps undone before, kTile x D each
  float* ds2 = ds + kTile * D;

  float y[K][D];
  bool act[K];
  tile_load<D, K>(a, p0, a.N, lane, y, act);
  if (warp == 0)
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        zs[(k * 32 + lane) * D + j] = y[k][j];
        ds[(k * 32 + lane) * D + j] = 0.0f;
        ds2[(k * 32 + lane) * D + j] = 0.0f;
      }
  float total[K];
  bool bad[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    total[k] = 0.0f;
    bad[k] = false;
  }
  int worst = 0;
  long long its = 0;
  for (int t = a.T - 1; t >= 0; --t) {
    __syncthreads();   // the step's target z and the last corrections (written by warp 0) are visible; y = z
    const float c1 = t <= a.T - 3 ? 2.0f : 1.0f, c2 = t <= a.T - 3 ? 1.0f : 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const int q = (k * 32 + lane) * D + j;
        y[k][j] += fmaf(c1, ds[q], -c2 * ds2[q]);
      }
    float ld[K];
    int it = 0;
    bool moving = true;
    while (moving && it < maxit) {
      float o[D];
      const bool expanded = ld_sweep<D, K>(a, y, act, o, smem, warp, lane);
      bool mv = false;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        float shat, gs[D], hs[D][D];
        ld_sample_terms<D, K>(red, k, lane, y[k], o, expanded, a.gamma, shat, gs, hs);
        float d1, d2;
        sigmoid_d12(shat + a.bias, d1, d2);
        ld[k] = step_logdet<D>(d1, d2, gs, hs, eta);
        const float c = eta * d1;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          const float yn = fmaf(c, gs[j], zs[(k * 32 + lane) * D + j]);   // z + eta sigma'(s) grad s(y)
          if (act[k] && fabsf(yn - y[k][j]) > tol * (1.0f + fabsf(yn))) mv = true;
          y[k][j] = yn;
        }
      }
      ++it;
      // every warp has read the reduction buffer before the next iteration rebuilds the stages
      moving = __syncthreads_or(mv) != 0;
    }
    if (moving && threadIdx.x == 0) raise_flag(FLAG_NOT_CONVERGED);
    worst = it > worst ? it : worst;
    its += it;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (!(ld[k] == ld[k])) bad[k] = true;
      total[k] += ld[k];
    }
    // the converged y is the next (earlier) step's target; every warp has
    // read zs in the last iteration (the barrier in __syncthreads_or)
    if (warp == 0)
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int j = 0; j < D; ++j) {
          const int q = (k * 32 + lane) * D + j;
          ds2[q] = ds[q];
          ds[q] = y[k][j] - zs[q];
          zs[q] = y[k][j];
        }
  }
  if (warp == 0) {
    bool any_bad = false;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (act[k]) {
        const int64_t n = (int64_t)a.perm[p0 + k * 32 + lane] - a.perm_base;
        logdet[n] = bad[k] ? nanf("") : total[k];
        any_bad = any_bad || bad[k];
#pragma unroll
        for (int j = 0; j < D; ++j) a.xT[n * D + j] = y[k][j];
        if (iters) iters[n] = worst;
      }
    if (any_bad) raise_flag(FLAG_NONPOSITIVE_PIVOT);
  }
  if (work != nullptr && threadIdx.x == 0) {
    const int64_t cnt = min64(kTile, a.N - p0);
    atomicAdd(work, (unsigned long long)its * (unsigned long long)cnt * (unsigned long long)a.M);
  }
}

template <int D>
static cudaError_t launch_logdet_rbf_fast(const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* ld,
                                          float* xT, void* ws, cudaStream_t st) {
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
  a.xT = xT;
  constexpr size_t smem = ld_rbf_smem<D>();
  e = cudaFuncSetAttribute(k_logdet_rbf_fast<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((N + LdRbf<D>::kTile - 1) / LdRbf<D>::kTile);
  k_logdet_rbf_fast<D><<<blocks, LdRbf<D>::kW * 32, smem, st>>>(a, ld);
  return cudaGetLastError();
}

template <int D, int K>
static cudaError_t launch_log_density_shape(const TileArgs& a, float tol, int maxit, float* ld, int32_t* iters,
                                            unsigned long long* work, cudaStream_t st) {
  constexpr size_t smem = ld_rbf_smem<D, K>() + 3 * (size_t)LdRbf<D, K>::kTile * D * sizeof(float);
  cudaError_t e =
      cudaFuncSetAttribute(k_log_density_rbf_fast<D, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((a.N + LdRbf<D, K>::kTile - 1) / LdRbf<D, K>::kTile);
  k_log_density_rbf_fast<D, K><<<blocks, LdRbf<D, K>::kW * 32, smem, st>>>(a, tol, maxit, ld, iters, work);
  return cudaGetLastError();
}

template <int D>
static cudaError_t launch_log_density_rbf_fast(const FieldArgs& fa, const float* z, int64_t N, int T, float eta,
                                               float tol, int maxit, float* y, float* ld, int32_t* iters,
                                               unsigned long long* work, void* ws, cudaStream_t st) {
  float4* tab = reinterpret_cast<float4*>(ws);
  SortWs sw = sort_layout((char*)ws + rbf_fast_table_bytes(D, fa.M), D, N);
  k_rbf_table<D><<<(unsigned)((fa.M + 255) / 256), 256, 0, st>>>(fa.centres, fa.w, fa.M, tab);
  cudaError_t e = spatial_sort(D, z, N, sw, st);
  if (e != cudaSuccess) return e;
  TileArgs a{};
  a.tab = tab;
  a.M = fa.M;
  a.gamma = fa.gamma;
  a.bias = fa.bias;
  a.eta = eta;
  a.T = T;
  a.x0 = z;
  a.perm = sw.perm;
  a.perm_base = 0;
  a.N = N;
  a.xT = y;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess || sms < 1)
    sms = 152;
  // 128-sample tiles for launches of fewer than two waves of the larger ones
  // (3 blocks per SM), which then fill the GPU and stop iterating tile by tile
  const int64_t tiles = (N + LdRbf<D>::kTile - 1) / LdRbf<D>::kTile;
  if (tiles < 2 * 3 * (int64_t)sms) return launch_log_density_shape<D, 4>(a, tol, maxit, ld, iters, work, st);
  return launch_log_density_shape<D, kLdK<D>>(a, tol, maxit, ld, iters, work, st);
}

cudaError_t log_density_rbf_fast(int d, const FieldArgs& fa, const float* z, int64_t N, int T, float eta, float tol,
                                 int maxit, float* y, float* ld, int32_t* iters, unsigned long long* work, void* ws,
                                 cudaStream_t st) {
  if (d == 2) return launch_log_density_rbf_fast<2>(fa, z, N, T, eta, tol, maxit, y, ld, iters, work, ws, st);
  if (d == 3) return launch_log_density_rbf_fast<3>(fa, z, N, T, eta, tol, maxit, y, ld, iters, work, ws, st);
  return cudaErrorInvalidValue;
}

cudaError_t logdet_rbf_fast(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* ld,
                            float* xT, void* ws, cudaStream_t st) {
  if (d == 2) return launch_logdet_rbf_fast<2>(fa, x0, N, T, eta, ld, xT, ws, st);
  if (d == 3) return launch_logdet_rbf_fast<3>(fa, x0, N, T, eta, ld, xT, ws, st);
  return cudaErrorInvalidValue;
}

}  // namespace pdmp
