// Per-tile device code of the fast RBF morph (d = 2, 3), shared by the
// single-field launch (morph_rbf_fast.cu) and the batched launch (batch.cu).
//
#pragma once
#include "field.cuh"

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
// TF32 tensor-core pieces: round to TF32 (nearest, ties away), and
// D += A B for one m16n8k8 tile (A row-major 16 x 8, B column-major 8 x 8, FP32
// accumulate).  Fragments: with g = lane / 4 and t = lane % 4, a0 = A[g][t],
// a1 = A[g + 8][t], a2 = A[g][t + 4], a3 = A[g + 8][t + 4]; b0 = B[t][g],
// b1 = B[t + 4][g]; d0 = D[g][2t], d1 = D[g][2t + 1], d2 = D[g + 8][2t],
// d3 = D[g + 8][2t + 1].
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ u64 ex2x2(u64 a) {
  float lo, hi;
  upk(a, lo, hi);
  return pk(ex2_approx(lo), ex2_approx(hi));
}
// 2^-a of both halves
__device__ __forceinline__ u64 ex2x2_neg(u64 a) {
  float lo, hi;
  upk(a, lo, hi);
  return pk(ex2_approx(-lo), ex2_approx(-hi));
}

// Tile shape: W warps per block (each summing over its share of M) and K
// samples per lane (even: f32x2 pairs).  The single-field launch uses
// W = 4, K = 10 (measured fastest on the 2-D fitted workload among K = 6..16,
// W = 2..8, unroll 1..4 and 32..128-centre stages); the batched launch picks
// among a few shapes (autotuned).  Shapes with K > 8 need more than 128
// registers a thread and run 12 warps per SM, the others 16.
// The expanded exponent a_m + b_m . u carries a rounding error of about
// 2^-24 (|a_m| + |b_m . u|) <= 2^-24 3 g' R^2 for the features that matter
// (those within a few widths of the sample), i.e. a relative error of about
// 1.4e-6 in each feature at g' R^2 = 8; wider tiles take the direct form.
#ifndef PDMP_EXPAND_LIMIT
#define PDMP_EXPAND_LIMIT 8.0f
#endif
#ifndef PDMP_WARP_STAGE
#define PDMP_WARP_STAGE 64
#endif
#ifndef PDMP_FAST_UNROLL
#define PDMP_FAST_UNROLL 2
#endif
constexpr int kWarpStage = PDMP_WARP_STAGE;    // centres per warp per shared-memory stage
constexpr int kFastUnroll = PDMP_FAST_UNROLL;  // centres per unrolled inner iteration

template <int W, int K>
struct Shape {
  static_assert(K % 2 == 0, "samples per lane must be even (f32x2 pairs)");
  static constexpr int kWarps = W, kThreads = 32 * W, kK = K, kPairs = K / 2, kTile = 32 * K;
  static constexpr int kMinBlocks = (K > 8 ? 12 : 16) / W;   // warps per SM / warps per block
};

using FastShape = Shape<4, 10>;                // the single-field launch

template <int D>
struct FastRec {
  static constexpr int kPairs = 2 * D + 2;     // u64 pairs per staged centre
  static constexpr int kTab = D == 2 ? 1 : 2;  // float4s per centre in the table
};

// Shared memory of one tile: per warp, two stages of transformed records
// (aliased, after a step's last stage, by the cross-warp reduction buffer),
// then per warp the raw table entries of the stage being prefetched.
template <int D, int W>
__host__ __device__ constexpr size_t fast_bufs_bytes() {
  return (size_t)W * 2 * kWarpStage * FastRec<D>::kPairs * sizeof(u64);
}
template <int W, int K>
__host__ __device__ constexpr size_t fast_red_bytes() {
  return (size_t)W * (32 * K) * sizeof(float4);
}
template <int D, int W, int K>
__host__ __device__ constexpr size_t fast_region0_bytes() {
  return fast_bufs_bytes<D, W>() > fast_red_bytes<W, K>() ? fast_bufs_bytes<D, W>() : fast_red_bytes<W, K>();
}
template <int D, int W, int K>
__host__ __device__ constexpr size_t fast_smem_bytes() {
  return fast_region0_bytes<D, W, K>() + (size_t)W * kWarpStage * FastRec<D>::kTab * sizeof(float4);
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

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

// One warp copies the table entries of centres [m0, m0 + kWarpStage) into
// its raw buffer (asynchronously; each lane copies the entries it later
// transforms).
template <int D>
__device__ __forceinline__ void stage_prefetch(const float4* __restrict__ tab, int64_t M, int64_t m0, float4* raw,
                                               int lane) {
  constexpr int KT = FastRec<D>::kTab;
  for (int i = lane; i < kWarpStage; i += 32) {
    const int64_t m = m0 + i;
    if (m < M)
#pragma unroll
      for (int q = 0; q < KT; ++q) cp_async16(raw + i * KT + q, tab + KT * m + q);
  }
  cp_async_commit();
}

// Waits for this lane's prefetched entries and writes the records of
// centres [m0, m0 + kWarpStage) into the warp's rec (kWarpStage x kPairs u64);
// the caller synchronises the warp before reading them.
//   expanded: [a a][b_0 b_0]..[b_{d-1} ..][sg sg][c~_0 c~_0]..  (c~ = sg (mu - o))
//   direct:   [-mu_0 -mu_0]..[-mu_{d-1} ..][lw lw][sg sg]
template <int D>
__device__ __forceinline__ void stage_build(int64_t M, int64_t m0, bool expanded, const float* o, float gl2e,
                                            const float4* raw, u64* rec, int lane) {
  constexpr int RP = FastRec<D>::kPairs;
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

// Arguments of one tile: a run of 256 (32 K) consecutive sorted positions
// [p0, min(p0 + tile, p_end)) of one field's samples.  perm maps a sorted
// position to a sample index; the sample's index in x0 / xT / ckpt / traj /
// steps is perm[p] - perm_base, and those arrays hold N samples.
struct TileArgs {
  const float4* tab;
  int64_t M;
  float gamma, bias, eta;
  int T;
  const float* x0;
  const int32_t* perm;
  int64_t perm_base;
  int64_t N;
  float* xT;
  float* ckpt;
  int kck;
  float* traj;
  float* steps;
  float* s_out;   // optional: the logit s(x_{T-1}) of the last step, per sample
  float* g_out;   // optional: grad c(x_{T-1}) of the last step, per sample (d values)
};

// Bounding box of the tile's active samples (identical in every warp: each
// warp holds all of them); its centre o is the origin of the expanded form,
// which the step uses only while g' R^2 <= PDMP_EXPAND_LIMIT (R the
// half-diagonal).
template <int D, int K>
__device__ __forceinline__ bool tile_frame(const float (&x)[K][D], const bool (&act)[K], float gl2e, float (&lo)[D],
                                           float (&hi)[D], float (&o)[D]) {
#pragma unroll
  for (int j = 0; j < D; ++j) { lo[j] = INFINITY; hi[j] = -INFINITY; }
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (act[k])
#pragma unroll
      for (int j = 0; j < D; ++j) { lo[j] = fminf(lo[j], x[k][j]); hi[j] = fmaxf(hi[j], x[k][j]); }
  float R2 = 0.0f;
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
  const bool expanded = (gl2e * R2 <= PDMP_EXPAND_LIMIT) && (o[0] == o[0]);
  if (!expanded)
#pragma unroll
    for (int j = 0; j < D; ++j) o[j] = 0.0f;
  return expanded;
}

// Adds the kWarpStage staged records rec to the pair sums S, G of this lane's
// samples (U: the samples relative to the origin, packed in pairs).
template <int D, int P>
__device__ __forceinline__ void stage_accumulate(const u64* rec, bool expanded, float gl2e, const u64 (&U)[P][D],
                                                 u64 (&S)[P], u64 (&G)[P][D]) {
  constexpr int RP = FastRec<D>::kPairs;
  if (expanded) {
#pragma unroll kFastUnroll
    for (int c = 0; c < kWarpStage; ++c) {
      const ulonglong2* q = reinterpret_cast<const ulonglong2*>(rec + (size_t)c * RP);
      u64 r[RP];
#pragma unroll
      for (int j = 0; j < RP / 2; ++j) {
        ulonglong2 v = q[j];
        r[2 * j] = v.x;
        r[2 * j + 1] = v.y;
      }
      // phased: the P arguments, their ex2, then each sum over the P pairs, so
      // that consecutive packed FMAs share the record's operand (1.2 % faster
      // than pair by pair, measured; identical results)
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
      }
    }
  }
}

// The direct form about the tile centre o for tiles too wide for the expanded
// one (the batched launch's tiles): x - mu per feature in coordinates scaled
// by sqrt(g'), so that -log2 e = |x' - mu'|^2 - log2|w| takes d FMAs from the
// record's -log2|w|, and the sign rides in S's FMA:
//   S = sum sg e,  G' = sum sg e (mu - o),  so  sum w phi (x - mu) = u S - G'
// with u = x - o: 3d + 1 packed operations per sample pair and feature
// (the direct form about 0 takes 3d + 3).  Records:
//   [-c'_0 -c'_0]..[-c'_{d-1} ..][-lw -lw][sg sg][c~_0 c~_0]..
//   (c = mu - o, c' = sqrt(g') c, c~ = sg c)
template <int D>
__device__ __forceinline__ void stage_build_origin(int64_t M, int64_t m0, const float* o, float gl2e,
                                                   const float4* raw, u64* rec, int lane) {
  constexpr int RP = FastRec<D>::kPairs;
  constexpr int KT = FastRec<D>::kTab;
  const float sc = sqrtf(gl2e);
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
      for (int j = 0; j < D; ++j) mu[j] = o[j];
    }
    u64 r[RP];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const float c = mu[j] - o[j], cs = -sc * c, ct = sg * c;
      r[j] = pk(cs, cs);
      r[D + 2 + j] = pk(ct, ct);
    }
    r[D] = pk(-lw, -lw);
    r[D + 1] = pk(sg, sg);
    ulonglong2* dst = reinterpret_cast<ulonglong2*>(rec + (size_t)i * RP);
#pragma unroll
    for (int j = 0; j < RP / 2; ++j) dst[j] = make_ulonglong2(r[2 * j], r[2 * j + 1]);
  }
}

// U holds sqrt(g') (x - o); S, G' as above
template <int D, int P>
__device__ __forceinline__ void stage_accumulate_origin(const u64* rec, const u64 (&U)[P][D], u64 (&S)[P],
                                                        u64 (&G)[P][D]) {
  constexpr int RP = FastRec<D>::kPairs;
  for (int c = 0; c < kWarpStage; ++c) {
    const u64* r = rec + (size_t)c * RP;
#pragma unroll
    for (int i = 0; i < P; ++i) {
      u64 q = r[D];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const u64 dx = add2(U[i][j], r[j]);
        q = fma2(dx, dx, q);
      }
      const u64 e = ex2x2_neg(q);
      S[i] = fma2(r[D + 1], e, S[i]);
#pragma unroll
      for (int j = 0; j < D; ++j) G[i][j] = fma2(e, r[D + 2 + j], G[i][j]);
    }
  }
}

// Loads the tile's samples (sorted positions [p0, p_end)).
template <int D, int K>
__device__ __forceinline__ void tile_load(const TileArgs& a, int64_t p0, int64_t p_end, int lane, float (&x)[K][D],
                                          bool (&act)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int64_t p = p0 + k * 32 + lane;
    act[k] = p < p_end;
    const int64_t n = act[k] ? (int64_t)a.perm[p] - a.perm_base : 0;
#pragma unroll
    for (int j = 0; j < D; ++j) x[k][j] = act[k] ? a.x0[n * D + j] : 0.0f;
  }
}

// End of step t: the warps' partial sums are added in a fixed order (every
// warp computes the same totals), then the Euler update of Eq. (1); warp 0
// writes the trace, the last logit and the checkpoint.  Begins and ends with
// a block barrier (the reduction buffer aliases the stage buffers).
template <int D, int W, int K, bool TRACE>
__device__ __forceinline__ void tile_finish_step(const TileArgs& a, int t, int64_t p0, const bool (&act)[K],
                                                 float (&x)[K][D], const float (&o)[D], bool expanded,
                                                 const u64 (&S)[K / 2], const u64 (&G)[K / 2][D], float4* red,
                                                 int warp, int lane) {
  constexpr int P = K / 2;
  constexpr int kTile = 32 * K;
  const int64_t N = a.N;
  const float gamma = a.gamma, bias = a.bias, eta = a.eta;
  const int T = a.T;
  const float gl2e = gamma * kLog2e;
  __syncthreads();   // every warp has finished its centres before the reduction buffer overwrites the stages
#pragma unroll
  for (int i = 0; i < P; ++i) {
    float s0, s1, g0[D], g1[D];
    upk(S[i], s0, s1);
#pragma unroll
    for (int j = 0; j < D; ++j) upk(G[i][j], g0[j], g1[j]);
    red[warp * kTile + (2 * i) * 32 + lane] = make_float4(s0, g0[0], g0[1], D == 3 ? g0[D - 1] : 0.0f);
    red[warp * kTile + (2 * i + 1) * 32 + lane] = make_float4(s1, g1[0], g1[1], D == 3 ? g1[D - 1] : 0.0f);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float4 acc = red[k * 32 + lane];
#pragma unroll
    for (int w = 1; w < W; ++w) {
      float4 b = red[w * kTile + k * 32 + lane];
      acc.x += b.x;
      acc.y += b.y;
      acc.z += b.z;
      acc.w += b.w;
    }
    const float Ssum = acc.x, Gs[3] = {acc.y, acc.z, acc.w};
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
    const int64_t p = p0 + k * 32 + lane;
    const bool own = act[k] && warp == 0;
    const bool last_out = t == T - 1 && (a.s_out != nullptr || a.g_out != nullptr);
    const int64_t n = (own && (TRACE || last_out)) ? (int64_t)a.perm[p] - a.perm_base : 0;
    if (own && a.s_out != nullptr && t == T - 1) a.s_out[n] = shat + bias;
    if (own && a.g_out != nullptr && t == T - 1)
#pragma unroll
      for (int j = 0; j < D; ++j) a.g_out[n * D + j] = d1 * (-2.0f * gamma * ghat[j]);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const float inc = __fmul_rn(c, -2.0f * gamma * ghat[j]);
      if (TRACE && act[k] && warp == 0) {
        a.traj[((int64_t)t * N + n) * D + j] = x[k][j];
        a.steps[((int64_t)t * N + n) * D + j] = inc;
      }
      x[k][j] = __fadd_rn(x[k][j], inc);
    }
  }
  __syncthreads();   // every warp has read the reduction buffer before the next step rebuilds the stages
  if (a.ckpt != nullptr && (t + 1) % a.kck == 0 && warp == 0) {
    float* dst = a.ckpt + (int64_t)((t + 1) / a.kck - 1) * N * D;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (act[k]) {
        const int64_t n = (int64_t)a.perm[p0 + k * 32 + lane] - a.perm_base;
#pragma unroll
        for (int j = 0; j < D; ++j) dst[n * D + j] = x[k][j];
      }
  }
}

// Writes x_T (and the trace's last state) of the tile's samples.
template <int D, int K, bool TRACE>
__device__ __forceinline__ void tile_store(const TileArgs& a, int64_t p0, const bool (&act)[K],
                                           const float (&x)[K][D], int warp, int lane) {
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (act[k]) {
        const int64_t n = (int64_t)a.perm[p0 + k * 32 + lane] - a.perm_base;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          if (a.xT) a.xT[n * D + j] = x[k][j];
          if (TRACE) a.traj[((int64_t)a.T * a.N + n) * D + j] = x[k][j];
        }
      }
  }
  __syncthreads();   // the next tile of this block reuses the shared memory
}

// ORIGIN: tiles too wide for the expanded form take the direct form about the
// tile centre (stage_build_origin) instead of the one about 0.  The
// single-field launch keeps the latter: there nearly every tile is expanded,
// and the kernel compiled with both forms ran 6 % slower on such tiles.
template <int D, int W, int K, bool TRACE, bool ORIGIN = false>
__device__ __forceinline__ void fast_tile(const TileArgs& a, int64_t p0, int64_t p_end, unsigned char* smem) {
  constexpr int RP = FastRec<D>::kPairs;
  constexpr int P = K / 2;
  constexpr int KT = FastRec<D>::kTab;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // each warp owns a contiguous slice of the centres and its own stage buffers
  u64* wbuf = reinterpret_cast<u64*>(smem) + (size_t)warp * 2 * kWarpStage * RP;
  float4* red = reinterpret_cast<float4*>(smem);   // aliases the stage buffers after a step's last stage
  float4* wraw = reinterpret_cast<float4*>(smem + fast_region0_bytes<D, W, K>()) + (size_t)warp * kWarpStage * KT;
  const float4* __restrict__ tab = a.tab;
  const int64_t M = a.M;
  const float gl2e = a.gamma * kLog2e;
  const int64_t Mw = ((M + W - 1) / W + kWarpStage - 1) / kWarpStage * kWarpStage;   // slice length
  const int64_t mbase = (int64_t)warp * Mw;
  const int nstage = (int)(Mw / kWarpStage);

  float x[K][D];
  bool act[K];
  tile_load<D, K>(a, p0, p_end, lane, x, act);

  for (int t = 0; t < a.T; ++t) {
    float lo[D], hi[D], o[D];
    const bool expanded = tile_frame<D, K>(x, act, gl2e, lo, hi, o);
    u64 U[P][D], S[P], G[P][D];
    if constexpr (ORIGIN) {
      if (!expanded)
#pragma unroll
        for (int j = 0; j < D; ++j) {   // the box's centre; 0 when the box is not finite
          const float c = 0.5f * (lo[j] + hi[j]);
          o[j] = c - c == 0.0f ? c : 0.0f;
        }
      const float us = expanded ? 1.0f : sqrtf(gl2e);
#pragma unroll
      for (int i = 0; i < P; ++i) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
          U[i][j] = pk(us * (x[2 * i][j] - o[j]), us * (x[2 * i + 1][j] - o[j]));
          G[i][j] = 0ull;
        }
        S[i] = 0ull;
      }
      stage_prefetch<D>(tab, M, mbase, wraw, lane);
      if (expanded)
        stage_build<D>(M, mbase, true, o, gl2e, wraw, wbuf, lane);
      else
        stage_build_origin<D>(M, mbase, o, gl2e, wraw, wbuf, lane);
      __syncwarp();
      for (int st = 0; st < nstage; ++st) {
        if (st + 1 < nstage) stage_prefetch<D>(tab, M, mbase + (int64_t)(st + 1) * kWarpStage, wraw, lane);
        u64* cur = wbuf + (size_t)(st & 1) * kWarpStage * RP;
        u64* nxt = wbuf + (size_t)((st + 1) & 1) * kWarpStage * RP;
        const int64_t mn = mbase + (int64_t)(st + 1) * kWarpStage;
        if (expanded) {
          stage_accumulate<D, P>(cur, true, gl2e, U, S, G);
          if (st + 1 < nstage) stage_build<D>(M, mn, true, o, gl2e, wraw, nxt, lane);
        } else {
          stage_accumulate_origin<D, P>(cur, U, S, G);
          if (st + 1 < nstage) stage_build_origin<D>(M, mn, o, gl2e, wraw, nxt, lane);
        }
        __syncwarp();
      }
      if (!expanded) {
        // to the direct form's moments: sum w phi (x - mu) = u S - G'
        const u64 m1 = pk(-1.0f, -1.0f);
#pragma unroll
        for (int i = 0; i < P; ++i)
#pragma unroll
          for (int j = 0; j < D; ++j)
            G[i][j] = fma2(pk(x[2 * i][j] - o[j], x[2 * i + 1][j] - o[j]), S[i], mul2(G[i][j], m1));
      }
    } else {
#pragma unroll
      for (int i = 0; i < P; ++i) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
          U[i][j] = pk(x[2 * i][j] - o[j], x[2 * i + 1][j] - o[j]);
          G[i][j] = 0ull;
        }
        S[i] = 0ull;
      }

      stage_prefetch<D>(tab, M, mbase, wraw, lane);
      stage_build<D>(M, mbase, expanded, o, gl2e, wraw, wbuf, lane);
      __syncwarp();
      for (int st = 0; st < nstage; ++st) {
        if (st + 1 < nstage) stage_prefetch<D>(tab, M, mbase + (int64_t)(st + 1) * kWarpStage, wraw, lane);
        stage_accumulate<D, P>(wbuf + (size_t)(st & 1) * kWarpStage * RP, expanded, gl2e, U, S, G);
        if (st + 1 < nstage)
          stage_build<D>(M, mbase + (int64_t)(st + 1) * kWarpStage, expanded, o, gl2e, wraw,
                         wbuf + (size_t)((st + 1) & 1) * kWarpStage * RP, lane);
        __syncwarp();
      }
    }
    tile_finish_step<D, W, K, TRACE>(a, t, p0, act, x, o, expanded, S, G, red, warp, lane);
  }
  tile_store<D, K, TRACE>(a, p0, act, x, warp, lane);
}

}  // namespace pdmp
