// Inverse of the T-step map (Eq. 2): every Euler step x_{t+1} = x_t - eta grad c(x_t)
// is undone, last step first, by the fixed point y = z + eta grad c(y), which
// is a contraction with rate eta L < 1.  Each iteration is one pass over the
// features for the block's samples; a block stops when every sample's update
// is at most tol (relative to 1 + |y|) or after maxit iterations.
//
// Warm start.  Undoing step t, the iteration starts from z + delta, delta =
// x_{t+1} - x_{t+2} = eta grad c(x_{t+1}) the correction just found for step
// t + 1 (0 for the first step undone).  Since z = x_{t+1}, that is exactly
// the first iterate of a start from z, so each step saves one pass; the
// stopping test and the fixed point are unchanged.  The sorted-tile kernel
// extrapolates one order further once two corrections are known, starting
// from z + 2 delta_{t+1} - delta_{t+2} (the corrections change smoothly from
// step to step, by about eta Hess c delta).
//
// Two kernels: a direct one (any field; 256 samples a block in input order,
// every feature from x - mu or omega . x + b) and, for RBF fields in d = 2, 3
// with a workspace, one on the forward's sorted tiles (Hilbert order, 320
// samples a block, the expanded exponent about the tile's current centre and
// packed f32x2 sums; each fixed-point iteration is one forward sweep).
#include "fast_tile.cuh"
#include "kernels.cuh"
#include "sort.cuh"

namespace pdmp {

constexpr int kInvThreads = 128;
constexpr int kInvTile = 256;

template <int KIND, int D, int K>
__global__ void __launch_bounds__(kInvThreads)
k_morph_inverse(FieldArgs fa, const float* __restrict__ z0, int64_t N, int T, float eta, float tol, int maxit,
                float* __restrict__ y_out, int32_t* __restrict__ iters, unsigned long long* __restrict__ work) {
  constexpr int R = RecLayout<D>::kFloats;
  __shared__ __align__(16) float sm[kInvTile * R];
  const float ngl2e = -fa.gamma * kLog2e;
  const int64_t base = (int64_t)blockIdx.x * (kInvThreads * K) + threadIdx.x;
  float z[K][D], y[K][D];
  bool act[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int64_t n = base + (int64_t)k * kInvThreads;
    act[k] = n < N;
#pragma unroll
    for (int j = 0; j < D; ++j) z[k][j] = act[k] ? z0[n * D + j] : 0.0f;
  }
  int worst = 0;
  long long total = 0;
  float dz[K][D];   // the correction of the step undone before (warm start)
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int j = 0; j < D; ++j) dz[k][j] = 0.0f;
  for (int t = T - 1; t >= 0; --t) {
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int j = 0; j < D; ++j) y[k][j] = z[k][j] + dz[k][j];
    int it = 0;
    bool converged = false;
    for (; it < maxit; ++it) {
      float s[K], gs[K][D];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        s[k] = 0.0f;
#pragma unroll
        for (int j = 0; j < D; ++j) gs[k][j] = 0.0f;
      }
      for (int64_t m0 = 0; m0 < fa.M; m0 += kInvTile) {
        __syncthreads();
        stage_tile<KIND, D>(fa, m0, kInvTile, sm);
        __syncthreads();
        const int cnt = (int)min64(kInvTile, fa.M - m0);
        for (int i = 0; i < cnt; ++i) {
          float rec[R];
          load_rec<D>(sm, i, rec);
#pragma unroll
          for (int k = 0; k < K; ++k) accum_grad<KIND, D>(rec, y[k], ngl2e, s[k], gs[k]);
        }
      }
      bool moving = false;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        float d1, d2, g[D];
        sigmoid_d12(s[k] + fa.bias, d1, d2);
        finish_grad_s<KIND, D>(gs[k], fa.gamma, g);
        const float c = eta * d1;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          const float yn = fmaf(c, g[j], z[k][j]);
          if (act[k] && fabsf(yn - y[k][j]) > tol * (1.0f + fabsf(yn))) moving = true;
          y[k][j] = yn;
        }
      }
      if (!__syncthreads_or(moving)) {
        ++it;
        converged = true;
        break;
      }
    }
    if (!converged && threadIdx.x == 0) raise_flag(FLAG_NOT_CONVERGED);
    worst = it > worst ? it : worst;
    total += it;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        dz[k][j] = y[k][j] - z[k][j];
        z[k][j] = y[k][j];
      }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int64_t n = base + (int64_t)k * kInvThreads;
    if (!act[k]) continue;
#pragma unroll
    for (int j = 0; j < D; ++j) y_out[n * D + j] = z[k][j];
    if (iters) iters[n] = worst;
  }
  if (work != nullptr && threadIdx.x == 0) {
    const int64_t first = (int64_t)blockIdx.x * (kInvThreads * K);
    const int64_t cnt = min64((int64_t)kInvThreads * K, N - first);
    atomicAdd(work, (unsigned long long)total * (unsigned long long)cnt * (unsigned long long)fa.M);
  }
}

// ---------------------------------------------------------------- sorted tiles
// One tile of 320 samples (sorted positions [p0, p_end)); a.x0 holds z.  Every
// warp holds all the tile's iterates y and sums over its own slice of the
// centres, as in the forward tile; the fixed-point update and the stopping
// test are made identically in every warp.  The step's target z is kept in
// shared memory (after the forward tile's buffers), read once per iteration.
template <int D, int W, int K>
__device__ __forceinline__ void inverse_tile(const TileArgs& a, float tol, int maxit, int32_t* __restrict__ iters,
                                             unsigned long long* __restrict__ work, int64_t p0, int64_t p_end,
                                             unsigned char* smem) {
  constexpr int RP = FastRec<D>::kPairs;
  constexpr int P = K / 2;
  constexpr int KT = FastRec<D>::kTab;
  constexpr int kTile = 32 * K;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64* wbuf = reinterpret_cast<u64*>(smem) + (size_t)warp * 2 * kWarpStage * RP;
  float4* red = reinterpret_cast<float4*>(smem);   // aliases the stage buffers after an iteration's last stage
  float4* wraw = reinterpret_cast<float4*>(smem + fast_region0_bytes<D, W, K>()) + (size_t)warp * kWarpStage * KT;
  const int64_t M = a.M;
  const float gl2e = a.gamma * kLog2e;
  const float m2g = -2.0f * a.gamma;
  const int64_t Mw = ((M + W - 1) / W + kWarpStage - 1) / kWarpStage * kWarpStage;
  const int64_t mbase = (int64_t)warp * Mw;
  const int nstage = (int)(Mw / kWarpStage);

  float* zs = reinterpret_cast<float*>(smem + fast_smem_bytes<D, W, K>());   // kTile x D
  float* ds = zs + kTile * D;    // the corrections of the two steps undone before (warm start),
  float* ds2 = ds + kTile * D;   // kTile x D each
  float y[K][D];
  bool act[K];
  tile_load<D, K>(a, p0, p_end, lane, y, act);
  if (warp == 0)
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        zs[(k * 32 + lane) * D + j] = y[k][j];
        ds[(k * 32 + lane) * D + j] = 0.0f;
        ds2[(k * 32 + lane) * D + j] = 0.0f;
      }
  int worst = 0;
  long long total = 0;
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
    int it = 0;
    bool moving = true;
    while (moving && it < maxit) {
      float lo[D], hi[D], o[D];
      const bool expanded = tile_frame<D, K>(y, act, gl2e, lo, hi, o);
      u64 U[P][D], S[P], G[P][D];
#pragma unroll
      for (int i = 0; i < P; ++i) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
          U[i][j] = pk(y[2 * i][j] - o[j], y[2 * i + 1][j] - o[j]);
          G[i][j] = 0ull;
        }
        S[i] = 0ull;
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
      bool mv = false;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        float4 acc = red[k * 32 + lane];
#pragma unroll
        for (int w = 1; w < W; ++w) {
          const float4 b = red[w * kTile + k * 32 + lane];
          acc.x += b.x;
          acc.y += b.y;
          acc.z += b.z;
          acc.w += b.w;
        }
        const float Gs[3] = {acc.y, acc.z, acc.w};
        float shat, ghat[D];
        if (expanded) {
          float u[D], u2 = 0.0f;
#pragma unroll
          for (int j = 0; j < D; ++j) {
            u[j] = y[k][j] - o[j];
            u2 = fmaf(u[j], u[j], u2);
          }
          const float f = ex2_approx(-gl2e * u2);
          shat = f * acc.x;
#pragma unroll
          for (int j = 0; j < D; ++j) ghat[j] = f * fmaf(u[j], acc.x, -Gs[j]);
        } else {
          shat = acc.x;
#pragma unroll
          for (int j = 0; j < D; ++j) ghat[j] = Gs[j];
        }
        float d1, d2;
        sigmoid_d12(shat + a.bias, d1, d2);
        const float c = a.eta * d1;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          const float yn = fmaf(c, m2g * ghat[j], zs[(k * 32 + lane) * D + j]);   // z + eta sigma'(s) grad s(y)
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
    total += it;
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
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (act[k]) {
        const int64_t n = (int64_t)a.perm[p0 + k * 32 + lane] - a.perm_base;
#pragma unroll
        for (int j = 0; j < D; ++j) a.xT[n * D + j] = y[k][j];
        if (iters) iters[n] = worst;
      }
  }
  if (work != nullptr && threadIdx.x == 0) {
    const int64_t cnt = min64(kTile, p_end - p0);
    atomicAdd(work, (unsigned long long)total * (unsigned long long)cnt * (unsigned long long)M);
  }
}

template <int D, int K>
__global__ void __launch_bounds__(Shape<4, K>::kThreads, Shape<4, K>::kMinBlocks)
k_morph_inverse_fast(TileArgs a, float tol, int maxit, int32_t* __restrict__ iters,
                     unsigned long long* __restrict__ work) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t p0 = (int64_t)blockIdx.x * Shape<4, K>::kTile;
  inverse_tile<D, 4, K>(a, tol, maxit, iters, work, p0, a.N, smem);
}

// Samples per lane: 10 (320-sample tiles, 3 blocks per SM), and 4 (128-sample
// tiles, 4 blocks per SM) for launches of fewer than two waves of the larger
// ones, which then fill the GPU and stop iterating tile by tile.
template <int D, int K>
static cudaError_t launch_inverse_shape(const TileArgs& a, float tol, int maxit, int32_t* iters,
                                        unsigned long long* work, cudaStream_t st) {
  constexpr size_t smem = fast_smem_bytes<D, 4, K>() + 3 * (size_t)Shape<4, K>::kTile * D * sizeof(float);
  cudaError_t e =
      cudaFuncSetAttribute(k_morph_inverse_fast<D, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((a.N + Shape<4, K>::kTile - 1) / Shape<4, K>::kTile);
  k_morph_inverse_fast<D, K><<<blocks, Shape<4, K>::kThreads, smem, st>>>(a, tol, maxit, iters, work);
  return cudaGetLastError();
}

template <int D>
static cudaError_t launch_inverse_fast(const FieldArgs& fa, const float* z, int64_t N, int T, float eta, float tol,
                                      int maxit, float* y, int32_t* iters, unsigned long long* work, void* ws,
                                      cudaStream_t st) {
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
  const int64_t tiles = (N + FastShape::kTile - 1) / FastShape::kTile;
  if (tiles < 2 * (int64_t)FastShape::kMinBlocks * sms) return launch_inverse_shape<D, 4>(a, tol, maxit, iters, work, st);
  return launch_inverse_shape<D, FastShape::kK>(a, tol, maxit, iters, work, st);
}

// ---------------------------------------------------------------- direct
template <int KIND, int D>
static cudaError_t launch_inverse(const FieldArgs& fa, const float* z, int64_t N, int T, float eta, float tol,
                                  int maxit, float* y, int32_t* iters, unsigned long long* work, cudaStream_t st) {
  constexpr int K = 2;
  const int64_t per = (int64_t)kInvThreads * K;
  const int64_t blocks = (N + per - 1) / per;
  if (blocks == 0) return cudaSuccess;
  k_morph_inverse<KIND, D, K><<<(unsigned)blocks, kInvThreads, 0, st>>>(fa, z, N, T, eta, tol, maxit, y, iters,
                                                                        work);
  return cudaGetLastError();
}

cudaError_t morph_inverse(int kind, int d, const FieldArgs& fa, const float* z, int64_t N, int T, float eta,
                          float tol, int maxit, float* y, int32_t* iters, void* ws, unsigned long long* work,
                          cudaStream_t st) {
  if (ws != nullptr && kind == PDMP_KIND_RBF && (d == 2 || d == 3)) {
    if (d == 2) return launch_inverse_fast<2>(fa, z, N, T, eta, tol, maxit, y, iters, work, ws, st);
    return launch_inverse_fast<3>(fa, z, N, T, eta, tol, maxit, y, iters, work, ws, st);
  }
  if (ws != nullptr && kind == PDMP_KIND_RFF && d <= 7)
    return inverse_rff_mma(d, fa, z, N, T, eta, tol, maxit, y, iters, work, ws, st);
#define PDMP_CASE(KD, DD) \
  if (kind == KD && d == DD) return launch_inverse<KD, DD>(fa, z, N, T, eta, tol, maxit, y, iters, work, st);
  PDMP_CASE(PDMP_KIND_RBF, 1) PDMP_CASE(PDMP_KIND_RBF, 2) PDMP_CASE(PDMP_KIND_RBF, 3)
  PDMP_CASE(PDMP_KIND_RFF, 1) PDMP_CASE(PDMP_KIND_RFF, 2) PDMP_CASE(PDMP_KIND_RFF, 3) PDMP_CASE(PDMP_KIND_RFF, 4)
  PDMP_CASE(PDMP_KIND_RFF, 5) PDMP_CASE(PDMP_KIND_RFF, 6) PDMP_CASE(PDMP_KIND_RFF, 7) PDMP_CASE(PDMP_KIND_RFF, 8)
#undef PDMP_CASE
  return cudaErrorInvalidValue;
}

// log p_z(z) = log p_0(y) - log det J(y) at y = phi^{-1}(z) (change of
// variables through the T-step map, Sec. 3.2 "Drawing Samples"), for a uniform
// base density on the box [lo, hi]: on entry lp holds log det J(y), on exit
// log p_z; outside the box the density is 0 (-inf).
struct BoxArgs {
  float lo[8], hi[8];
  float log_vol;
  int d;
};

__global__ void k_uniform_log_density(const float* __restrict__ y, int64_t N, BoxArgs b, float* __restrict__ lp) {
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    bool inside = true;
    for (int j = 0; j < b.d; ++j) {
      const float v = y[n * b.d + j];
      inside = inside && v >= b.lo[j] && v <= b.hi[j];
    }
    lp[n] = inside ? -b.log_vol - lp[n] : -INFINITY;
  }
}

cudaError_t uniform_log_density(const float* y, int64_t N, int d, const double* lo, const double* hi, float* lp,
                                cudaStream_t st) {
  BoxArgs b{};
  double lv = 0.0;
  for (int j = 0; j < d; ++j) {
    b.lo[j] = (float)lo[j];
    b.hi[j] = (float)hi[j];
    lv += log(hi[j] - lo[j]);
  }
  b.log_vol = (float)lv;
  b.d = d;
  const int64_t blocks = min64((N + 255) / 256, 152 * 8);
  k_uniform_log_density<<<(unsigned)blocks, 256, 0, st>>>(y, N, b, lp);
  return cudaGetLastError();
}

}  // namespace pdmp
