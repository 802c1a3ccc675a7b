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
// form only while g' R^2 <= 8 (R the tile's half-diagonal; about 1.4e-6
// relative error per feature there) and otherwise the direct form x - mu_m
// for that step.
//
// Work split.  A block of 4 warps owns a tile of 320 samples; every warp holds
// all 320 (10 per lane, five f32x2 pairs) and sums over its own contiguous
// quarter of the centres; the four partial sums are added in a fixed order
// once per step.  Launches too small to fill the GPU take 128-sample tiles
// (below).
#include "fast_tile.cuh"
#include "kernels.cuh"
#include "sort.cuh"

namespace pdmp {

template <int D, bool TRACE, int K>
__global__ void __launch_bounds__(Shape<4, K>::kThreads, Shape<4, K>::kMinBlocks)
k_morph_rbf_fast(TileArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t p0 = (int64_t)blockIdx.x * Shape<4, K>::kTile;
  fast_tile<D, 4, K, TRACE>(a, p0, a.N, smem);
}

// Samples per lane.  A launch of fewer 320-sample tiles than fit on the GPU at
// once (3 per SM) leaves SMs idle; it takes 128-sample tiles instead (16
// warps per SM).  Measured on a 3-D field (M = 8192, T = 40): 2^16 samples
// 9.3 ms against 13.2 ms; from one wave of 320-sample tiles up (197,641 and
// 2^18 samples) the larger tiles are as fast or faster.
constexpr int kSmallK = 4;

static int fast_samples_per_lane(int64_t N) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess || sms < 1)
    sms = 152;
  const int64_t tiles = (N + FastShape::kTile - 1) / FastShape::kTile;
  return tiles < (int64_t)FastShape::kMinBlocks * sms ? kSmallK : FastShape::kK;
}

// ------------------------------------------------------------------ host
size_t rbf_fast_table_bytes(int d, int64_t M) {
  return (((size_t)M * 16 * (d == 2 ? 1 : 2)) + 255) & ~size_t(255);
}

size_t morph_rbf_fast_workspace(int d, int64_t M, int64_t N) {
  return rbf_fast_table_bytes(d, M) + sort_workspace(d, N);
}

template <int D, int K>
static cudaError_t launch_shape(const TileArgs& a, int64_t N, bool trace, cudaStream_t st) {
  constexpr size_t smem = fast_smem_bytes<D, 4, K>();
  const unsigned blocks = (unsigned)((N + Shape<4, K>::kTile - 1) / Shape<4, K>::kTile);
  cudaError_t e;
  if (trace) {
    e = cudaFuncSetAttribute(k_morph_rbf_fast<D, true, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_morph_rbf_fast<D, true, K><<<blocks, Shape<4, K>::kThreads, smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_morph_rbf_fast<D, false, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_morph_rbf_fast<D, false, K><<<blocks, Shape<4, K>::kThreads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

template <int D>
static cudaError_t launch_fast(const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* xT,
                               float* ckpt, int k, float* traj, float* steps, void* ws, cudaStream_t st,
                               float* s_out, float* g_out = nullptr) {
  float4* tab = reinterpret_cast<float4*>(ws);
  SortWs sw = sort_layout((char*)ws + rbf_fast_table_bytes(D, fa.M), D, N);
  cudaError_t e = spatial_sort(D, x0, N, sw, st);
  if (e != cudaSuccess) return e;
  if (morph_rbf_tc05_eligible(D, N))
    return morph_rbf_tc05(D, fa, x0, sw.perm, N, T, eta, xT, ckpt, k, traj, steps, s_out, g_out, st);
  k_rbf_table<D><<<(unsigned)((fa.M + 255) / 256), 256, 0, st>>>(fa.centres, fa.w, fa.M, tab);
  TileArgs a;
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
  a.ckpt = ckpt;
  a.kck = k;
  a.traj = traj;
  a.steps = steps;
  a.s_out = s_out;
  a.g_out = g_out;
  if (fast_samples_per_lane(N) == kSmallK) return launch_shape<D, kSmallK>(a, N, traj != nullptr, st);
  return launch_shape<D, FastShape::kK>(a, N, traj != nullptr, st);
}

cudaError_t morph_rbf_fast(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* xT,
                           float* ckpt, int k, float* traj, float* steps, void* ws, cudaStream_t st, float* s_out) {
  if (d == 2) return launch_fast<2>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st, s_out);
  if (d == 3) return launch_fast<3>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st, s_out);
  return cudaErrorInvalidValue;
}

cudaError_t grad_rbf_fast(int d, const FieldArgs& fa, const float* x, int64_t N, float* g, void* ws,
                          cudaStream_t st) {
  // one step with the update discarded: the per-sample gradient output only
  if (d == 2) return launch_fast<2>(fa, x, N, 1, 0.0f, nullptr, nullptr, 0, nullptr, nullptr, ws, st, nullptr, g);
  if (d == 3) return launch_fast<3>(fa, x, N, 1, 0.0f, nullptr, nullptr, 0, nullptr, nullptr, ws, st, nullptr, g);
  return cudaErrorInvalidValue;
}

}  // namespace pdmp
