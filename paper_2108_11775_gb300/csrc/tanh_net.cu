// The paper's own occupancy model as the morph cost (Sec. 3.1): a fully
// connected network with tanh between its hidden layers and a sigmoid output,
//   a1 = W1 x + b1, h1 = tanh(a1), a2 = W2 h1 + b2, h2 = tanh(a2),
//   s = w3 . h2 + b3,  c = sigma(s),
// and the T Euler steps of Eq. (1) through it.  The input gradient is the
// backward pass  v2 = w3 (.) (1 - h2^2),  u1 = W2^T v2,  g1 = u1 (.) (1 - h1^2),
// grad s = W1^T g1.
//
// Kernel.  A persistent block of 128 threads owns tiles of 64 samples and keeps
// their state in shared memory across all T steps.  Both dense H x H products
// of a step (W2 h1 forward, W2^T v2 backward) run as register tiles: a thread
// computes 4 samples x 8 units, with packed f32x2 FMAs over pairs of units
// (the weight pair from shared memory, the activation duplicated), reading
// per inner step one 16-byte activation vector and two 16-byte weight pairs.
// W2 is staged once per block in both layouts (unit pairs of a column for the
// forward product, of a row for the backward one); the activation tile holds
// h1 for the forward product and then v2 for the backward one, and each
// thread keeps 1 - h1^2 of its own units in registers (62.6 KB of shared
// memory a block for H = 64: three blocks per SM).  Partial sums over the
// 8 unit groups are added in a fixed order, so results are deterministic.
#include "fast_tile.cuh"
#include "kernels.cuh"

namespace pdmp {

constexpr int kNetThreads = 128;
constexpr int kNetTile = 64;     // samples per tile
constexpr int kNetSG = 16;       // sample groups of 4
constexpr int kNetUG = 8;        // unit groups of 8 (for H = 64; of 4 for H = 32)

template <int H>
struct NetSmem {
  static constexpr int kUnitsPerThread = H / kNetUG;             // 8 (H = 64) or 4 (H = 32)
  static constexpr int kPairsPerThread = kUnitsPerThread / 2;
  // offsets in floats
  static constexpr int kW2f = 0;                                  // forward pairs: [j][i/2] (W2[i][j], W2[i+1][j])
  static constexpr int kW2b = kW2f + H * H;                       // backward pairs: [i][j/2] = W2 row-major
  static constexpr int kH1 = kW2b + H * H;                        // h1 [j][sample], then v2 [i][sample]
  static constexpr int kV2 = kH1;
  static constexpr int kW1 = kH1 + H * kNetTile;                  // W1: H x d (d <= 4)
  static constexpr int kB1 = kW1 + H * 4;
  static constexpr int kB2 = kB1 + H;
  static constexpr int kW3 = kB2 + H;
  static constexpr int kX = kW3 + H;                              // x: [sample][4]
  static constexpr int kSP = kX + kNetTile * 4;                   // s partials: [ug][sample]
  static constexpr int kGP = kSP + kNetUG * kNetTile;             // grad partials: [ug][sample][4]
  static constexpr int kEnd = kGP + kNetUG * kNetTile * 4;
  static constexpr size_t bytes() { return (size_t)kEnd * sizeof(float); }
};

__device__ __forceinline__ u64 dup2(float v) { return pk(v, v); }

template <int D, int H>
__global__ void __launch_bounds__(kNetThreads, 3)
k_tanh_net_morph(TanhNetArgs net, const float* __restrict__ x0, int64_t N, int T, float eta, float* __restrict__ xT,
                 float* __restrict__ ckpt, int kck) {
  using L = NetSmem<H>;
  constexpr int UP = L::kUnitsPerThread, PP = L::kPairsPerThread;
  extern __shared__ __align__(16) float sm[];
  const int tid = threadIdx.x;
  const int sg = tid & (kNetSG - 1), ug = tid >> 4;   // 16 sample groups x 8 unit groups
  // stage the weights once
  for (int e = tid; e < H * H; e += kNetThreads) {
    const int i = e / H, j = e % H;                    // W2[i][j]
    const float w = net.W2[e];
    sm[L::kW2f + j * H + i] = w;                       // transposed: units (i, i+1) of column j adjacent
    sm[L::kW2b + e] = w;                               // row-major: (j, j+1) adjacent
  }
  for (int e = tid; e < H * D; e += kNetThreads) sm[L::kW1 + e] = net.W1[e];
  for (int e = tid; e < H; e += kNetThreads) {
    sm[L::kB1 + e] = net.b1[e];
    sm[L::kB2 + e] = net.b2[e];
    sm[L::kW3 + e] = net.w3[e];
  }
  __syncthreads();
  const int64_t ntiles = (N + kNetTile - 1) / kNetTile;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t n0 = tile * kNetTile;
    const int nt = (int)min64(kNetTile, N - n0);
    for (int e = tid; e < kNetTile * D; e += kNetThreads) {
      const int s = e / D;
      sm[L::kX + s * 4 + e % D] = s < nt ? x0[n0 * D + e] : 0.0f;
    }
    __syncthreads();
    for (int t = 0; t < T; ++t) {
      // layer 1 (h1 for this thread's 4 samples x UP units); the thread keeps
      // 1 - h1^2 of exactly the units whose backward it computes
      float t1[4][UP];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int s = sg * 4 + q;
        float xs[D];
#pragma unroll
        for (int k = 0; k < D; ++k) xs[k] = sm[L::kX + s * 4 + k];
#pragma unroll
        for (int u = 0; u < UP; ++u) {
          const int i = ug * UP + u;
          float a = sm[L::kB1 + i];
#pragma unroll
          for (int k = 0; k < D; ++k) a = fmaf(sm[L::kW1 + i * D + k], xs[k], a);
          const float h = tanhf(a);
          sm[L::kH1 + i * kNetTile + s] = h;
          t1[q][u] = fmaf(-h, h, 1.0f);
        }
      }
      __syncthreads();
      // layer 2: a2 = W2 h1 + b2 as a 4 x UP register tile
      u64 acc[4][PP];
#pragma unroll
      for (int p = 0; p < PP; ++p) {
        const u64 b = pk(sm[L::kB2 + ug * UP + 2 * p], sm[L::kB2 + ug * UP + 2 * p + 1]);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q][p] = b;
      }
#pragma unroll 4
      for (int j = 0; j < H; ++j) {
        const float4 h = *reinterpret_cast<const float4*>(sm + L::kH1 + j * kNetTile + sg * 4);
        const ulonglong2* wp = reinterpret_cast<const ulonglong2*>(sm + L::kW2f + j * H + ug * UP);
        u64 w[PP];
#pragma unroll
        for (int p = 0; p < PP / 2; ++p) {
          const ulonglong2 v2w = wp[p];
          w[2 * p] = v2w.x;
          w[2 * p + 1] = v2w.y;
        }
        const u64 hv[4] = {dup2(h.x), dup2(h.y), dup2(h.z), dup2(h.w)};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int p = 0; p < PP; ++p) acc[q][p] = fma2(w[p], hv[q], acc[q][p]);
      }
      __syncthreads();   // every thread has read h1 before v2 takes its place
      // h2 = tanh(a2); s partial over this thread's units; v2 = w3 (.) (1 - h2^2)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int s = sg * 4 + q;
        float sp = 0.0f;
#pragma unroll
        for (int p = 0; p < PP; ++p) {
          float a0, a1;
          upk(acc[q][p], a0, a1);
          const int i = ug * UP + 2 * p;
          const float h0 = tanhf(a0), h1 = tanhf(a1);
          const float w0 = sm[L::kW3 + i], w1 = sm[L::kW3 + i + 1];
          sp = fmaf(w0, h0, sp);
          sp = fmaf(w1, h1, sp);
          sm[L::kV2 + i * kNetTile + s] = w0 * fmaf(-h0, h0, 1.0f);
          sm[L::kV2 + (i + 1) * kNetTile + s] = w1 * fmaf(-h1, h1, 1.0f);
        }
        sm[L::kSP + ug * kNetTile + s] = sp;
      }
      __syncthreads();
      // backward: u1 = W2^T v2 as a 4 x UP register tile over units j
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int p = 0; p < PP; ++p) acc[q][p] = 0ull;
#pragma unroll 4
      for (int i = 0; i < H; ++i) {
        const float4 v = *reinterpret_cast<const float4*>(sm + L::kV2 + i * kNetTile + sg * 4);
        const ulonglong2* wp = reinterpret_cast<const ulonglong2*>(sm + L::kW2b + i * H + ug * UP);
        u64 w[PP];
#pragma unroll
        for (int p = 0; p < PP / 2; ++p) {
          const ulonglong2 v2w = wp[p];
          w[2 * p] = v2w.x;
          w[2 * p + 1] = v2w.y;
        }
        const u64 vv[4] = {dup2(v.x), dup2(v.y), dup2(v.z), dup2(v.w)};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int p = 0; p < PP; ++p) acc[q][p] = fma2(w[p], vv[q], acc[q][p]);
      }
      // g1 = u1 (.) (1 - h1^2); grad s partial = W1^T g1 over this thread's units
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int s = sg * 4 + q;
        float gp[D];
#pragma unroll
        for (int k = 0; k < D; ++k) gp[k] = 0.0f;
#pragma unroll
        for (int p = 0; p < PP; ++p) {
          float u0, u1;
          upk(acc[q][p], u0, u1);
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const int j = ug * UP + 2 * p + r;
            const float g = (r ? u1 : u0) * t1[q][2 * p + r];
#pragma unroll
            for (int k = 0; k < D; ++k) gp[k] = fmaf(sm[L::kW1 + j * D + k], g, gp[k]);
          }
        }
#pragma unroll
        for (int k = 0; k < D; ++k) sm[L::kGP + (ug * kNetTile + s) * 4 + k] = gp[k];
      }
      __syncthreads();
      // Euler step of Eq. (1): partial sums over the unit groups in a fixed order
      if (tid < kNetTile) {
        const int s = tid;
        float sv = net.b3, g[D];
#pragma unroll
        for (int k = 0; k < D; ++k) g[k] = 0.0f;
        for (int u = 0; u < kNetUG; ++u) {
          sv += sm[L::kSP + u * kNetTile + s];
#pragma unroll
          for (int k = 0; k < D; ++k) g[k] += sm[L::kGP + (u * kNetTile + s) * 4 + k];
        }
        float d1, d2;
        sigmoid_d12(sv, d1, d2);
        const float c = -eta * d1;
#pragma unroll
        for (int k = 0; k < D; ++k) sm[L::kX + s * 4 + k] = __fadd_rn(sm[L::kX + s * 4 + k], __fmul_rn(c, g[k]));
        if (ckpt != nullptr && (t + 1) % kck == 0 && s < nt)
#pragma unroll
          for (int k = 0; k < D; ++k) ckpt[((int64_t)((t + 1) / kck - 1) * N + n0 + s) * D + k] = sm[L::kX + s * 4 + k];
      }
      __syncthreads();
    }
    for (int e = tid; e < nt * D; e += kNetThreads) xT[n0 * D + e] = sm[L::kX + (e / D) * 4 + e % D];
    __syncthreads();
  }
}

// c, s and grad c at points: one thread per point, plain loops (for queries
// and tests; the morph kernel above is the hot path)
template <int D, int H>
__global__ void k_tanh_net_query(TanhNetArgs net, const float* __restrict__ x, int64_t N, float* __restrict__ c_out,
                                 float* __restrict__ s_out, float* __restrict__ g_out) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float xs[D], h1[H], v2[H];
#pragma unroll
  for (int k = 0; k < D; ++k) xs[k] = x[n * D + k];
  for (int i = 0; i < H; ++i) {
    float a = net.b1[i];
#pragma unroll
    for (int k = 0; k < D; ++k) a = fmaf(net.W1[i * D + k], xs[k], a);
    h1[i] = tanhf(a);
  }
  float s = net.b3;
  for (int i = 0; i < H; ++i) {
    float a = net.b2[i];
    for (int j = 0; j < H; ++j) a = fmaf(net.W2[i * H + j], h1[j], a);
    const float h = tanhf(a);
    s = fmaf(net.w3[i], h, s);
    v2[i] = net.w3[i] * fmaf(-h, h, 1.0f);
  }
  float g[D];
#pragma unroll
  for (int k = 0; k < D; ++k) g[k] = 0.0f;
  for (int j = 0; j < H; ++j) {
    float u = 0.0f;
    for (int i = 0; i < H; ++i) u = fmaf(net.W2[i * H + j], v2[i], u);
    const float gj = u * fmaf(-h1[j], h1[j], 1.0f);
#pragma unroll
    for (int k = 0; k < D; ++k) g[k] = fmaf(net.W1[j * D + k], gj, g[k]);
  }
  float d1, d2;
  sigmoid_d12(s, d1, d2);
  if (s_out) s_out[n] = s;
  if (c_out) c_out[n] = s >= 0.0f ? 1.0f / (1.0f + __expf(-s)) : __expf(s) / (1.0f + __expf(s));
  if (g_out)
#pragma unroll
    for (int k = 0; k < D; ++k) g_out[n * D + k] = d1 * g[k];
}

template <int D, int H>
static cudaError_t launch_net(const TanhNetArgs& net, const float* x0, int64_t N, int T, float eta, float* xT,
                              float* ckpt, int k, cudaStream_t st) {
  constexpr size_t smem = NetSmem<H>::bytes();
  cudaError_t e = cudaFuncSetAttribute(k_tanh_net_morph<D, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tanh_net_morph<D, H>, kNetThreads, smem);
  const int64_t ntiles = (N + kNetTile - 1) / kNetTile;
  const int64_t grid = min64(ntiles, (int64_t)sms * (per_sm > 0 ? per_sm : 1));
  k_tanh_net_morph<D, H><<<(unsigned)grid, kNetThreads, smem, st>>>(net, x0, N, T, eta, xT, ckpt, k);
  return cudaGetLastError();
}

cudaError_t tanh_net_morph(const TanhNetArgs& net, const float* x0, int64_t N, int T, float eta, float* xT,
                           float* ckpt, int k, cudaStream_t st) {
  if (net.d == 2 && net.H == 64) return launch_net<2, 64>(net, x0, N, T, eta, xT, ckpt, k, st);
  if (net.d == 3 && net.H == 64) return launch_net<3, 64>(net, x0, N, T, eta, xT, ckpt, k, st);
  if (net.d == 2 && net.H == 32) return launch_net<2, 32>(net, x0, N, T, eta, xT, ckpt, k, st);
  if (net.d == 3 && net.H == 32) return launch_net<3, 32>(net, x0, N, T, eta, xT, ckpt, k, st);
  return cudaErrorInvalidValue;
}

cudaError_t tanh_net_query(const TanhNetArgs& net, const float* x, int64_t N, float* c, float* s, float* g,
                           cudaStream_t st) {
  const unsigned blocks = (unsigned)((N + 127) / 128);
#define PDMP_NETQ(DD, HH) \
  if (net.d == DD && net.H == HH) { k_tanh_net_query<DD, HH><<<blocks, 128, 0, st>>>(net, x, N, c, s, g); return cudaGetLastError(); }
  PDMP_NETQ(2, 64) PDMP_NETQ(3, 64) PDMP_NETQ(2, 32) PDMP_NETQ(3, 32)
#undef PDMP_NETQ
  return cudaErrorInvalidValue;
}

}  // namespace pdmp
