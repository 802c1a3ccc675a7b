// The paper's own occupancy model as the morph cost (Sec. 3.1): a fully
// connected network with tanh between its hidden layers and a sigmoid output,
//   a1 = W1 x + b1, h1 = tanh(a1), a2 = W2 h1 + b2, h2 = tanh(a2),
//   s = w3 . h2 + b3,  c = sigma(s),
// and the T Euler steps of Eq. (1) through it.  The input gradient is the
// backward pass  v2 = w3 (.) (1 - h2^2),  u1 = W2^T v2,  g1 = u1 (.) (1 - h1^2),
// grad s = W1^T g1.
//
// Kernel.  A persistent block of 128 threads owns tiles of 64 samples and
// keeps their state in shared memory across all T steps; both dense H x H
// products of a step run on the tensor cores (below).  An earlier FP32 kernel
// (4-sample x 8-unit register tiles of packed f32x2 FMAs) ran at 0.58 of the
// FP32 roofline on the d = 2, H = 64 workload; this one at 0.70 (1.21x), and
// 1.53x for d = 3, H = 32.
#include "fast_tile.cuh"
#include "kernels.cuh"

namespace pdmp {

constexpr int kNetThreads = 128;
constexpr int kNetTile = 64;     // samples per tile

// Both H x H products on the tensor cores (m16n8k8 TF32,
// hi/lo splits of both operands, three MMAs each).  A warp owns 16 samples
// (one MMA row tile) and needs no other warp within a step.
//   forward   A2 = H1 W2^T + b2:  A = h1 (rows: samples, k: units j),
//             B[k = j][n = i] = W2[i][j]
//   backward  U1 = V2 W2:         A = v2 = w3 (.) (1 - h2^2), B = W2
// Lane (g, t) evaluates layer 1 exactly at its A-fragment positions (units
// 8kk + t and 8kk + t + 4 of samples g and g + 8).  The forward D fragment
// (units 8n + 2t, 8n + 2t + 1) is the backward A fragment once k slot t holds
// unit 8kk + 2t and slot t + 4 unit 8kk + 2t + 1; the backward's output
// columns are permuted (column 8n + 2t + e <-> unit 8n + t + 4e) so that u1
// arrives at the lane's own layer-1 units, where 1 - h1^2 waits in registers.
// The B fragments of both products (hi, lo) are built once per block.
template <int H>
struct NetMma {
  static constexpr int kNT = H / 8;                          // n tiles = k steps
  static constexpr int kFrag = kNT * kNT * 32;               // float4 fragments (hi, lo) per product
  static constexpr int kW1 = 2 * kFrag * 4;                  // floats: W1 (H x 4)
  static constexpr int kB1 = kW1 + H * 4;
  static constexpr int kB2 = kB1 + H;
  static constexpr int kW3 = kB2 + H;
  static constexpr int kX = kW3 + H;                         // [64 samples][4]
  static constexpr int kT1Row = H + 4;                       // padded: rows 4 banks apart
  static constexpr int kT1 = kX + kNetTile * 4;              // 1 - h1^2: [64 samples][H + 4]
  static constexpr int kEnd = kT1 + kNetTile * kT1Row;
  static constexpr size_t bytes() { return (size_t)kEnd * sizeof(float); }
};

__device__ __forceinline__ float4 tf32_pair_split(float a, float b) {
  const float ha = __uint_as_float(tf32_rna(a)), hb = __uint_as_float(tf32_rna(b));
  return make_float4(ha, hb, __uint_as_float(tf32_rna(a - ha)), __uint_as_float(tf32_rna(b - hb)));
}

template <int D, int H>
__global__ void __launch_bounds__(kNetThreads, 3)
k_tanh_net_mma(TanhNetArgs net, const float* __restrict__ x0, int64_t N, int T, float eta, float* __restrict__ xT,
               float* __restrict__ ckpt, int kck) {
  using L = NetMma<H>;
  constexpr int NT = L::kNT;
  extern __shared__ __align__(16) float sm[];
  float4* w2f = reinterpret_cast<float4*>(sm);
  float4* w2b = w2f + L::kFrag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  for (int e = tid; e < L::kFrag; e += kNetThreads) {
    const int kk = e / (NT * 32), nt = (e / 32) % NT, l = e & 31, gg = l >> 2, tt = l & 3;
    // forward: b0 = W2[8nt + gg][8kk + tt], b1 = W2[8nt + gg][8kk + tt + 4]
    const float f0 = net.W2[(8 * nt + gg) * H + 8 * kk + tt], f1 = net.W2[(8 * nt + gg) * H + 8 * kk + tt + 4];
    // backward: rows (units i) 8kk + 2tt, 8kk + 2tt + 1; column gg <-> unit j = 8nt + gg / 2 + 4 (gg % 2)
    const int j = 8 * nt + (gg >> 1) + 4 * (gg & 1);
    const float q0 = net.W2[(8 * kk + 2 * tt) * H + j], q1 = net.W2[(8 * kk + 2 * tt + 1) * H + j];
    w2f[e] = tf32_pair_split(f0, f1);
    w2b[e] = tf32_pair_split(q0, q1);
  }
  for (int e = tid; e < H * D; e += kNetThreads) sm[L::kW1 + (e / D) * 4 + e % D] = net.W1[e];
  for (int e = tid; e < H; e += kNetThreads) {
    sm[L::kB1 + e] = net.b1[e];
    sm[L::kB2 + e] = net.b2[e];
    sm[L::kW3 + e] = net.w3[e];
  }
  __syncthreads();
  const u64 c12 = pk(6144.0f, 6144.0f), nc12 = pk(-6144.0f, -6144.0f), mone = pk(-1.0f, -1.0f);
  const u64 c13 = pk(8193.0f, 8193.0f);
  const int r0 = warp * 16 + g, r1 = r0 + 8;                 // this lane's two samples in the tile
  const int64_t ntiles = (N + kNetTile - 1) / kNetTile;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t n0 = tile * kNetTile;
    const int nt_s = (int)min64(kNetTile, N - n0);
    for (int e = tid; e < kNetTile * D; e += kNetThreads) {
      const int s = e / D;
      sm[L::kX + s * 4 + e % D] = s < nt_s ? x0[n0 * D + e] : 0.0f;
    }
    __syncthreads();
    for (int step = 0; step < T; ++step) {
      float xr[2][D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        xr[0][k] = sm[L::kX + r0 * 4 + k];
        xr[1][k] = sm[L::kX + r1 * 4 + k];
      }
      // forward product, layer 1 evaluated per k step at the A-fragment positions
      // (1 - h1^2 kept in shared memory at the same positions for the backward)
      float acc[NT][4];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const float ba = sm[L::kB2 + 8 * nt + 2 * t], bb = sm[L::kB2 + 8 * nt + 2 * t + 1];
        acc[nt][0] = ba;
        acc[nt][1] = bb;
        acc[nt][2] = ba;
        acc[nt][3] = bb;
      }
#pragma unroll 1
      for (int kk = 0; kk < NT; ++kk) {
        float h[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int unit = 8 * kk + t + 4 * (q >> 1);
          float a = sm[L::kB1 + unit];
#pragma unroll
          for (int k = 0; k < D; ++k) a = fmaf(sm[L::kW1 + unit * 4 + k], xr[q & 1][k], a);
          h[q] = tanhf(a);
          sm[L::kT1 + ((q & 1) ? r1 : r0) * L::kT1Row + unit] = fmaf(-h[q], h[q], 1.0f);
        }
        // |h| <= 1: the shift split (exact TF32 head, the tail read as TF32)
        const u64 a01 = pk(h[0], h[1]), a23 = pk(h[2], h[3]);
        const u64 h01 = add2(add2(a01, c12), nc12), h23 = add2(add2(a23, c12), nc12);
        const u64 l01 = fma2(h01, mone, a01), l23 = fma2(h23, mone, a23);
        float ah[4], al[4];
        upk(h01, ah[0], ah[1]);
        upk(h23, ah[2], ah[3]);
        upk(l01, al[0], al[1]);
        upk(l23, al[2], al[3]);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          const float4 b = w2f[(kk * NT + nt) * 32 + lane];
          mma_tf32(acc[nt], __float_as_uint(al[0]), __float_as_uint(al[1]), __float_as_uint(al[2]),
                   __float_as_uint(al[3]), __float_as_uint(b.x), __float_as_uint(b.y));
          mma_tf32(acc[nt], __float_as_uint(ah[0]), __float_as_uint(ah[1]), __float_as_uint(ah[2]),
                   __float_as_uint(ah[3]), __float_as_uint(b.z), __float_as_uint(b.w));
          mma_tf32(acc[nt], __float_as_uint(ah[0]), __float_as_uint(ah[1]), __float_as_uint(ah[2]),
                   __float_as_uint(ah[3]), __float_as_uint(b.x), __float_as_uint(b.y));
        }
      }
      // h2 = tanh(a2); the logit's partial sums; v2 = w3 (.) (1 - h2^2) in place
      float sp0 = 0.0f, sp1 = 0.0f;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const float w = sm[L::kW3 + 8 * nt + 2 * t + e];
          const float ha = tanhf(acc[nt][e]), hb = tanhf(acc[nt][2 + e]);
          sp0 = fmaf(w, ha, sp0);
          sp1 = fmaf(w, hb, sp1);
          acc[nt][e] = w * fmaf(-ha, ha, 1.0f);
          acc[nt][2 + e] = w * fmaf(-hb, hb, 1.0f);
        }
      sp0 += __shfl_xor_sync(0xffffffffu, sp0, 1);
      sp0 += __shfl_xor_sync(0xffffffffu, sp0, 2);
      sp1 += __shfl_xor_sync(0xffffffffu, sp1, 1);
      sp1 += __shfl_xor_sync(0xffffffffu, sp1, 2);
      // backward product: k slot t <-> unit 8kk + 2t, slot t + 4 <-> 8kk + 2t + 1
      float u[NT][4];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) u[nt][q] = 0.0f;
#pragma unroll
      for (int kk = 0; kk < NT; ++kk) {
        // v2 has no bound: Veltkamp's split (2^13 + 1: an 11-bit head)
        const u64 a01 = pk(acc[kk][0], acc[kk][2]), a23 = pk(acc[kk][1], acc[kk][3]);
        const u64 g01 = mul2(a01, c13), g23 = mul2(a23, c13);
        const u64 h01 = fma2(fma2(a01, mone, g01), mone, g01), h23 = fma2(fma2(a23, mone, g23), mone, g23);
        const u64 l01 = fma2(h01, mone, a01), l23 = fma2(h23, mone, a23);
        float vh[4], vl[4];
        upk(h01, vh[0], vh[1]);
        upk(h23, vh[2], vh[3]);
        upk(l01, vl[0], vl[1]);
        upk(l23, vl[2], vl[3]);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          const float4 b = w2b[(kk * NT + nt) * 32 + lane];
          mma_tf32(u[nt], __float_as_uint(vl[0]), __float_as_uint(vl[1]), __float_as_uint(vl[2]),
                   __float_as_uint(vl[3]), __float_as_uint(b.x), __float_as_uint(b.y));
          mma_tf32(u[nt], __float_as_uint(vh[0]), __float_as_uint(vh[1]), __float_as_uint(vh[2]),
                   __float_as_uint(vh[3]), __float_as_uint(b.z), __float_as_uint(b.w));
          mma_tf32(u[nt], __float_as_uint(vh[0]), __float_as_uint(vh[1]), __float_as_uint(vh[2]),
                   __float_as_uint(vh[3]), __float_as_uint(b.x), __float_as_uint(b.y));
        }
      }
      // u[nt]: (r0, unit 8nt+t), (r0, 8nt+t+4), (r1, 8nt+t), (r1, 8nt+t+4); g1 = u1 (.) (1 - h1^2); grad = W1^T g1
      float gp0[D], gp1[D];
#pragma unroll
      for (int k = 0; k < D; ++k) gp0[k] = gp1[k] = 0.0f;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int unit = 8 * nt + t + 4 * e;
          const float ga = u[nt][e] * sm[L::kT1 + r0 * L::kT1Row + unit];
          const float gb = u[nt][2 + e] * sm[L::kT1 + r1 * L::kT1Row + unit];
#pragma unroll
          for (int k = 0; k < D; ++k) {
            const float w = sm[L::kW1 + unit * 4 + k];
            gp0[k] = fmaf(w, ga, gp0[k]);
            gp1[k] = fmaf(w, gb, gp1[k]);
          }
        }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        gp0[k] += __shfl_xor_sync(0xffffffffu, gp0[k], 1);
        gp0[k] += __shfl_xor_sync(0xffffffffu, gp0[k], 2);
        gp1[k] += __shfl_xor_sync(0xffffffffu, gp1[k], 1);
        gp1[k] += __shfl_xor_sync(0xffffffffu, gp1[k], 2);
      }
      // Euler step of Eq. (1) for the lane's two samples (lane t = 0 of the quad writes)
      if (t == 0) {
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int r = h2 ? r1 : r0;
          float d1, d2;
          sigmoid_d12((h2 ? sp1 : sp0) + net.b3, d1, d2);
          const float c = -eta * d1;
#pragma unroll
          for (int k = 0; k < D; ++k)
            sm[L::kX + r * 4 + k] = __fadd_rn(xr[h2][k], __fmul_rn(c, h2 ? gp1[k] : gp0[k]));
          if (ckpt != nullptr && (step + 1) % kck == 0 && r < nt_s)
#pragma unroll
            for (int k = 0; k < D; ++k)
              ckpt[((int64_t)((step + 1) / kck - 1) * N + n0 + r) * D + k] = sm[L::kX + r * 4 + k];
        }
      }
      __syncwarp();
    }
    __syncthreads();
    for (int e = tid; e < nt_s * D; e += kNetThreads) xT[n0 * D + e] = sm[L::kX + (e / D) * 4 + e % D];
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
  constexpr size_t smem = NetMma<H>::bytes();
  cudaError_t e = cudaFuncSetAttribute(k_tanh_net_mma<D, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tanh_net_mma<D, H>, kNetThreads, smem);
  const int64_t ntiles = (N + kNetTile - 1) / kNetTile;
  const int64_t grid = min64(ntiles, (int64_t)sms * (per_sm > 0 ? per_sm : 1));
  k_tanh_net_mma<D, H><<<(unsigned)grid, kNetThreads, smem, st>>>(net, x0, N, T, eta, xT, ckpt, k);
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
