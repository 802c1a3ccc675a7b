// Random-Fourier-feature morph (Eq. 1 with phi_m = cos(omega_m . x + b_m),
// d <= 7) with both contractions of a step on the tensor cores.
//
// Per tile of 16 samples x 8 features:
//   tau   = [x, 1] [Omega, b]^T / (2 pi)        theta in turns: m16n8k8 TF32
//   grad s += sin(theta) (-w Omega)             m16n8k8 TF32
// each with a hi/lo split of both operands (lo.hi + hi.lo + hi.hi, three
// MMAs; relative error about 2^-21 for theta, absolute about 2^-22 for the
// sines).  Between them, on the CUDA cores:
// tau reduced to [-1/2, 1/2] turn (round-to-integer by the 1.5 * 2^23 shift)
// and scaled to radians, sin and cos on the special-function unit, and
// s += w cos(theta) as packed f32x2 FMAs.
//
// The D fragment of the first product holds, per lane (g = lane / 4,
// t = lane % 4), tau at samples g, g + 8 and features 2t, 2t + 1.  It is
// the A fragment of the second product as it stands once feature 2t sits in
// k slot t and 2t + 1 in slot t + 4 (the table permutes B's rows to match),
// so nothing moves between lanes.  The gradient arrives as a D fragment
// (samples g, g + 8; dimensions 2t, 2t + 1): exactly the coordinates the lane
// updates, after the quad's partial logits are summed.
//
// A block of 4 warps owns 4 x 32 samples; each warp sweeps all features
// for its own 32 (two 16-row tiles), the features staged for the whole
// block in double-buffered shared-memory stages of 128 (cp.async).  A
// sample's state stays in the warp's shared memory for all T steps.
#include "fast_tile.cuh"
#include "kernels.cuh"

namespace pdmp {

// Measured on the 7-D workload (N = 2^20, M = 4096, T = 20): two row tiles
// a warp, k tiles unrolled by two and stages of 16 k tiles ran fastest among
// 1 / 2 / 4 row tiles, unroll 1 / 2 / 4 and 16 / 32 k tiles a stage.
constexpr int kRmWarps = 4;
constexpr int kRmRows = 2;                              // 16-sample row tiles per warp
constexpr int kRmUnroll = 2;
constexpr int kRmWarpSamples = kRmRows * 16;
constexpr int kRmSamples = kRmWarps * kRmWarpSamples;   // per block
constexpr int kRmStageKT = 16;                          // k tiles (8 features each) per stage
// per k tile: theta B fragments (32 lanes x float4), gradient B fragments
// (32 lanes x float4), the 8 weights
constexpr int kRmKtFloats = 128 + 128 + 8;
constexpr int kRmStageFloats = kRmStageKT * kRmKtFloats;

__host__ __device__ constexpr size_t rm_smem_bytes() {
  return (2 * (size_t)kRmStageFloats + (size_t)kRmWarps * kRmWarpSamples * 8) * sizeof(float);
}

static int64_t rm_tiles(int64_t M) {   // k tiles, padded to whole stages
  const int64_t kt = (M + 7) / 8;
  return (kt + kRmStageKT - 1) / kRmStageKT * kRmStageKT;
}

size_t morph_rff_mma_workspace(int64_t M) {
  return ((size_t)rm_tiles(M) * kRmKtFloats * sizeof(float) + 255) & ~size_t(255);
}

// Table of B fragments, one thread per (k tile, lane).  Features past M are
// zero (w = 0 and omega = 0: cos = 1 and sin = 0 add nothing).
template <int D>
__global__ void k_rff_mma_table(FieldArgs fa, int64_t n_kt, float* __restrict__ tab) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_kt * 32) return;
  const int64_t kt = i >> 5;
  const int lane = (int)(i & 31), g = lane >> 2, t = lane & 3;
  float* rec = tab + kt * kRmKtFloats;
  // theta: B[k = dimension][n = feature] = omega / 2 pi, the phase in row 7
  const int64_t m = kt * 8 + g;
  float p[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int j = t + 4 * h;
    float v = 0.0f;
    if (m < fa.M) v = j < D ? fa.centres[m * D + j] * kInv2Pi : (j == 7 ? fa.phase[m] * kInv2Pi : 0.0f);
    p[h] = v;
  }
  const float h0 = __uint_as_float(tf32_rna(p[0])), h1 = __uint_as_float(tf32_rna(p[1]));
  reinterpret_cast<float4*>(rec)[lane] = make_float4(h0, h1, __uint_as_float(tf32_rna(p[0] - h0)),
                                                     __uint_as_float(tf32_rna(p[1] - h1)));
  // gradient: B[k][n = dimension g] = -w omega of feature 2t (k = t) and 2t + 1 (k = t + 4)
  float q[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t mm = kt * 8 + 2 * t + h;
    q[h] = (mm < fa.M && g < D) ? -fa.w[mm] * fa.centres[mm * D + g] : 0.0f;
  }
  const float e0 = __uint_as_float(tf32_rna(q[0])), e1 = __uint_as_float(tf32_rna(q[1]));
  reinterpret_cast<float4*>(rec + 128)[lane] = make_float4(e0, e1, __uint_as_float(tf32_rna(q[0] - e0)),
                                                           __uint_as_float(tf32_rna(q[1] - e1)));
  if (lane < 8) rec[256 + lane] = kt * 8 + lane < fa.M ? fa.w[kt * 8 + lane] : 0.0f;
}

__device__ __forceinline__ void rm_stage_load(const float* __restrict__ src, float* dst) {
  constexpr int kChunks = kRmStageFloats / 4;
  for (int i = threadIdx.x; i < kChunks; i += kRmWarps * 32) cp_async16(dst + 4 * i, src + 4 * i);
  cp_async_commit();
}

// tau (turns, a packed pair) -> 2 pi (tau - rint(tau)) in [-pi, pi]
__device__ __forceinline__ u64 rm_turns_to_rad(u64 tau) {
  const u64 shift = pk(12582912.0f, 12582912.0f), nshift = pk(-12582912.0f, -12582912.0f);
  const u64 mone = pk(-1.0f, -1.0f), twopi = pk(k2PiHi, k2PiHi);
  const u64 r = add2(add2(tau, shift), nshift);   // rint(tau) for |tau| < 2^22
  return mul2(fma2(r, mone, tau), twopi);         // the difference is exact
}

template <int D, bool TRACE>
__global__ void __launch_bounds__(kRmWarps * 32, 4)
k_morph_rff_mma(const float* __restrict__ tab, int nstage, float bias, const float* __restrict__ x0, int64_t N, int T,
                float eta, float* __restrict__ xT, float* __restrict__ ckpt, int kck, float* __restrict__ traj,
                float* __restrict__ steps) {
  static_assert(D >= 1 && D <= 7, "dimensions and the phase share the 8 k slots");
  extern __shared__ __align__(16) float sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  float* xs = sm + 2 * kRmStageFloats + warp * (kRmWarpSamples * 8);   // [32 samples][8]: x, 0 .., 1
  const int64_t s0 = (int64_t)blockIdx.x * kRmSamples + warp * kRmWarpSamples;
  for (int i = lane; i < kRmWarpSamples * 8; i += 32) {
    const int r = i >> 3, j = i & 7;
    const int64_t n = s0 + r;
    xs[i] = j < D ? (n < N ? x0[n * D + j] : 0.0f) : (j == 7 ? 1.0f : 0.0f);
  }
  __syncwarp();

  for (int step = 0; step < T; ++step) {
    // A fragments of [x, 1], hi and lo
    uint32_t ah[kRmRows][4], al[kRmRows][4];
#pragma unroll
    for (int r = 0; r < kRmRows; ++r) {
      const float* xr = xs + r * 16 * 8;
      const float v[4] = {xr[g * 8 + t], xr[(g + 8) * 8 + t], xr[g * 8 + t + 4], xr[(g + 8) * 8 + t + 4]};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        ah[r][q] = tf32_rna(v[q]);
        al[r][q] = tf32_rna(v[q] - __uint_as_float(ah[r][q]));
      }
    }
    float G[kRmRows][4];
    u64 S[kRmRows][2];
#pragma unroll
    for (int r = 0; r < kRmRows; ++r) {
#pragma unroll
      for (int q = 0; q < 4; ++q) G[r][q] = 0.0f;
      S[r][0] = S[r][1] = 0ull;
    }
    __syncthreads();   // every warp is done with the previous step's stages
    rm_stage_load(tab, sm);
    for (int st = 0; st < nstage; ++st) {
      cp_async_wait_all();
      __syncthreads();   // stage st is visible; stage st - 1's buffer is free
      if (st + 1 < nstage)
        rm_stage_load(tab + (size_t)(st + 1) * kRmStageFloats, sm + ((st + 1) & 1) * kRmStageFloats);
      const float* sb = sm + (st & 1) * kRmStageFloats;
#pragma unroll kRmUnroll
      for (int kt = 0; kt < kRmStageKT; ++kt) {
        const float* rec = sb + kt * kRmKtFloats;
        const float4 bt = reinterpret_cast<const float4*>(rec)[lane];
        const float4 bg = reinterpret_cast<const float4*>(rec + 128)[lane];
        const u64 wp = reinterpret_cast<const u64*>(rec + 256)[t];   // w of features 2t, 2t + 1
        const uint32_t bth0 = __float_as_uint(bt.x), bth1 = __float_as_uint(bt.y);
        const uint32_t btl0 = __float_as_uint(bt.z), btl1 = __float_as_uint(bt.w);
        const uint32_t bgh0 = __float_as_uint(bg.x), bgh1 = __float_as_uint(bg.y);
        const uint32_t bgl0 = __float_as_uint(bg.z), bgl1 = __float_as_uint(bg.w);
#pragma unroll
        for (int r = 0; r < kRmRows; ++r) {
          float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
          mma_tf32(d, al[r][0], al[r][1], al[r][2], al[r][3], bth0, bth1);
          mma_tf32(d, ah[r][0], ah[r][1], ah[r][2], ah[r][3], btl0, btl1);
          mma_tf32(d, ah[r][0], ah[r][1], ah[r][2], ah[r][3], bth0, bth1);
          float f0, f1, f2, f3;
          upk(rm_turns_to_rad(pk(d[0], d[1])), f0, f1);   // sample g: features 2t, 2t + 1
          upk(rm_turns_to_rad(pk(d[2], d[3])), f2, f3);   // sample g + 8
          S[r][0] = fma2(wp, pk(cos_approx(f0), cos_approx(f1)), S[r][0]);
          S[r][1] = fma2(wp, pk(cos_approx(f2), cos_approx(f3)), S[r][1]);
          // A of the gradient product: k slot t <-> feature 2t, slot t + 4 <-> 2t + 1
          // |sin| <= 1: rounding to a multiple of 2^-11 (by adding and removing 1.5 * 2^12) leaves at
          // most 11 significant bits, an exact TF32 value; the remainder (|lo| <= 2^-12) goes in as FP32
          // bits, of which the tensor core takes the TF32 part (absolute error <= 2^-22).  All FP32-pipe
          // work: rounding conversions here would load the ALU pipe instead.
          const u64 c12 = pk(6144.0f, 6144.0f), nc12 = pk(-6144.0f, -6144.0f), mone = pk(-1.0f, -1.0f);
          const u64 a01 = pk(sin_approx(f0), sin_approx(f2)), a23 = pk(sin_approx(f1), sin_approx(f3));
          const u64 h01 = add2(add2(a01, c12), nc12), h23 = add2(add2(a23, c12), nc12);
          const u64 l01 = fma2(h01, mone, a01), l23 = fma2(h23, mone, a23);
          float h[4], l[4];
          upk(h01, h[0], h[1]);
          upk(h23, h[2], h[3]);
          upk(l01, l[0], l[1]);
          upk(l23, l[2], l[3]);
          const uint32_t h0 = __float_as_uint(h[0]), h1 = __float_as_uint(h[1]);
          const uint32_t h2 = __float_as_uint(h[2]), h3 = __float_as_uint(h[3]);
          mma_tf32(G[r], __float_as_uint(l[0]), __float_as_uint(l[1]), __float_as_uint(l[2]), __float_as_uint(l[3]),
                   bgh0, bgh1);
          mma_tf32(G[r], h0, h1, h2, h3, bgl0, bgl1);
          mma_tf32(G[r], h0, h1, h2, h3, bgh0, bgh1);
        }
      }
    }
    // logits: the quad's partial sums; then the Euler update of dimensions 2t, 2t + 1
#pragma unroll
    for (int r = 0; r < kRmRows; ++r) {
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        float sa, sb2;
        upk(S[r][hh], sa, sb2);
        float s = sa + sb2;
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        float d1, d2;
        sigmoid_d12(s + bias, d1, d2);
        const float c = -eta * d1;
        const int row = r * 16 + g + 8 * hh;
        const int64_t n = s0 + row;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int j = 2 * t + e;
          if (j < D) {
            const float inc = __fmul_rn(c, G[r][2 * hh + e]);
            if (TRACE && n < N) {
              traj[((int64_t)step * N + n) * D + j] = xs[row * 8 + j];
              steps[((int64_t)step * N + n) * D + j] = inc;
            }
            xs[row * 8 + j] = __fadd_rn(xs[row * 8 + j], inc);
          }
        }
      }
    }
    __syncwarp();
    if (ckpt != nullptr && (step + 1) % kck == 0) {
      float* dst = ckpt + (int64_t)((step + 1) / kck - 1) * N * D;
      for (int i = lane; i < kRmWarpSamples * D; i += 32) {
        const int r = i / D, j = i % D;
        if (s0 + r < N) dst[(s0 + r) * D + j] = xs[r * 8 + j];
      }
    }
  }
  for (int i = lane; i < kRmWarpSamples * D; i += 32) {
    const int r = i / D, j = i % D;
    const int64_t n = s0 + r;
    if (n < N) {
      if (xT) xT[n * D + j] = xs[r * 8 + j];
      if (TRACE) traj[((int64_t)T * N + n) * D + j] = xs[r * 8 + j];
    }
  }
}

template <int D>
static cudaError_t launch_rff_mma(const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* xT,
                                  float* ckpt, int k, float* traj, float* steps, void* ws, cudaStream_t st) {
  float* tab = reinterpret_cast<float*>(ws);
  const int64_t n_kt = rm_tiles(fa.M);
  k_rff_mma_table<D><<<(unsigned)((n_kt * 32 + 255) / 256), 256, 0, st>>>(fa, n_kt, tab);
  const int nstage = (int)(n_kt / kRmStageKT);
  constexpr size_t smem = rm_smem_bytes();
  const unsigned blocks = (unsigned)((N + kRmSamples - 1) / kRmSamples);
  cudaError_t e;
  if (traj != nullptr) {
    e = cudaFuncSetAttribute(k_morph_rff_mma<D, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_morph_rff_mma<D, true><<<blocks, kRmWarps * 32, smem, st>>>(tab, nstage, fa.bias, x0, N, T, eta, xT, ckpt, k,
                                                                  traj, steps);
  } else {
    e = cudaFuncSetAttribute(k_morph_rff_mma<D, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_morph_rff_mma<D, false><<<blocks, kRmWarps * 32, smem, st>>>(tab, nstage, fa.bias, x0, N, T, eta, xT, ckpt, k,
                                                                   nullptr, nullptr);
  }
  return cudaGetLastError();
}

cudaError_t morph_rff_mma(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* xT,
                          float* ckpt, int k, float* traj, float* steps, void* ws, cudaStream_t st) {
  switch (d) {
    case 1: return launch_rff_mma<1>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
    case 2: return launch_rff_mma<2>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
    case 3: return launch_rff_mma<3>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
    case 4: return launch_rff_mma<4>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
    case 5: return launch_rff_mma<5>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
    case 6: return launch_rff_mma<6>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
    case 7: return launch_rff_mma<7>(fa, x0, N, T, eta, xT, ckpt, k, traj, steps, ws, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace pdmp
