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
// block in double-buffered shared-memory stages of 128 (one bulk copy each).  A
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

// Log-det records: the morph's 264 floats per k tile, then the B fragments of
// the Hessian contraction, kLdNT n tiles of 8 lower-triangle entries (hi, lo).
constexpr int kLdNT = 4;                                // 28 entries of a 7 x 7 symmetric matrix
constexpr int kLdKtFloats = kRmKtFloats + kLdNT * 128;
constexpr int kLdStageKT = 8;                           // k tiles per log-det stage
constexpr int kLdStageFloats = kLdStageKT * kLdKtFloats;
static_assert(kRmStageKT % kLdStageKT == 0, "the table is padded to whole stages of both kernels");

size_t morph_rff_mma_workspace(int64_t M) {
  return ((size_t)rm_tiles(M) * kLdKtFloats * sizeof(float) + 255) & ~size_t(255);
}

// Table of B fragments, one thread per (k tile, lane).  Features past M are
// zero (w = 0 and omega = 0: cos = 1 and sin = 0 add nothing).
// With HESS, also B[k][n] = -w omega_a omega_b for the lower-triangle entry
// n = a (a + 1) / 2 + b of feature 2t (k = t) and 2t + 1 (k = t + 4), so
// that sum_m cos(theta_m) B gives Hess s; the record stride is then kLdKtFloats.
template <int D, bool HESS>
__global__ void k_rff_mma_table(FieldArgs fa, int64_t n_kt, float* __restrict__ tab) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_kt * 32) return;
  const int64_t kt = i >> 5;
  const int lane = (int)(i & 31), g = lane >> 2, t = lane & 3;
  float* rec = tab + kt * (HESS ? kLdKtFloats : kRmKtFloats);
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
  if (HESS) {
#pragma unroll
    for (int nt = 0; nt < kLdNT; ++nt) {
      const int n = 8 * nt + g;
      int a = 0;
      while (a < 7 && (a + 1) * (a + 2) / 2 <= n) ++a;   // row of entry n
      const int b = n - a * (a + 1) / 2;
      float q2[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t mm = kt * 8 + 2 * t + h;
        q2[h] = (mm < fa.M && a < D && n < D * (D + 1) / 2)
                    ? -fa.w[mm] * fa.centres[mm * D + a] * fa.centres[mm * D + b] : 0.0f;
      }
      const float u0 = __uint_as_float(tf32_rna(q2[0])), u1 = __uint_as_float(tf32_rna(q2[1]));
      reinterpret_cast<float4*>(rec + kRmKtFloats + 128 * nt)[lane] =
          make_float4(u0, u1, __uint_as_float(tf32_rna(q2[0] - u0)), __uint_as_float(tf32_rna(q2[1] - u1)));
    }
  }
}

// Staging of the B-fragment table (TMA bulk copies).  A stage is one
// contiguous run of the table, so thread 0 moves it with a single
// cp.async.bulk (both ends 16-byte aligned, a multiple of 16 bytes long) that
// completes on the block's mbarrier; thread 0 waits for it and the block
// barrier that follows publishes the stage to every thread.  The wait is
// bounded (kRmWaitClocks, about a second): past it the block raises
// FLAG_STAGE_TIMEOUT and then issues and waits for no further copies, so the
// kernel ends (with results the flag marks as invalid).
constexpr long long kRmWaitClocks = 1ll << 31;

struct RmStageState {
  unsigned long long bar;   // the mbarrier
  uint32_t phase;           // parity of the next completion
  uint32_t failed;          // a wait gave up
};

// The block's staging state (static shared memory; only thread 0 touches it).
__device__ __forceinline__ RmStageState* rm_stage_state() {
  __shared__ RmStageState st;
  return &st;
}

// Once per kernel, before the first stage load.
__device__ __forceinline__ void rm_stage_init() {
  if (threadIdx.x == 0) {
    RmStageState* s = rm_stage_state();
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(&s->bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s->phase = 0u;
    s->failed = 0u;
  }
}

// Thread 0 starts the copy of kFloats floats from src to dst; the caller has
// passed a block barrier since dst was last read.
template <int kFloats = kRmStageFloats>
__device__ __forceinline__ void rm_stage_load(const float* __restrict__ src, float* dst) {
  static_assert((kFloats * sizeof(float)) % 16 == 0, "bulk copies move multiples of 16 bytes");
  if (threadIdx.x != 0) return;
  RmStageState* s = rm_stage_state();
  if (s->failed) return;
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&s->bar);
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  const uint32_t bytes = (uint32_t)(kFloats * sizeof(float));
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(d), "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Thread 0 waits for the copy in flight; the caller's block barrier follows.
__device__ __forceinline__ void rm_stage_wait(long long limit = kRmWaitClocks) {
  if (threadIdx.x != 0) return;
  RmStageState* s = rm_stage_state();
  if (s->failed) return;
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&s->bar);
  const uint32_t parity = s->phase;
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) {
      s->phase = parity ^ 1u;
      return;
    }
    if (clock64() - t0 > limit) {
      s->failed = 1u;
      raise_flag(FLAG_STAGE_TIMEOUT);
      return;
    }
  }
}

// tau (turns, a packed pair) -> 2 pi (tau - rint(tau)) in [-pi, pi]
__device__ __forceinline__ u64 rm_turns_to_rad(u64 tau) {
  const u64 shift = pk(12582912.0f, 12582912.0f), nshift = pk(-12582912.0f, -12582912.0f);
  const u64 mone = pk(-1.0f, -1.0f), twopi = pk(k2PiHi, k2PiHi);
  const u64 r = add2(add2(tau, shift), nshift);   // rint(tau) for |tau| < 2^22
  return mul2(fma2(r, mone, tau), twopi);         // the difference is exact
}

// A fragments (hi, lo) of the warp's 32 rows of a [32][8] state array.
__device__ __forceinline__ void rm_frags(const float* xs, int g, int t, uint32_t (&ah)[kRmRows][4],
                                         uint32_t (&al)[kRmRows][4]) {
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
}

// Veltkamp's split of a packed pair with the constant 2^13 + 1: hi keeps
// 24 - 13 = 11 significant bits (an exact TF32 value, for any magnitude),
// lo = a - hi exactly.
__device__ __forceinline__ void rm_split(u64 a, u64& hi, u64& lo) {
  const u64 c = pk(8193.0f, 8193.0f), mone = pk(-1.0f, -1.0f);
  const u64 gm = mul2(a, c);
  hi = fma2(fma2(a, mone, gm), mone, gm);   // gm - (gm - a)
  lo = fma2(hi, mone, a);
}

// One pass over all features for the warp's 32 samples.  In:
// A fragments of [x, 1] (ah, al) and, with HVP, of [v, 0] (vh, vl).  Out:
// S (packed partial logits: row g / g + 8, features 2t / 2t + 1), G (D
// fragments of grad s) and, with HVP, P (D fragments of
// sum_m cos(theta_m) (omega_m . v / 2 pi) (-w_m omega_m) = (Hess s) v / 2 pi).
// Block-wide: every warp of the block makes the same sequence of passes.
template <bool HVP>
__device__ __forceinline__ void rm_sweep(const float* __restrict__ tab, int nstage, float* sm,
                                         const uint32_t (&ah)[kRmRows][4], const uint32_t (&al)[kRmRows][4],
                                         const uint32_t (&vh)[kRmRows][4], const uint32_t (&vl)[kRmRows][4],
                                         u64 (&S)[kRmRows][2], float (&G)[kRmRows][4], float (&P)[kRmRows][4]) {
  const int lane = threadIdx.x & 31, t = lane & 3;
#pragma unroll
  for (int r = 0; r < kRmRows; ++r) {
#pragma unroll
    for (int q = 0; q < 4; ++q) G[r][q] = P[r][q] = 0.0f;
    S[r][0] = S[r][1] = 0ull;
  }
  __syncthreads();   // every warp is done with the previous pass's stages
  rm_stage_load(tab, sm);
  for (int st = 0; st < nstage; ++st) {
    rm_stage_wait();
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
        float o[4] = {0.0f, 0.0f, 0.0f, 0.0f};   // omega . v / 2 pi (the phase row meets v's zero)
        if (HVP) {
          mma_tf32(o, vl[r][0], vl[r][1], vl[r][2], vl[r][3], bth0, bth1);
          mma_tf32(o, vh[r][0], vh[r][1], vh[r][2], vh[r][3], btl0, btl1);
          mma_tf32(o, vh[r][0], vh[r][1], vh[r][2], vh[r][3], bth0, bth1);
        }
        float f0, f1, f2, f3;
        upk(rm_turns_to_rad(pk(d[0], d[1])), f0, f1);   // sample g: features 2t, 2t + 1
        upk(rm_turns_to_rad(pk(d[2], d[3])), f2, f3);   // sample g + 8
        const float c0 = cos_approx(f0), c1 = cos_approx(f1), c2 = cos_approx(f2), c3 = cos_approx(f3);
        S[r][0] = fma2(wp, pk(c0, c1), S[r][0]);
        S[r][1] = fma2(wp, pk(c2, c3), S[r][1]);
        // A of the products over features: k slot t <-> feature 2t, slot t + 4 <-> 2t + 1.
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
        mma_tf32(G[r], __float_as_uint(l[0]), __float_as_uint(l[1]), __float_as_uint(l[2]), __float_as_uint(l[3]),
                 bgh0, bgh1);
        mma_tf32(G[r], __float_as_uint(h[0]), __float_as_uint(h[1]), __float_as_uint(h[2]), __float_as_uint(h[3]),
                 bgl0, bgl1);
        mma_tf32(G[r], __float_as_uint(h[0]), __float_as_uint(h[1]), __float_as_uint(h[2]), __float_as_uint(h[3]),
                 bgh0, bgh1);
        if (HVP) {
          // cos(theta) (omega . v / 2 pi): unbounded, so Veltkamp's split
          u64 ph01, pl01, ph23, pl23;
          rm_split(mul2(pk(c0, c2), pk(o[0], o[2])), ph01, pl01);
          rm_split(mul2(pk(c1, c3), pk(o[1], o[3])), ph23, pl23);
          float ph[4], pl[4];
          upk(ph01, ph[0], ph[1]);
          upk(ph23, ph[2], ph[3]);
          upk(pl01, pl[0], pl[1]);
          upk(pl23, pl[2], pl[3]);
          mma_tf32(P[r], __float_as_uint(pl[0]), __float_as_uint(pl[1]), __float_as_uint(pl[2]),
                   __float_as_uint(pl[3]), bgh0, bgh1);
          mma_tf32(P[r], __float_as_uint(ph[0]), __float_as_uint(ph[1]), __float_as_uint(ph[2]),
                   __float_as_uint(ph[3]), bgl0, bgl1);
          mma_tf32(P[r], __float_as_uint(ph[0]), __float_as_uint(ph[1]), __float_as_uint(ph[2]),
                   __float_as_uint(ph[3]), bgh0, bgh1);
        }
      }
    }
  }
}

// the logit of rows g (hh = 0) and g + 8 (hh = 1) of row tile r: the quad's partial sums
__device__ __forceinline__ float rm_logit(const u64 (&S)[kRmRows][2], int r, int hh) {
  float sa, sb;
  upk(S[r][hh], sa, sb);
  float s = sa + sb;
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  return s;
}

// One Euler step of the warp's 32 samples held in xs ([32][8], column 7 = 1).
template <int D, bool TRACE>
__device__ __forceinline__ void rm_euler_step(const float* __restrict__ tab, int nstage, float* sm, float* xs,
                                              float bias, float eta, int64_t s0, int64_t N, int step,
                                              float* __restrict__ traj, float* __restrict__ steps) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t ah[kRmRows][4], al[kRmRows][4];
  rm_frags(xs, g, t, ah, al);
  float G[kRmRows][4], P[kRmRows][4];
  u64 S[kRmRows][2];
  rm_sweep<false>(tab, nstage, sm, ah, al, ah, al, S, G, P);
#pragma unroll
  for (int r = 0; r < kRmRows; ++r) {
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const float s = rm_logit(S, r, hh);
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
}

// rows [s0, s0 + 32) of an N x D array into xs ([32][8]; column 7 = col7)
template <int D>
__device__ __forceinline__ void rm_load_rows(const float* __restrict__ src, int64_t s0, int64_t N, float col7,
                                             float* xs) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < kRmWarpSamples * 8; i += 32) {
    const int r = i >> 3, j = i & 7;
    const int64_t n = s0 + r;
    xs[i] = j < D ? (n < N ? src[n * D + j] : 0.0f) : (j == 7 ? col7 : 0.0f);
  }
  __syncwarp();
}

template <int D>
__device__ __forceinline__ void rm_store_rows(const float* xs, int64_t s0, int64_t N, float* __restrict__ dst) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < kRmWarpSamples * D; i += 32) {
    const int r = i / D, j = i % D;
    if (s0 + r < N) dst[(s0 + r) * D + j] = xs[r * 8 + j];
  }
}

template <int D, bool TRACE>
__global__ void __launch_bounds__(kRmWarps * 32, 4)
k_morph_rff_mma(const float* __restrict__ tab, int nstage, float bias, const float* __restrict__ x0, int64_t N, int T,
                float eta, float* __restrict__ xT, float* __restrict__ ckpt, int kck, float* __restrict__ traj,
                float* __restrict__ steps) {
  static_assert(D >= 1 && D <= 7, "dimensions and the phase share the 8 k slots");
  extern __shared__ __align__(16) float sm[];
  rm_stage_init();
  const int warp = threadIdx.x >> 5;
  float* xs = sm + 2 * kRmStageFloats + warp * (kRmWarpSamples * 8);   // [32 samples][8]: x, 0 .., 1
  const int64_t s0 = (int64_t)blockIdx.x * kRmSamples + warp * kRmWarpSamples;
  rm_load_rows<D>(x0, s0, N, 1.0f, xs);
  for (int step = 0; step < T; ++step) {
    rm_euler_step<D, TRACE>(tab, nstage, sm, xs, bias, eta, s0, N, step, traj, steps);
    if (ckpt != nullptr && (step + 1) % kck == 0)
      rm_store_rows<D>(xs, s0, N, ckpt + (int64_t)((step + 1) / kck - 1) * N * D);
  }
  if (xT) rm_store_rows<D>(xs, s0, N, xT);
  if (TRACE) rm_store_rows<D>(xs, s0, N, traj + (int64_t)T * N * D);
}

// Weight-gradient pass at x (A fragments ah, al) with v = g (vh, vl), both
// before the step's update of g: adds to row[m], for every feature m, the
// block's sum over its samples of
//   cA_n cos(theta_nm) + cB_n (grad phi_m . g_n),   grad phi_m . g = -sin(theta_m) omega_m . g,
// with cA_n = -eta sigma''(s_n) (grad s_n . g_n) and cB_n = -eta sigma'(s_n)
// (per lane, for its rows g and g + 8 of each row tile).  Per k tile the
// lanes sharing t add their rows (shuffles over g), the warps' partials go
// through shared memory and are added to the block's row in a fixed order.
__device__ __forceinline__ void rm_gw_sweep(const float* __restrict__ tab, int nstage, float* sm, float* part,
                                            const uint32_t (&ah)[kRmRows][4], const uint32_t (&al)[kRmRows][4],
                                            const uint32_t (&vh)[kRmRows][4], const uint32_t (&vl)[kRmRows][4],
                                            const float (&cA)[kRmRows][2], const float (&cB)[kRmRows][2],
                                            float* __restrict__ row, int64_t M) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const float twopi = k2PiHi;
  __syncthreads();   // every warp is done with the previous pass's stages
  rm_stage_load(tab, sm);
  for (int st = 0; st < nstage; ++st) {
    rm_stage_wait();
    __syncthreads();   // stage st is visible; stage st - 1's buffer and the partials are free
    if (st + 1 < nstage)
      rm_stage_load(tab + (size_t)(st + 1) * kRmStageFloats, sm + ((st + 1) & 1) * kRmStageFloats);
    const float* sb = sm + (st & 1) * kRmStageFloats;
#pragma unroll 1
    for (int kt = 0; kt < kRmStageKT; ++kt) {
      const float4 bt = reinterpret_cast<const float4*>(sb + kt * kRmKtFloats)[lane];
      const uint32_t bth0 = __float_as_uint(bt.x), bth1 = __float_as_uint(bt.y);
      const uint32_t btl0 = __float_as_uint(bt.z), btl1 = __float_as_uint(bt.w);
      float p0 = 0.0f, p1 = 0.0f;   // features 2t and 2t + 1 of the k tile
#pragma unroll
      for (int r = 0; r < kRmRows; ++r) {
        float d[4] = {0.0f, 0.0f, 0.0f, 0.0f}, o[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        mma_tf32(d, al[r][0], al[r][1], al[r][2], al[r][3], bth0, bth1);
        mma_tf32(d, ah[r][0], ah[r][1], ah[r][2], ah[r][3], btl0, btl1);
        mma_tf32(d, ah[r][0], ah[r][1], ah[r][2], ah[r][3], bth0, bth1);
        mma_tf32(o, vl[r][0], vl[r][1], vl[r][2], vl[r][3], bth0, bth1);
        mma_tf32(o, vh[r][0], vh[r][1], vh[r][2], vh[r][3], btl0, btl1);
        mma_tf32(o, vh[r][0], vh[r][1], vh[r][2], vh[r][3], bth0, bth1);
        float f[4];
        upk(rm_turns_to_rad(pk(d[0], d[1])), f[0], f[1]);
        upk(rm_turns_to_rad(pk(d[2], d[3])), f[2], f[3]);
        // element q: row g + 8 (q >> 1), feature 2t + (q & 1)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float c = fmaf(-cB[r][q >> 1] * twopi * sin_approx(f[q]), o[q], cA[r][q >> 1] * cos_approx(f[q]));
          if (q & 1) p1 += c; else p0 += c;
        }
      }
#pragma unroll
      for (int off = 4; off < 32; off <<= 1) {
        p0 += __shfl_xor_sync(0xffffffffu, p0, off);
        p1 += __shfl_xor_sync(0xffffffffu, p1, off);
      }
      if (g == 0) {
        part[warp * (kRmStageKT * 8) + kt * 8 + 2 * t] = p0;
        part[warp * (kRmStageKT * 8) + kt * 8 + 2 * t + 1] = p1;
      }
    }
    __syncthreads();   // every warp's partials of this stage
    for (int fi = threadIdx.x; fi < kRmStageKT * 8; fi += kRmWarps * 32) {
      const int64_t m = (int64_t)st * (kRmStageKT * 8) + fi;
      if (m < M) {
        float a = part[fi];
#pragma unroll
        for (int w = 1; w < kRmWarps; ++w) a += part[w * (kRmStageKT * 8) + fi];
        row[m] += a;
      }
    }
  }
}

// VJP of the T-step map (g_t = (I - eta Hess c(x_t)) g_{t+1}), segment by
// segment from the checkpoints: the segment's states are recomputed into the
// warp's shared memory (kseg x [32][8]), then each step back is one
// Hessian-vector pass with v = g.
template <int D>
__global__ void __launch_bounds__(kRmWarps * 32, 3)
k_vjp_rff_mma(const float* __restrict__ tab, int nstage, float bias, const float* __restrict__ x0, int64_t N, int T,
              float eta, int kseg, const float* __restrict__ ckpt, const float* __restrict__ gT, float* __restrict__ g0,
              float* __restrict__ rows, int64_t M) {
  extern __shared__ __align__(16) float sm[];
  rm_stage_init();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  float* gs = sm + 2 * kRmStageFloats + warp * (kseg + 1) * (kRmWarpSamples * 8);   // [32][8], column 7 = 0
  float* seg = gs + kRmWarpSamples * 8;                                              // kseg x [32][8]
  // weight gradient (rows != nullptr): this block's row of rows_[blocks][M + 1], warp partials, bias partials
  float* part = sm + 2 * kRmStageFloats + kRmWarps * (kseg + 1) * (kRmWarpSamples * 8);   // [4][128]
  float* gbw = part + kRmWarps * kRmStageKT * 8;                                        // [4]
  float* row = rows ? rows + (int64_t)blockIdx.x * (M + 1) : nullptr;
  if (row)
    for (int64_t m = threadIdx.x; m <= M; m += blockDim.x) row[m] = 0.0f;
  float gb_acc = 0.0f;
  const int64_t s0 = (int64_t)blockIdx.x * kRmSamples + warp * kRmWarpSamples;
  rm_load_rows<D>(gT, s0, N, 0.0f, gs);
  const float twopi = k2PiHi;
  const int nseg = T / kseg;
  for (int sgi = nseg - 1; sgi >= 0; --sgi) {
    if (sgi == 0 || ckpt == nullptr) {
      rm_load_rows<D>(x0, s0, N, 1.0f, seg);
      for (int q = 0; q < sgi * kseg; ++q)
        rm_euler_step<D, false>(tab, nstage, sm, seg, bias, eta, s0, N, 0, nullptr, nullptr);
    } else {
      rm_load_rows<D>(ckpt + (int64_t)(sgi - 1) * N * D, s0, N, 1.0f, seg);
    }
    for (int i = 1; i < kseg; ++i) {
      float* dst = seg + i * (kRmWarpSamples * 8);
      for (int q = lane; q < kRmWarpSamples * 8; q += 32) dst[q] = dst[q - kRmWarpSamples * 8];
      __syncwarp();
      rm_euler_step<D, false>(tab, nstage, sm, dst, bias, eta, s0, N, 0, nullptr, nullptr);
    }
    for (int i = kseg - 1; i >= 0; --i) {
      const float* xi = seg + i * (kRmWarpSamples * 8);
      uint32_t ah[kRmRows][4], al[kRmRows][4], vh[kRmRows][4], vl[kRmRows][4];
      rm_frags(xi, g, t, ah, al);
      rm_frags(gs, g, t, vh, vl);
      float G[kRmRows][4], P[kRmRows][4];
      u64 S[kRmRows][2];
      rm_sweep<true>(tab, nstage, sm, ah, al, vh, vl, S, G, P);
      float D1[kRmRows][2], D2[kRmRows][2], GD[kRmRows][2];
#pragma unroll
      for (int r = 0; r < kRmRows; ++r)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int rw = r * 16 + g + 8 * hh;
          sigmoid_d12(rm_logit(S, r, hh) + bias, D1[r][hh], D2[r][hh]);
          // grad s . g over the quad (dimensions 2t, 2t + 1 per lane)
          float gd = fmaf(G[r][2 * hh], gs[rw * 8 + 2 * t], G[r][2 * hh + 1] * gs[rw * 8 + 2 * t + 1]);
          gd += __shfl_xor_sync(0xffffffffu, gd, 1);
          gd += __shfl_xor_sync(0xffffffffu, gd, 2);
          GD[r][hh] = gd;
        }
      if (row) {   // d/dw with g_{t+1}, before the update
        float cA[kRmRows][2], cB[kRmRows][2];
#pragma unroll
        for (int r = 0; r < kRmRows; ++r)
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            cA[r][hh] = -eta * D2[r][hh] * GD[r][hh];
            cB[r][hh] = -eta * D1[r][hh];
            if (t == 0) gb_acc += cA[r][hh];
          }
        rm_gw_sweep(tab, nstage, sm, part, ah, al, vh, vl, cA, cB, row, M);
      }
#pragma unroll
      for (int r = 0; r < kRmRows; ++r) {
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int rw = r * 16 + g + 8 * hh;
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int j = 2 * t + e;
            if (j < D) {
              const float hv = twopi * P[r][2 * hh + e];      // (Hess s) v
              const float gj = gs[rw * 8 + j];
              gs[rw * 8 + j] = gj - eta * fmaf(D1[r][hh], hv, D2[r][hh] * GD[r][hh] * G[r][2 * hh + e]);
            }
          }
        }
      }
      __syncwarp();
    }
  }
  rm_store_rows<D>(gs, s0, N, g0);
  if (row) {
    // the bias term: lanes t = 0 hold their rows' sums; warp totals, then the block's in a fixed order
#pragma unroll
    for (int off = 4; off < 32; off <<= 1) gb_acc += __shfl_xor_sync(0xffffffffu, gb_acc, off);
    if (lane == 0) gbw[warp] = gb_acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      float a = gbw[0];
      for (int w = 1; w < kRmWarps; ++w) a += gbw[w];
      row[M] = a;
    }
  }
}

template <int D>
static cudaError_t launch_rff_mma(const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* xT,
                                  float* ckpt, int k, float* traj, float* steps, void* ws, cudaStream_t st) {
  float* tab = reinterpret_cast<float*>(ws);
  const int64_t n_kt = rm_tiles(fa.M);
  k_rff_mma_table<D, false><<<(unsigned)((n_kt * 32 + 255) / 256), 256, 0, st>>>(fa, n_kt, tab);
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

// Log-det of the T-step map (Sec. 3.2, "Drawing Samples"): per step
// log det(I - eta Hess c(x_t)) with Hess c = sigma'(s) Hess s + sigma''(s)
// grad s grad s^T.  The sweep adds to the forward's two products the
// Hessian contraction Hess s = sum_m cos(theta_m) (-w_m omega_m omega_m^T) over
// the 28 lower-triangle entries (4 n tiles, TF32 with hi/lo splits; cos split
// like the sines).  At the step end each sample's s, grad s and Hess s are
// gathered through shared memory to one lane, which forms I - eta Hess c, its
// Cholesky log-det and the Euler update.
// per sample: Hess s (32 slots), s, grad s (7); 41 floats a row so that the
// lanes reading one row each (stride 41, odd) hit distinct banks
constexpr int kLdGather = 41;

__host__ __device__ constexpr size_t ld_rff_smem_bytes() {
  return (2 * (size_t)kLdStageFloats + (size_t)kRmWarps * kRmWarpSamples * (8 + kLdGather)) * sizeof(float);
}

template <int D>
__global__ void __launch_bounds__(kRmWarps * 32, 3)
k_logdet_rff_mma(const float* __restrict__ tab, int nstage, float bias, const float* __restrict__ x0, int64_t N,
                 int T, float eta, float* __restrict__ logdet, float* __restrict__ xT) {
  static_assert(D >= 1 && D <= 7, "dimensions and the phase share the 8 k slots");
  extern __shared__ __align__(16) float sm[];
  rm_stage_init();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  float* xs = sm + 2 * kLdStageFloats + warp * kRmWarpSamples * (8 + kLdGather);
  float* gat = xs + kRmWarpSamples * 8;
  const int64_t s0 = (int64_t)blockIdx.x * kRmSamples + warp * kRmWarpSamples;
  rm_load_rows<D>(x0, s0, N, 1.0f, xs);
  float total = 0.0f;
  bool bad = false;
  const u64 c12 = pk(6144.0f, 6144.0f), nc12 = pk(-6144.0f, -6144.0f), mone = pk(-1.0f, -1.0f);

  for (int step = 0; step < T; ++step) {
    uint32_t ah[kRmRows][4], al[kRmRows][4];
    rm_frags(xs, g, t, ah, al);
    float G[kRmRows][4], Q[kRmRows][kLdNT][4];
    u64 S[kRmRows][2];
#pragma unroll
    for (int r = 0; r < kRmRows; ++r) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        G[r][q] = 0.0f;
#pragma unroll
        for (int nt = 0; nt < kLdNT; ++nt) Q[r][nt][q] = 0.0f;
      }
      S[r][0] = S[r][1] = 0ull;
    }
    __syncthreads();   // every warp is done with the previous step's stages
    rm_stage_load<kLdStageFloats>(tab, sm);
    for (int st = 0; st < nstage; ++st) {
      rm_stage_wait();
      __syncthreads();
      if (st + 1 < nstage)
        rm_stage_load<kLdStageFloats>(tab + (size_t)(st + 1) * kLdStageFloats,
                                      sm + ((st + 1) & 1) * kLdStageFloats);
      const float* sb = sm + (st & 1) * kLdStageFloats;
#pragma unroll 1
      for (int kt = 0; kt < kLdStageKT; ++kt) {
        const float* rec = sb + kt * kLdKtFloats;
        const float4 bt = reinterpret_cast<const float4*>(rec)[lane];
        const float4 bg = reinterpret_cast<const float4*>(rec + 128)[lane];
        const u64 wp = reinterpret_cast<const u64*>(rec + 256)[t];
        float4 bh[kLdNT];
#pragma unroll
        for (int nt = 0; nt < kLdNT; ++nt) bh[nt] = reinterpret_cast<const float4*>(rec + kRmKtFloats + 128 * nt)[lane];
#pragma unroll
        for (int r = 0; r < kRmRows; ++r) {
          float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
          mma_tf32(d, al[r][0], al[r][1], al[r][2], al[r][3], __float_as_uint(bt.x), __float_as_uint(bt.y));
          mma_tf32(d, ah[r][0], ah[r][1], ah[r][2], ah[r][3], __float_as_uint(bt.z), __float_as_uint(bt.w));
          mma_tf32(d, ah[r][0], ah[r][1], ah[r][2], ah[r][3], __float_as_uint(bt.x), __float_as_uint(bt.y));
          float f0, f1, f2, f3;
          upk(rm_turns_to_rad(pk(d[0], d[1])), f0, f1);
          upk(rm_turns_to_rad(pk(d[2], d[3])), f2, f3);
          const float c0 = cos_approx(f0), c1 = cos_approx(f1), c2 = cos_approx(f2), c3 = cos_approx(f3);
          S[r][0] = fma2(wp, pk(c0, c1), S[r][0]);
          S[r][1] = fma2(wp, pk(c2, c3), S[r][1]);
          // sines (gradient) and cosines (Hessian), each split by the 1.5 * 2^12 shift
          const u64 s01 = pk(sin_approx(f0), sin_approx(f2)), s23 = pk(sin_approx(f1), sin_approx(f3));
          const u64 sh01 = add2(add2(s01, c12), nc12), sh23 = add2(add2(s23, c12), nc12);
          const u64 sl01 = fma2(sh01, mone, s01), sl23 = fma2(sh23, mone, s23);
          const u64 k01 = pk(c0, c2), k23 = pk(c1, c3);
          const u64 kh01 = add2(add2(k01, c12), nc12), kh23 = add2(add2(k23, c12), nc12);
          const u64 kl01 = fma2(kh01, mone, k01), kl23 = fma2(kh23, mone, k23);
          float sh[4], sl[4], kh[4], kl[4];
          upk(sh01, sh[0], sh[1]);
          upk(sh23, sh[2], sh[3]);
          upk(sl01, sl[0], sl[1]);
          upk(sl23, sl[2], sl[3]);
          upk(kh01, kh[0], kh[1]);
          upk(kh23, kh[2], kh[3]);
          upk(kl01, kl[0], kl[1]);
          upk(kl23, kl[2], kl[3]);
#define PDMP_U(x) __float_as_uint(x)
          mma_tf32(G[r], PDMP_U(sl[0]), PDMP_U(sl[1]), PDMP_U(sl[2]), PDMP_U(sl[3]), PDMP_U(bg.x), PDMP_U(bg.y));
          mma_tf32(G[r], PDMP_U(sh[0]), PDMP_U(sh[1]), PDMP_U(sh[2]), PDMP_U(sh[3]), PDMP_U(bg.z), PDMP_U(bg.w));
          mma_tf32(G[r], PDMP_U(sh[0]), PDMP_U(sh[1]), PDMP_U(sh[2]), PDMP_U(sh[3]), PDMP_U(bg.x), PDMP_U(bg.y));
#pragma unroll
          for (int nt = 0; nt < kLdNT; ++nt) {
            mma_tf32(Q[r][nt], PDMP_U(kl[0]), PDMP_U(kl[1]), PDMP_U(kl[2]), PDMP_U(kl[3]), PDMP_U(bh[nt].x),
                     PDMP_U(bh[nt].y));
            mma_tf32(Q[r][nt], PDMP_U(kh[0]), PDMP_U(kh[1]), PDMP_U(kh[2]), PDMP_U(kh[3]), PDMP_U(bh[nt].z),
                     PDMP_U(bh[nt].w));
            mma_tf32(Q[r][nt], PDMP_U(kh[0]), PDMP_U(kh[1]), PDMP_U(kh[2]), PDMP_U(kh[3]), PDMP_U(bh[nt].x),
                     PDMP_U(bh[nt].y));
          }
#undef PDMP_U
        }
      }
    }
    // gather each sample's sums: Hess s columns from the quad, s and grad s
#pragma unroll
    for (int r = 0; r < kRmRows; ++r)
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const float s = rm_logit(S, r, hh);
        float* row = gat + (r * 16 + g + 8 * hh) * kLdGather;
#pragma unroll
        for (int nt = 0; nt < kLdNT; ++nt) {
          row[nt * 8 + 2 * t] = Q[r][nt][2 * hh];
          row[nt * 8 + 2 * t + 1] = Q[r][nt][2 * hh + 1];
        }
        if (t == 0) row[32] = s;
#pragma unroll
        for (int e = 0; e < 2; ++e)
          if (2 * t + e < D) row[33 + 2 * t + e] = G[r][2 * hh + e];
      }
    __syncwarp();
    {
      // lane = sample: I - eta Hess c, its Cholesky log-det, the Euler update
      const float* row = gat + lane * kLdGather;
      float gsv[D];
#pragma unroll
      for (int j = 0; j < D; ++j) gsv[j] = row[33 + j];
      float d1, d2;
      sigmoid_d12(row[32] + bias, d1, d2);
      float A[D][D];
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
          if (b <= a) {
            const float hc = fmaf(d1, row[a * (a + 1) / 2 + b], d2 * gsv[a] * gsv[b]);
            A[a][b] = (a == b ? 1.0f : 0.0f) - eta * hc;
          } else {
            A[a][b] = 0.0f;
          }
        }
      const float ld = chol_logdet<D>(A);
      if (!(ld == ld)) bad = true;
      total += ld;
      const float c = -eta * d1;
#pragma unroll
      for (int j = 0; j < D; ++j) xs[lane * 8 + j] = __fadd_rn(xs[lane * 8 + j], __fmul_rn(c, gsv[j]));
    }
    __syncwarp();
  }
  const int64_t own = s0 + lane;
  if (own < N) {
    if (bad) raise_flag(FLAG_NONPOSITIVE_PIVOT);
    logdet[own] = bad ? nanf("") : total;
  }
  if (xT) rm_store_rows<D>(xs, s0, N, xT);
}

template <int D>
static cudaError_t launch_logdet_rff_mma(const FieldArgs& fa, const float* x0, int64_t N, int T, float eta,
                                         float* ld, float* xT, void* ws, cudaStream_t st) {
  float* tab = reinterpret_cast<float*>(ws);
  const int64_t n_kt = rm_tiles(fa.M);
  k_rff_mma_table<D, true><<<(unsigned)((n_kt * 32 + 255) / 256), 256, 0, st>>>(fa, n_kt, tab);
  constexpr size_t smem = ld_rff_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_logdet_rff_mma<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((N + kRmSamples - 1) / kRmSamples);
  k_logdet_rff_mma<D><<<blocks, kRmWarps * 32, smem, st>>>(tab, (int)(n_kt / kLdStageKT), fa.bias, x0, N, T, eta,
                                                           ld, xT);
  return cudaGetLastError();
}

cudaError_t logdet_rff_mma(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* ld,
                           float* xT, void* ws, cudaStream_t st) {
  switch (d) {
    case 1: return launch_logdet_rff_mma<1>(fa, x0, N, T, eta, ld, xT, ws, st);
    case 2: return launch_logdet_rff_mma<2>(fa, x0, N, T, eta, ld, xT, ws, st);
    case 3: return launch_logdet_rff_mma<3>(fa, x0, N, T, eta, ld, xT, ws, st);
    case 4: return launch_logdet_rff_mma<4>(fa, x0, N, T, eta, ld, xT, ws, st);
    case 5: return launch_logdet_rff_mma<5>(fa, x0, N, T, eta, ld, xT, ws, st);
    case 6: return launch_logdet_rff_mma<6>(fa, x0, N, T, eta, ld, xT, ws, st);
    case 7: return launch_logdet_rff_mma<7>(fa, x0, N, T, eta, ld, xT, ws, st);
  }
  return cudaErrorInvalidValue;
}

// Inverse of the T-step map (Eq. 2) for RFF fields, d <= 7: each Euler step,
// last first, undone by the fixed point y = z + eta grad c(y), every
// iteration one pass of the forward's tensor-core sweep.  The block iterates
// until none of its samples moves by more than tol (1 + |y|) per coordinate,
// or maxit times (the sweep synchronises the block, so the stopping test is
// block-wide).
template <int D>
__global__ void __launch_bounds__(kRmWarps * 32, 4)
k_inverse_rff_mma(const float* __restrict__ tab, int nstage, float bias, const float* __restrict__ z0, int64_t N,
                  int T, float eta, float tol, int maxit, float* __restrict__ y_out, int32_t* __restrict__ iters,
                  unsigned long long* __restrict__ work, int64_t M) {
  extern __shared__ __align__(16) float sm[];
  rm_stage_init();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  float* ys = sm + 2 * kRmStageFloats + warp * (3 * kRmWarpSamples * 8);   // iterate [32][8], column 7 = 1
  float* zs = ys + kRmWarpSamples * 8;                                     // target  [32][8]
  float* ds = zs + kRmWarpSamples * 8;                                     // last step's correction, column 7 = 0
  const int64_t s0 = (int64_t)blockIdx.x * kRmSamples + warp * kRmWarpSamples;
  rm_load_rows<D>(z0, s0, N, 1.0f, zs);
  for (int i = lane; i < kRmWarpSamples * 8; i += 32) ds[i] = 0.0f;
  int worst = 0;
  long long total = 0;
  for (int step = T - 1; step >= 0; --step) {
    // start from z + (the correction of the step undone before): the cold start's first iterate
    for (int i = lane; i < kRmWarpSamples * 8; i += 32) ys[i] = zs[i] + ds[i];
    __syncwarp();
    int it = 0;
    bool moving = true;
    while (moving && it < maxit) {
      uint32_t ah[kRmRows][4], al[kRmRows][4];
      rm_frags(ys, g, t, ah, al);
      float G[kRmRows][4], P[kRmRows][4];
      u64 S[kRmRows][2];
      rm_sweep<false>(tab, nstage, sm, ah, al, ah, al, S, G, P);
      bool mv = false;
#pragma unroll
      for (int r = 0; r < kRmRows; ++r)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const float s = rm_logit(S, r, hh);
          float d1, d2;
          sigmoid_d12(s + bias, d1, d2);
          const float c = eta * d1;
          const int row = r * 16 + g + 8 * hh;
          const bool act = s0 + row < N;
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int j = 2 * t + e;
            if (j < D) {
              const float yn = fmaf(c, G[r][2 * hh + e], zs[row * 8 + j]);   // z + eta sigma'(s) grad s(y)
              if (act && fabsf(yn - ys[row * 8 + j]) > tol * (1.0f + fabsf(yn))) mv = true;
              ys[row * 8 + j] = yn;
            }
          }
        }
      __syncwarp();
      ++it;
      moving = __syncthreads_or(mv) != 0;
    }
    if (moving && threadIdx.x == 0) raise_flag(FLAG_NOT_CONVERGED);
    worst = it > worst ? it : worst;
    total += it;
    for (int i = lane; i < kRmWarpSamples * 8; i += 32) {
      ds[i] = ys[i] - zs[i];
      zs[i] = ys[i];
    }
    __syncwarp();
  }
  rm_store_rows<D>(zs, s0, N, y_out);
  if (iters)
    for (int r = lane; r < kRmWarpSamples; r += 32)
      if (s0 + r < N) iters[s0 + r] = worst;
  if (work != nullptr && threadIdx.x == 0) {
    const int64_t first = (int64_t)blockIdx.x * kRmSamples;
    const int64_t cnt = min64((int64_t)kRmSamples, N - first);
    atomicAdd(work, (unsigned long long)total * (unsigned long long)cnt * (unsigned long long)M);
  }
}

template <int D>
static cudaError_t launch_inverse_rff_mma(const FieldArgs& fa, const float* z, int64_t N, int T, float eta, float tol,
                                          int maxit, float* y, int32_t* iters, unsigned long long* work, void* ws,
                                          cudaStream_t st) {
  float* tab = reinterpret_cast<float*>(ws);
  const int64_t n_kt = rm_tiles(fa.M);
  k_rff_mma_table<D, false><<<(unsigned)((n_kt * 32 + 255) / 256), 256, 0, st>>>(fa, n_kt, tab);
  constexpr size_t smem = (2 * (size_t)kRmStageFloats + (size_t)kRmWarps * 3 * kRmWarpSamples * 8) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_inverse_rff_mma<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((N + kRmSamples - 1) / kRmSamples);
  k_inverse_rff_mma<D><<<blocks, kRmWarps * 32, smem, st>>>(tab, (int)(n_kt / kRmStageKT), fa.bias, z, N, T, eta, tol,
                                                            maxit, y, iters, work, fa.M);
  return cudaGetLastError();
}

cudaError_t inverse_rff_mma(int d, const FieldArgs& fa, const float* z, int64_t N, int T, float eta, float tol,
                            int maxit, float* y, int32_t* iters, unsigned long long* work, void* ws, cudaStream_t st) {
  switch (d) {
    case 1: return launch_inverse_rff_mma<1>(fa, z, N, T, eta, tol, maxit, y, iters, work, ws, st);
    case 2: return launch_inverse_rff_mma<2>(fa, z, N, T, eta, tol, maxit, y, iters, work, ws, st);
    case 3: return launch_inverse_rff_mma<3>(fa, z, N, T, eta, tol, maxit, y, iters, work, ws, st);
    case 4: return launch_inverse_rff_mma<4>(fa, z, N, T, eta, tol, maxit, y, iters, work, ws, st);
    case 5: return launch_inverse_rff_mma<5>(fa, z, N, T, eta, tol, maxit, y, iters, work, ws, st);
    case 6: return launch_inverse_rff_mma<6>(fa, z, N, T, eta, tol, maxit, y, iters, work, ws, st);
    case 7: return launch_inverse_rff_mma<7>(fa, z, N, T, eta, tol, maxit, y, iters, work, ws, st);
  }
  return cudaErrorInvalidValue;
}

// Self-test of the staging wait (one block of 32 threads): the stage barrier
// is initialised and, with `with_copy`, 16 floats go from src to shared
// memory by the staging path and on to dst; thread 0 then waits with the
// given limit.  Without the copy nothing completes the barrier's phase, so
// the wait runs out and raises FLAG_STAGE_TIMEOUT (nothing is left in flight).
__global__ void k_stage_wait_selftest(const float* __restrict__ src, float* __restrict__ dst, long long limit,
                                      int with_copy) {
  __shared__ __align__(16) float buf[16];
  rm_stage_init();
  if (with_copy) rm_stage_load<16>(src, buf);
  rm_stage_wait(limit);
  __syncthreads();
  if (with_copy && threadIdx.x < 16) dst[threadIdx.x] = buf[threadIdx.x];
}

cudaError_t stage_wait_selftest(const float* src, float* dst, long long limit, int with_copy, cudaStream_t st) {
  k_stage_wait_selftest<<<1, 32, 0, st>>>(src, dst, limit, with_copy);
  return cudaGetLastError();
}

int64_t vjp_rff_mma_blocks(int64_t N) { return (N + kRmSamples - 1) / kRmSamples; }

// the tensor-core VJP keeps a segment of states in shared memory: k <= 16
size_t vjp_rff_mma_smem(int k) {
  return (2 * (size_t)kRmStageFloats + (size_t)kRmWarps * (k + 1) * kRmWarpSamples * 8 +
          (size_t)kRmWarps * kRmStageKT * 8 + kRmWarps) * sizeof(float);
}

template <int D>
static cudaError_t launch_vjp_rff_mma(const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, int k,
                                      const float* ckpt, const float* gT, float* g0, float* rows, float* gw,
                                      float* gbias, void* ws, cudaStream_t st) {
  float* tab = reinterpret_cast<float*>(ws);
  const int64_t n_kt = rm_tiles(fa.M);
  k_rff_mma_table<D, false><<<(unsigned)((n_kt * 32 + 255) / 256), 256, 0, st>>>(fa, n_kt, tab);
  const size_t smem = vjp_rff_mma_smem(k);
  cudaError_t e = cudaFuncSetAttribute(k_vjp_rff_mma<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)vjp_rff_mma_blocks(N);
  k_vjp_rff_mma<D><<<blocks, kRmWarps * 32, smem, st>>>(tab, (int)(n_kt / kRmStageKT), fa.bias, x0, N, T, eta, k,
                                                        ckpt, gT, g0, rows, fa.M);
  e = cudaGetLastError();
  if (e != cudaSuccess || rows == nullptr) return e;
  return sum_vjp_rows(rows, (int64_t)blocks, fa.M + 1, gw, gbias, st);
}

cudaError_t vjp_rff_mma(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, int k,
                        const float* ckpt, const float* gT, float* g0, float* rows, float* gw, float* gbias, void* ws,
                        cudaStream_t st) {
  switch (d) {
    case 1: return launch_vjp_rff_mma<1>(fa, x0, N, T, eta, k, ckpt, gT, g0, rows, gw, gbias, ws, st);
    case 2: return launch_vjp_rff_mma<2>(fa, x0, N, T, eta, k, ckpt, gT, g0, rows, gw, gbias, ws, st);
    case 3: return launch_vjp_rff_mma<3>(fa, x0, N, T, eta, k, ckpt, gT, g0, rows, gw, gbias, ws, st);
    case 4: return launch_vjp_rff_mma<4>(fa, x0, N, T, eta, k, ckpt, gT, g0, rows, gw, gbias, ws, st);
    case 5: return launch_vjp_rff_mma<5>(fa, x0, N, T, eta, k, ckpt, gT, g0, rows, gw, gbias, ws, st);
    case 6: return launch_vjp_rff_mma<6>(fa, x0, N, T, eta, k, ckpt, gT, g0, rows, gw, gbias, ws, st);
    case 7: return launch_vjp_rff_mma<7>(fa, x0, N, T, eta, k, ckpt, gT, g0, rows, gw, gbias, ws, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace pdmp
