// Log-det of the T-step map for 7-D random Fourier features with the Hessian
// contraction on the tensor cores.
//
// Per sample and step the log-det needs Hess s = -Q with
//   Q = sum_m c_m P_m,   c_m = w_m cos(theta_m),   P_m = omega_m omega_m^T,
// i.e. a [samples x centres] x [centres x 28] product (the 28 lower-triangle
// entries of P_m).  It runs as m16n8k8 TF32 MMAs with hi/lo splits of both
// operands (c_hi P_hi + c_hi P_lo + c_lo P_hi: relative error about 2^-21).
// The A fragment of one 16-sample x 8-centre tile holds, per lane, exactly
// the four (sample, centre) pairs the lane evaluates itself (samples g and
// g + 8, centres t and t + 4), so theta, its sin and cos, s and the gradient
// (FP32 on the CUDA cores) are computed once per pair, and the quad's lanes
// add their partial s and gradient at the step end.  The lane forms its own
// B fragments (the eight products omega_a omega_b of its two centres) from
// the staged records.  At the step end each
// sample's 28 + 7 + 1 sums are gathered through shared memory to one lane,
// which forms I - eta Hess c and its Cholesky log-det.
#include "fast_tile.cuh"
#include "kernels.cuh"

namespace pdmp {

constexpr int kLdD = 7;
constexpr int kLdQ = kLdD * (kLdD + 1) / 2;     // 28
constexpr int kLdWarps = 4;
constexpr int kLdRows = 2;                       // 16-sample row tiles per warp
static_assert(kLdRows * 16 == 32, "the step-end gather gives each lane of a warp one sample");
constexpr int kLdSamples = kLdWarps * kLdRows * 16;   // 128 per block
constexpr int kLdStage = 64;                     // centres per stage (8 k tiles)
constexpr int kLdKT = kLdStage / 8;
constexpr int kLdRawFloats = 12;                 // omega 0..6, b, w, -w, pad
constexpr int kLdGather = 40;                    // per sample: Q (32 slots), s, grad (7)

struct LdSmem {
  static constexpr int kRaw = 0;                                     // floats: kLdStage x 12
  static constexpr int kGather = kRaw + kLdStage * kLdRawFloats;     // floats: per warp 32 samples x 40
  static constexpr int kInc = kGather + kLdWarps * 32 * kLdGather;   // floats: per warp 32 samples x 8
  static constexpr int kEnd = kInc + kLdWarps * 32 * 8;
  static constexpr size_t bytes() { return (size_t)kEnd * 4; }
};

// the lower-triangle entry (a, b) of column n = a (a + 1) / 2 + b (0..27)
__device__ __forceinline__ void q_entry(int n, int& a, int& b) {
  a = (int)((sqrtf(8.0f * n + 1.0f) - 1.0f) * 0.5f);
  if ((a + 1) * (a + 2) / 2 <= n) ++a;        // guard the float root at exact squares
  if (a * (a + 1) / 2 > n) --a;
  b = n - a * (a + 1) / 2;
}

__global__ void __launch_bounds__(kLdWarps * 32, 3)
k_logdet_rff7_mma(FieldArgs fa, const float* __restrict__ x0, int64_t N, int T, float eta,
                  float* __restrict__ logdet, float* __restrict__ xT) {
  extern __shared__ __align__(16) float sm[];
  float* raw = sm + LdSmem::kRaw;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  // the lower-triangle entries (a, b) of this lane's B-fragment columns 8 nt + g
  int qa[4], qb[4];
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int n = 8 * nt + g;
    if (n < kLdQ) {
      q_entry(n, qa[nt], qb[nt]);
    } else {
      qa[nt] = 0;
      qb[nt] = -1;   // padding column: P = 0
    }
  }
  float* gat = sm + LdSmem::kGather + warp * 32 * kLdGather;
  float* incs = sm + LdSmem::kInc + warp * 32 * 8;
  const int64_t s0 = (int64_t)blockIdx.x * kLdSamples + warp * (kLdRows * 16);
  // this lane's samples: rows g and g + 8 of each row tile (shared by the quad)
  float x[kLdRows][2][kLdD];
#pragma unroll
  for (int r = 0; r < kLdRows; ++r)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t n = s0 + r * 16 + g + 8 * h;
#pragma unroll
      for (int j = 0; j < kLdD; ++j) x[r][h][j] = n < N ? x0[n * kLdD + j] : 0.0f;
    }
  // the sample whose log-det this lane owns (lanes 0..31 <-> the warp's 32 samples)
  const int64_t own = s0 + lane;
  float total = 0.0f;
  bool bad = false;
  const int nstage = (int)((fa.M + kLdStage - 1) / kLdStage);

  for (int step = 0; step < T; ++step) {
    float acc[kLdRows][4][4];
    float S[kLdRows][2], G[kLdRows][2][kLdD];
#pragma unroll
    for (int r = 0; r < kLdRows; ++r) {
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[r][nt][e] = 0.0f;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        S[r][h] = 0.0f;
#pragma unroll
        for (int j = 0; j < kLdD; ++j) G[r][h][j] = 0.0f;
      }
    }
    for (int sidx = 0; sidx < nstage; ++sidx) {
      const int64_t m0 = (int64_t)sidx * kLdStage;
      __syncthreads();   // the previous stage is fully read
      // raw records
      for (int c = threadIdx.x; c < kLdStage; c += kLdWarps * 32) {
        const int64_t m = m0 + c;
        float* rr = raw + c * kLdRawFloats;
        const bool ok = m < fa.M;
#pragma unroll
        for (int j = 0; j < kLdD; ++j) rr[j] = ok ? fa.centres[m * kLdD + j] : 0.0f;
        const float w = ok ? fa.w[m] : 0.0f;
        rr[7] = ok ? fa.phase[m] : 0.0f;
        rr[8] = w;
        rr[9] = -w;
        rr[10] = rr[11] = 0.0f;
      }
      __syncthreads();
#pragma unroll 1
      for (int kt = 0; kt < kLdKT; ++kt) {
        // this lane's two centres of the k tile: kt * 8 + t and kt * 8 + t + 4
        float om[2][kLdD], bb[2], ww[2], nw[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const float4* rr = reinterpret_cast<const float4*>(raw + (kt * 8 + t + 4 * q) * kLdRawFloats);
          const float4 v0 = rr[0], v1 = rr[1], v2 = rr[2];
          om[q][0] = v0.x; om[q][1] = v0.y; om[q][2] = v0.z; om[q][3] = v0.w;
          om[q][4] = v1.x; om[q][5] = v1.y; om[q][6] = v1.z;
          bb[q] = v1.w; ww[q] = v2.x; nw[q] = v2.y;
        }
        // B fragments: column 8 nt + g of centres t (b0) and t + 4 (b1), P = omega_a omega_b, hi and lo
        uint4 fr[4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          float p0 = 0.0f, p1 = 0.0f;
          if (qb[nt] >= 0) {
            const float* r0 = raw + (kt * 8 + t) * kLdRawFloats;
            const float* r1 = raw + (kt * 8 + t + 4) * kLdRawFloats;
            p0 = r0[qa[nt]] * r0[qb[nt]];
            p1 = r1[qa[nt]] * r1[qb[nt]];
          }
          const uint32_t p0h = tf32_rna(p0), p1h = tf32_rna(p1);
          fr[nt] = make_uint4(p0h, p1h, tf32_rna(p0 - __uint_as_float(p0h)), tf32_rna(p1 - __uint_as_float(p1h)));
        }
#pragma unroll
        for (int r = 0; r < kLdRows; ++r) {
          float c[2][2];   // [sample h][centre q]
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              float th = bb[q];
#pragma unroll
              for (int j = 0; j < kLdD; ++j) th = fmaf(om[q][j], x[r][h][j], th);
              th = reduce_2pi(th);
              const float cs = cos_approx(th), sn = sin_approx(th);
              c[h][q] = ww[q] * cs;
              const float gsn = nw[q] * sn;
              S[r][h] += c[h][q];
#pragma unroll
              for (int j = 0; j < kLdD; ++j) G[r][h][j] = fmaf(gsn, om[q][j], G[r][h][j]);
            }
          // A fragment: a0 (row g, k t), a1 (row g + 8, k t), a2 (row g, k t + 4), a3 (row g + 8, k t + 4)
          const uint32_t h0 = tf32_rna(c[0][0]), h1 = tf32_rna(c[1][0]), h2 = tf32_rna(c[0][1]), h3 = tf32_rna(c[1][1]);
          const uint32_t l0 = tf32_rna(c[0][0] - __uint_as_float(h0)), l1 = tf32_rna(c[1][0] - __uint_as_float(h1));
          const uint32_t l2 = tf32_rna(c[0][1] - __uint_as_float(h2)), l3 = tf32_rna(c[1][1] - __uint_as_float(h3));
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            mma_tf32(acc[r][nt], h0, h1, h2, h3, fr[nt].x, fr[nt].y);   // hi x hi
            mma_tf32(acc[r][nt], h0, h1, h2, h3, fr[nt].z, fr[nt].w);   // hi x lo
            mma_tf32(acc[r][nt], l0, l1, l2, l3, fr[nt].x, fr[nt].y);   // lo x hi
          }
        }
      }
    }
    // quad totals of s and the gradient
#pragma unroll
    for (int r = 0; r < kLdRows; ++r)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int o = 1; o < 4; o <<= 1) {
          S[r][h] += __shfl_xor_sync(0xffffffffu, S[r][h], o);
#pragma unroll
          for (int j = 0; j < kLdD; ++j) G[r][h][j] += __shfl_xor_sync(0xffffffffu, G[r][h][j], o);
        }
      }
    // gather each sample's sums: Q columns from the quad, s and the gradient from lane t = 0
    __syncwarp();
#pragma unroll
    for (int r = 0; r < kLdRows; ++r)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float* row = gat + (r * 16 + g + 8 * h) * kLdGather;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          row[nt * 8 + 2 * t] = acc[r][nt][2 * h];
          row[nt * 8 + 2 * t + 1] = acc[r][nt][2 * h + 1];
        }
        if (t == 0) {
          row[32] = S[r][h];
#pragma unroll
          for (int j = 0; j < kLdD; ++j) row[33 + j] = G[r][h][j];
        }
      }
    __syncwarp();
    {
      const float* row = gat + lane * kLdGather;
      const float sv = row[32];
      float gsv[kLdD];
#pragma unroll
      for (int j = 0; j < kLdD; ++j) gsv[j] = row[33 + j];
      float d1, d2;
      sigmoid_d12(sv + fa.bias, d1, d2);
      float A[kLdD][kLdD];
      int q = 0;
#pragma unroll
      for (int a = 0; a < kLdD; ++a)
#pragma unroll
        for (int b = 0; b < kLdD; ++b) {
          if (b <= a) {
            const float hs = -row[a * (a + 1) / 2 + b];          // Hess s = -Q
            const float hc = fmaf(d1, hs, d2 * gsv[a] * gsv[b]);
            A[a][b] = (a == b ? 1.0f : 0.0f) - eta * hc;
            ++q;
          } else {
            A[a][b] = 0.0f;
          }
        }
      const float ld = chol_logdet<kLdD>(A);
      if (!(ld == ld)) bad = true;
      total += ld;
      const float cinc = -eta * d1;
#pragma unroll
      for (int j = 0; j < kLdD; ++j) incs[lane * 8 + j] = __fmul_rn(cinc, gsv[j]);
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < kLdRows; ++r)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < kLdD; ++j) x[r][h][j] = __fadd_rn(x[r][h][j], incs[(r * 16 + g + 8 * h) * 8 + j]);
    __syncwarp();
  }
  if (own < N) {
    if (bad) raise_flag(FLAG_NONPOSITIVE_PIVOT);
    logdet[own] = bad ? nanf("") : total;
  }
  if (xT != nullptr && t == 0)
#pragma unroll
    for (int r = 0; r < kLdRows; ++r)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t n = s0 + r * 16 + g + 8 * h;
        if (n < N)
#pragma unroll
          for (int j = 0; j < kLdD; ++j) xT[n * kLdD + j] = x[r][h][j];
      }
}

cudaError_t logdet_rff7_mma(const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float* ld, float* xT,
                            cudaStream_t st) {
  const int64_t blocks = (N + kLdSamples - 1) / kLdSamples;
  if (blocks == 0) return cudaSuccess;
  constexpr size_t smem = LdSmem::bytes();
  cudaError_t e = cudaFuncSetAttribute(k_logdet_rff7_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_logdet_rff7_mma<<<(unsigned)blocks, kLdWarps * 32, smem, st>>>(fa, x0, N, T, eta, ld, xT);
  return cudaGetLastError();
}

}  // namespace pdmp
