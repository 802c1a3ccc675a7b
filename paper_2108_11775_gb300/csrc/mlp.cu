// Learned surrogate of the T-step morph (no counterpart in the paper): an MLP
// 39 -> 128 -> 128 -> 128 -> 3 with SiLU between the linear layers, predicting
// the normalised displacement (x_T - x_0) / out_scale from a Fourier encoding
// of the normalised input u = (x_0 - lo) * in_scale - 1:
//   enc(u) = [u_0..u_2, sin(2^k pi u_0..u_2), cos(2^k pi u_0..u_2) for k = 0..5]
// (without it the displacement field, sharp near obstacle boundaries, is out
// of reach of a small SiLU network).  BF16 weights, FP32 accumulation.
//
// Inference runs on the fifth-generation tensor cores (mlp_tc05.cu).  The
// training kernels here use warp-level MMAs (mma.sync m16n8k16, BF16 x BF16 ->
// FP32) over the batch: a warp owns 16 samples, and the accumulator fragments
// of one layer, after bias + SiLU and rounding to BF16, are exactly the A
// fragments of the next layer, so activations never leave registers.  The
// 39 -> 128 input layer is FP32 on the CUDA cores.
//
// Training: forward with saved pre-activations, backward through the same
// fragment layouts (dA = dZ W on the tensor cores with transposed weight
// copies), then the weight and bias gradients of every layer as one more
// tensor-core contraction per layer, [dW | db] = dZ^T [a | 1] over the batch
// (BF16 operands staged transposed in shared memory, FP32 accumulation;
// blocks of 64 samples write partial sums that a second kernel adds in a
// fixed order), and Adam on FP32 master weights that rewrites the BF16 copies.
//
// FP32-activation mode (diagnostic): the same kernels and fragment layouts
// with every activation and backward signal fed to the tensor cores as the
// sum of three BF16 pieces (hi + mid + lo, which carry 24 bits and more of
// the FP32 value), so the products are those of FP32 activations with the
// BF16 weights.  The network's arithmetic then matches an FP64 evaluation of
// the same BF16 weights to FP32 rounding, which separates a fragment-layout
// fault from BF16 rounding.
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "mlp_common.cuh"

namespace pdmp {

constexpr int kH = 128;          // hidden width
constexpr int kFreq = 6;         // octaves of the input encoding
constexpr int kEnc = 3 + 6 * kFreq;   // encoded input width (39)
constexpr int kRowU32 = 68;      // padded smem row: 136 bf16 = 68 words (conflict-free fragment loads)
constexpr int kMlpWarps = 4;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_grad_f(float z) {
  const float s = 1.0f / (1.0f + __expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

// Device copy of the network (all pointers device; bf16 as raw uint16).
struct MlpArgs {
  const uint16_t* W1;   // 128 x 39
  const uint16_t* W2;   // 128 x 128  [out][in]
  const uint16_t* W3;   // 128 x 128
  const uint16_t* W4;   // 3 x 128
  const uint16_t* W2t;  // 128 x 128  [in][out] (backward)
  const uint16_t* W3t;  // 128 x 128
  const float *b1, *b2, *b3, *b4;
  float lo[3], in_scale[3], out_scale[3];
};

// shared-memory image of the weights
struct MlpSmem {
  uint32_t W2[kH * kRowU32];
  uint32_t W3[kH * kRowU32];
  uint32_t W4[8 * kRowU32];      // rows 3..7 zero (one n8 tile)
  float W1[kH * kEnc];
  float b1[kH], b2[kH], b3[kH], b4[4];
};

__device__ void load_weights(const MlpArgs& a, MlpSmem* s, bool transposed) {
  const uint16_t* w2 = transposed ? a.W2t : a.W2;
  const uint16_t* w3 = transposed ? a.W3t : a.W3;
  for (int i = threadIdx.x; i < kH * (kH / 2); i += blockDim.x) {
    const int r = i / (kH / 2), c = i % (kH / 2);
    const uint32_t* s2 = reinterpret_cast<const uint32_t*>(w2);
    const uint32_t* s3 = reinterpret_cast<const uint32_t*>(w3);
    s->W2[r * kRowU32 + c] = s2[i];
    s->W3[r * kRowU32 + c] = s3[i];
  }
  for (int i = threadIdx.x; i < 8 * (kH / 2); i += blockDim.x) {
    const int r = i / (kH / 2), c = i % (kH / 2);
    s->W4[r * kRowU32 + c] = r < 3 ? reinterpret_cast<const uint32_t*>(a.W4)[r * (kH / 2) + c] : 0u;
  }
  for (int i = threadIdx.x; i < kH * kEnc; i += blockDim.x) s->W1[i] = __uint_as_float((uint32_t)a.W1[i] << 16);
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    s->b1[i] = a.b1[i];
    s->b2[i] = a.b2[i];
    s->b3[i] = a.b3[i];
  }
  if (threadIdx.x < 4) s->b4[threadIdx.x] = threadIdx.x < 3 ? a.b4[threadIdx.x] : 0.0f;
}

// piece p (0, 1, 2) of the three-way BF16 split of x: x = hi + mid + lo up to
// 2^-27 |x| (piece 2 is rounded to BF16 when packed)
__device__ __forceinline__ float bf16_piece(float x, int p) {
  const float h = __bfloat162float(__float2bfloat16_rn(x));
  if (p == 0) return h;
  const float r = x - h;
  const float m = __bfloat162float(__float2bfloat16_rn(r));
  return p == 1 ? m : r - m;
}

// bias + SiLU in place on acc[16][4] (C fragments over 128 columns); Z
// (optional, B x 128 rows) receives the pre-activations of rows r0, r1 (< B)
__device__ __forceinline__ void bias_silu(float (&acc)[16][4], const float* bias, int t, float* Z = nullptr,
                                          int64_t r0 = 0, int64_t r1 = 0, int64_t B = 0) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int c = 8 * j + 2 * t;
    float v0 = acc[j][0] + bias[c], v1 = acc[j][1] + bias[c + 1];
    float v2 = acc[j][2] + bias[c], v3 = acc[j][3] + bias[c + 1];
    if (Z) {
      if (r0 < B) *reinterpret_cast<float2*>(Z + r0 * kH + c) = make_float2(v0, v1);
      if (r1 < B) *reinterpret_cast<float2*>(Z + r1 * kH + c) = make_float2(v2, v3);
    }
    acc[j][0] = silu_f(v0);
    acc[j][1] = silu_f(v1);
    acc[j][2] = silu_f(v2);
    acc[j][3] = silu_f(v3);
  }
}

// C fragments over 128 columns -> A fragments [8][4] of BF16 piece p: the
// accumulator of column tiles 2kk, 2kk + 1 is the A fragment of k tile kk
__device__ __forceinline__ void to_afrag(const float (&v)[16][4], int p, uint32_t (&af)[8][4]) {
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    af[kk][0] = pack_bf16(bf16_piece(v[2 * kk][0], p), bf16_piece(v[2 * kk][1], p));
    af[kk][1] = pack_bf16(bf16_piece(v[2 * kk][2], p), bf16_piece(v[2 * kk][3], p));
    af[kk][2] = pack_bf16(bf16_piece(v[2 * kk + 1][0], p), bf16_piece(v[2 * kk + 1][1], p));
    af[kk][3] = pack_bf16(bf16_piece(v[2 * kk + 1][2], p), bf16_piece(v[2 * kk + 1][3], p));
  }
}

// acc += A (16 x 128) * W^T for a 128 x 128 smem weight image W[n][k]
__device__ __forceinline__ void gemm_128_acc(const uint32_t (&af)[8][4], const uint32_t* W, int g, int t,
                                             float (&acc)[16][4]) {
#pragma unroll
  for (int kk = 0; kk < 8; ++kk)
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint32_t* row = W + (8 * j + g) * kRowU32 + 8 * kk;
      mma16816(acc[j], af[kk], row[t], row[4 + t]);
    }
}

// v <- v W^T (v: a warp's 16 rows of activations in C-fragment layout).
// EXACT: v enters as three BF16 pieces (FP32-activation mode).
template <bool EXACT>
__device__ __forceinline__ void dense_128(float (&v)[16][4], const uint32_t* W, int g, int t) {
  if constexpr (EXACT) {
    float h[16][4];
#pragma unroll
    for (int j = 0; j < 16; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        h[j][q] = v[j][q];
        v[j][q] = 0.0f;
      }
#pragma unroll 1
    for (int p = 0; p < 3; ++p) {
      uint32_t af[8][4];
      to_afrag(h, p, af);
      gemm_128_acc(af, W, g, t, v);
    }
  } else {
    uint32_t af[8][4];
    to_afrag(v, 0, af);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j][0] = v[j][1] = v[j][2] = v[j][3] = 0.0f;
    gemm_128_acc(af, W, g, t, v);
  }
}

// o (one n8 tile: columns 2t, 2t + 1 of rows g, g + 8) = v W4^T
template <bool EXACT>
__device__ __forceinline__ void dense_out(const float (&v)[16][4], const uint32_t* W4, int g, int t, float (&o)[4]) {
  o[0] = o[1] = o[2] = o[3] = 0.0f;
#pragma unroll 1
  for (int p = 0; p < (EXACT ? 3 : 1); ++p) {
    uint32_t af[8][4];
    to_afrag(v, p, af);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const uint32_t* row = W4 + g * kRowU32 + 8 * kk;
      mma16816(o, af[kk], row[t], row[4 + t]);
    }
  }
}

// the Fourier encoding of x's normalised coordinates (mlp_common.cuh); the
// training kernels take sin / cos on the special-function unit, the
// FP32-activation mode CUDA's sinf / cosf
template <bool EXACT>
__device__ __forceinline__ void encode(const MlpArgs& a, const float* x, float* e) {
  MlpEncIn in;
  mlp_enc_prepare(x, a.lo, a.in_scale, in);
#pragma unroll
  for (int f = 0; f < kEnc; ++f) e[f] = mlp_enc_feature<EXACT>(f, in);
}

// input layer (FP32): acc[j] = W1 enc for rows g, g + 8 of the warp's tile
__device__ __forceinline__ void input_layer(const MlpSmem* s, const float* e0, const float* e1, int t,
                                            float (&acc)[16][4]) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int c = 8 * j + 2 * t;
    const float* wa = s->W1 + c * kEnc;
    const float* wb = s->W1 + (c + 1) * kEnc;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
#pragma unroll
    for (int i = 0; i < kEnc; ++i) {
      a0 = fmaf(wa[i], e0[i], a0);
      a1 = fmaf(wb[i], e0[i], a1);
      a2 = fmaf(wa[i], e1[i], a2);
      a3 = fmaf(wb[i], e1[i], a3);
    }
    acc[j][0] = a0;
    acc[j][1] = a1;
    acc[j][2] = a2;
    acc[j][3] = a3;
  }
}

// ---------------------------------------------------------------- training
// Forward over a batch, saving z1..z3 (B x 128 each, FP32), the normalised
// input u (B x 3) and dY = d loss / d output (B x 3) for the MSE loss against
// target (x_T - x_0) / out_scale; loss_rows[tile * 16 + r] gets row r's
// squared error (summed in a fixed order later).
template <bool EXACT>
__global__ void __launch_bounds__(32 * kMlpWarps) k_mlp_train_forward(MlpArgs a, const float* __restrict__ x0,
                                                                       const float* __restrict__ xT, int B,
                                                                       float* __restrict__ Z,   // 3 x B x 128
                                                                       float* __restrict__ U,   // B x kEnc
                                                                       float* __restrict__ dY,  // B x 3
                                                                       float* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem* s = reinterpret_cast<MlpSmem*>(smem_raw);
  load_weights(a, s, false);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const int tiles = (B + 15) / 16;
  const float inv = 2.0f / (3.0f * (float)B);
  for (int tile = blockIdx.x * kMlpWarps + warp; tile < tiles; tile += gridDim.x * kMlpWarps) {
    const int r0 = tile * 16 + g, r1 = r0 + 8;
    float x_0[3] = {0, 0, 0}, x_1[3] = {0, 0, 0};
    if (r0 < B)
#pragma unroll
      for (int i = 0; i < 3; ++i) x_0[i] = x0[r0 * 3 + i];
    if (r1 < B)
#pragma unroll
      for (int i = 0; i < 3; ++i) x_1[i] = x0[r1 * 3 + i];
    float e0[kEnc], e1[kEnc];
    encode<EXACT>(a, x_0, e0);
    encode<EXACT>(a, x_1, e1);
    if (t == 0) {
      if (r0 < B)
#pragma unroll
        for (int i = 0; i < kEnc; ++i) U[(size_t)r0 * kEnc + i] = e0[i];
      if (r1 < B)
#pragma unroll
        for (int i = 0; i < kEnc; ++i) U[(size_t)r1 * kEnc + i] = e1[i];
    }
    float acc[16][4];
    input_layer(s, e0, e1, t, acc);
    bias_silu(acc, s->b1, t, Z, r0, r1, B);
    dense_128<EXACT>(acc, s->W2, g, t);
    bias_silu(acc, s->b2, t, Z + (size_t)B * kH, r0, r1, B);
    dense_128<EXACT>(acc, s->W3, g, t);
    bias_silu(acc, s->b3, t, Z + (size_t)2 * B * kH, r0, r1, B);
    float o[4];
    dense_out<EXACT>(acc, s->W4, g, t, o);
    float q0 = 0.0f, q1 = 0.0f;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int c = 2 * t + q;
      if (c < 3) {
        if (r0 < B) {
          const float tgt = (xT[r0 * 3 + c] - x_0[c]) / a.out_scale[c];
          const float r = o[q] + s->b4[c] - tgt;
          dY[r0 * 3 + c] = inv * r;
          q0 += r * r;
        }
        if (r1 < B) {
          const float tgt = (xT[r1 * 3 + c] - x_1[c]) / a.out_scale[c];
          const float r = o[2 + q] + s->b4[c] - tgt;
          dY[r1 * 3 + c] = inv * r;
          q1 += r * r;
        }
      }
    }
    // row sums of the squared errors: lanes t = 0, 1 hold the columns
    q0 += __shfl_xor_sync(0xffffffffu, q0, 1);
    q1 += __shfl_xor_sync(0xffffffffu, q1, 1);
    if (t == 0) {
      if (r0 < B) err[r0] = q0;
      if (r1 < B) err[r1] = q1;
    }
  }
}

// Backward through the activations: dZ3 = (dY W4) * silu'(z3), dZ2 = (dZ3 W3) * silu'(z2),
// dZ1 = (dZ2 W2) * silu'(z1), into dZ (3 x B x 128); Z holds the pre-activations.
template <bool EXACT>
__global__ void __launch_bounds__(32 * kMlpWarps) k_mlp_train_backward(MlpArgs a, int B, const float* __restrict__ dY,
                                                                        const float* __restrict__ Z,
                                                                        float* __restrict__ dZ) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem* s = reinterpret_cast<MlpSmem*>(smem_raw);
  load_weights(a, s, true);   // W2, W3 images hold the transposes
  __shared__ float W4f[3 * kH];
  for (int i = threadIdx.x; i < 3 * kH; i += blockDim.x) W4f[i] = __uint_as_float((uint32_t)a.W4[i] << 16);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const int tiles = (B + 15) / 16;
  for (int tile = blockIdx.x * kMlpWarps + warp; tile < tiles; tile += gridDim.x * kMlpWarps) {
    const int r0 = tile * 16 + g, r1 = r0 + 8;
    float dy0[3] = {0, 0, 0}, dy1[3] = {0, 0, 0};
    if (r0 < B)
#pragma unroll
      for (int i = 0; i < 3; ++i) dy0[i] = dY[r0 * 3 + i];
    if (r1 < B)
#pragma unroll
      for (int i = 0; i < 3; ++i) dy1[i] = dY[r1 * 3 + i];
    float acc[16][4];
    // dA3 = dY W4 (FP32)
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int c = 8 * j + 2 * t;
      acc[j][0] = dy0[0] * W4f[c] + dy0[1] * W4f[kH + c] + dy0[2] * W4f[2 * kH + c];
      acc[j][1] = dy0[0] * W4f[c + 1] + dy0[1] * W4f[kH + c + 1] + dy0[2] * W4f[2 * kH + c + 1];
      acc[j][2] = dy1[0] * W4f[c] + dy1[1] * W4f[kH + c] + dy1[2] * W4f[2 * kH + c];
      acc[j][3] = dy1[0] * W4f[c + 1] + dy1[1] * W4f[kH + c + 1] + dy1[2] * W4f[2 * kH + c + 1];
    }
#pragma unroll 1
    for (int l = 2; l >= 0; --l) {
      const float* Zl = Z + (size_t)l * B * kH;
      float* dZl = dZ + (size_t)l * B * kH;
      // dZ_l = dA_l * silu'(z_l)
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = 8 * j + 2 * t;
        float zz[4] = {0, 0, 0, 0};
        if (r0 < B) {
          zz[0] = Zl[(size_t)r0 * kH + c];
          zz[1] = Zl[(size_t)r0 * kH + c + 1];
        }
        if (r1 < B) {
          zz[2] = Zl[(size_t)r1 * kH + c];
          zz[3] = Zl[(size_t)r1 * kH + c + 1];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[j][q] *= silu_grad_f(zz[q]);
        if (r0 < B) *reinterpret_cast<float2*>(dZl + (size_t)r0 * kH + c) = make_float2(acc[j][0], acc[j][1]);
        if (r1 < B) *reinterpret_cast<float2*>(dZl + (size_t)r1 * kH + c) = make_float2(acc[j][2], acc[j][3]);
      }
      if (l == 0) break;
      // dA_{l-1} = dZ_l W_l: B operand (k = out, n = in) from the transposed image W_l^T[in][out]
      dense_128<EXACT>(acc, l == 2 ? s->W3 : s->W2, g, t);
    }
  }
}

// Weight and bias gradients on the tensor cores: for layer l,
//   [dW_l | db_l] = dZ_l^T [a_{l-1} | 1]   (out x (in + 1)), summed over the batch,
// with a_0 = enc(u), a_l = silu(z_l) recomputed from the saved pre-activations
// and dZ_4 = dY.  blockIdx.x takes 64 samples, blockIdx.y the layer; both
// operands are staged transposed (rows = output / input unit, 32 BF16 pairs of
// samples per row) so that fragments are 32-bit loads, and the block writes its
// partial sums to part[blockIdx.x] (weights then biases, the layout of gW, gb).
// EXACT: both operands as three BF16 pieces, the six products of pieces whose
// orders add up to at most 2.
constexpr int kGradKC = 64;                         // samples per block
constexpr int kGradRow = kGradKC / 2 + 4;           // u32 per staged row (36: conflict-free fragment loads)
constexpr int kGradRowsA = 128, kGradRowsB = 136;   // output units; input units + the ones row, padded

template <bool EXACT>
constexpr size_t grad_smem_bytes() {
  return sizeof(uint32_t) * (EXACT ? 3 : 1) * (kGradRowsA + kGradRowsB) * kGradRow;
}

__device__ __forceinline__ size_t layer_woff(int l) {
  return l == 0 ? 0 : (size_t)kEnc * kH + (size_t)(l - 1) * kH * kH;
}

// stage rows [0, rows) x the block's samples of one operand (value(b, r)) as BF16 pieces
template <int P, typename F>
__device__ __forceinline__ void stage_t(uint32_t* dst, int rows, int b0, int B, F value) {
  for (int i = threadIdx.x; i < rows * (kGradKC / 2); i += blockDim.x) {
    const int r = i % rows, pr = i / rows;
    const int b = b0 + 2 * pr;
    const float v0 = b < B ? value(b, r) : 0.0f;
    const float v1 = b + 1 < B ? value(b + 1, r) : 0.0f;
#pragma unroll
    for (int p = 0; p < P; ++p)
      dst[(p * rows + r) * kGradRow + pr] = pack_bf16(bf16_piece(v0, p), bf16_piece(v1, p));
  }
}

// one warp: MTW m tiles from mt0 x NTW n tiles nt0, nt0 + NS, ... (< NT) of C = A^T-staged x B^T-staged
template <bool EXACT, int MTW, int NTW, int NS, int NT>
__device__ __forceinline__ void grad_tiles(const uint32_t* sA, int rowsA, const uint32_t* sB, int rowsB, int mt0,
                                           int nt0, int O, int I, size_t woff, size_t boff, float* __restrict__ part) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float acc[MTW][NTW][4];
#pragma unroll
  for (int i = 0; i < MTW; ++i)
#pragma unroll
    for (int j = 0; j < NTW; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.0f;
#pragma unroll 1
  for (int pp = 0; pp < (EXACT ? 6 : 1); ++pp) {
    // piece pairs (pa, pb) with pa + pb <= 2
    const int pa = pp < 3 ? 0 : (pp < 5 ? 1 : 2), pb = pp < 3 ? pp : (pp < 5 ? pp - 3 : 0);
    const uint32_t* A = sA + (size_t)pa * rowsA * kGradRow;
    const uint32_t* Bm = sB + (size_t)pb * rowsB * kGradRow;
#pragma unroll
    for (int kk = 0; kk < kGradKC / 16; ++kk) {
      uint32_t af[MTW][4];
#pragma unroll
      for (int i = 0; i < MTW; ++i) {
        const uint32_t* r0 = A + (16 * (mt0 + i) + g) * kGradRow + 8 * kk;
        const uint32_t* r1 = r0 + 8 * kGradRow;
        af[i][0] = r0[t];
        af[i][1] = r1[t];
        af[i][2] = r0[4 + t];
        af[i][3] = r1[4 + t];
      }
#pragma unroll
      for (int j = 0; j < NTW; ++j) {
        const int nt = nt0 + j * NS;
        if (nt < NT) {
          const uint32_t* row = Bm + (8 * nt + g) * kGradRow + 8 * kk;
          const uint32_t b0 = row[t], b1 = row[4 + t];
#pragma unroll
          for (int i = 0; i < MTW; ++i) mma16816(acc[i][j], af[i], b0, b1);
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < MTW; ++i)
#pragma unroll
    for (int j = 0; j < NTW; ++j) {
      const int nt = nt0 + j * NS;
      if (nt >= NT) continue;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int o = 16 * (mt0 + i) + g + (q >= 2 ? 8 : 0), c = 8 * nt + 2 * t + (q & 1);
        if (o >= O) continue;
        if (c < I) part[woff + (size_t)o * I + c] = acc[i][j][q];
        else if (c == I) part[(size_t)kMlpNW + boff + o] = acc[i][j][q];
      }
    }
}

template <bool EXACT>
__global__ void __launch_bounds__(128, 1) k_mlp_weight_grads(int B, const float* __restrict__ U,
                                                             const float* __restrict__ Zf, const float* __restrict__ dZ,
                                                             const float* __restrict__ dY, float* __restrict__ part) {
  extern __shared__ __align__(16) uint32_t gsm[];
  constexpr int P = EXACT ? 3 : 1;
  const int layer = blockIdx.y, b0 = blockIdx.x * kGradKC, warp = threadIdx.x >> 5;
  const int I = layer == 0 ? kEnc : kH, O = layer == 3 ? 3 : kH;
  const int rowsA = layer == 3 ? 16 : kGradRowsA, rowsB = layer == 0 ? 40 : kGradRowsB;
  uint32_t* sA = gsm;
  uint32_t* sB = gsm + (size_t)P * rowsA * kGradRow;
  float* out = part + (size_t)blockIdx.x * (kMlpNW + kMlpNB);
  if (layer == 3)
    stage_t<P>(sA, rowsA, b0, B, [&](int b, int r) { return r < 3 ? dY[(size_t)b * 3 + r] : 0.0f; });
  else
    stage_t<P>(sA, rowsA, b0, B, [&](int b, int r) { return dZ[((size_t)layer * B + b) * kH + r]; });
  if (layer == 0)
    stage_t<P>(sB, rowsB, b0, B, [&](int b, int r) { return r < kEnc ? U[(size_t)b * kEnc + r] : (r == kEnc ? 1.0f : 0.0f); });
  else
    stage_t<P>(sB, rowsB, b0, B, [&](int b, int r) {
      return r < kH ? silu_f(Zf[((size_t)(layer - 1) * B + b) * kH + r]) : (r == kH ? 1.0f : 0.0f);
    });
  __syncthreads();
  const size_t woff = layer_woff(layer), boff = (size_t)layer * kH;
  if (layer == 0)
    grad_tiles<EXACT, 2, 5, 1, 5>(sA, rowsA, sB, rowsB, 2 * warp, 0, O, I, woff, boff, out);
  else if (layer < 3)
    grad_tiles<EXACT, 2, 17, 1, 17>(sA, rowsA, sB, rowsB, 2 * warp, 0, O, I, woff, boff, out);
  else
    grad_tiles<EXACT, 1, 5, 4, 17>(sA, rowsA, sB, rowsB, 0, warp, O, I, woff, boff, out);
}

// gW, gb = the blocks' partial sums added in block order
__global__ void k_mlp_grad_sum(const float* __restrict__ part, int nparts, float* __restrict__ gW,
                               float* __restrict__ gb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpNW + kMlpNB) return;
  float acc = 0.0f;
  for (int c = 0; c < nparts; ++c) acc += part[(size_t)c * (kMlpNW + kMlpNB) + i];
  if (i < kMlpNW) gW[i] = acc;
  else gb[i - kMlpNW] = acc;
}

// Adam on FP32 masters; rewrites the BF16 copies (and the transposed copies of W2, W3)
__global__ void k_mlp_adam(int64_t nW, int64_t nb, float* __restrict__ W, float* __restrict__ b,
                           const float* __restrict__ gW, const float* __restrict__ gb, float* __restrict__ mW,
                           float* __restrict__ vW, float* __restrict__ mb, float* __restrict__ vb, float lr, float beta1,
                           float beta2, float eps, float c1, float c2, uint16_t* __restrict__ Wbf,
                           uint16_t* __restrict__ W2t, uint16_t* __restrict__ W3t) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nW) {
    const float gr = gW[i];
    const float m = beta1 * mW[i] + (1.0f - beta1) * gr;
    const float v = beta2 * vW[i] + (1.0f - beta2) * gr * gr;
    mW[i] = m;
    vW[i] = v;
    const float w = W[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    W[i] = w;
    __nv_bfloat16 wb = __float2bfloat16_rn(w);
    const uint16_t bits = *reinterpret_cast<uint16_t*>(&wb);
    Wbf[i] = bits;
    const int64_t o2 = (int64_t)kEnc * kH, o3 = o2 + kH * kH;
    if (i >= o2 && i < o3) {
      const int64_t r = (i - o2) / kH, c = (i - o2) % kH;
      W2t[c * kH + r] = bits;
    } else if (i >= o3 && i < o3 + kH * kH) {
      const int64_t r = (i - o3) / kH, c = (i - o3) % kH;
      W3t[c * kH + r] = bits;
    }
  } else if (i < nW + nb) {
    const int64_t k = i - nW;
    const float gr = gb[k];
    const float m = beta1 * mb[k] + (1.0f - beta1) * gr;
    const float v = beta2 * vb[k] + (1.0f - beta2) * gr * gr;
    mb[k] = m;
    vb[k] = v;
    b[k] = b[k] - lr * (m / c1) / (sqrtf(v / c2) + eps);
  }
}

// fixed-order sum of the per-row squared errors -> mean loss
__global__ void __launch_bounds__(1024) k_mlp_loss(const float* __restrict__ err, int B, float* __restrict__ loss) {
  __shared__ double sh[1024];
  double a = 0.0;
  for (int i = threadIdx.x; i < B; i += blockDim.x) a += err[i];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = (float)(sh[0] / (3.0 * B));
}

// BF16 copies of the FP32 masters (and the transposes of W2, W3)
__global__ void k_mlp_refresh(const float* __restrict__ W, uint16_t* __restrict__ Wbf, uint16_t* __restrict__ W2t,
                              uint16_t* __restrict__ W3t) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpNW) return;
  __nv_bfloat16 wb = __float2bfloat16_rn(W[i]);
  const uint16_t bits = *reinterpret_cast<uint16_t*>(&wb);
  Wbf[i] = bits;
  const int64_t o2 = (int64_t)kEnc * kH, o3 = o2 + kH * kH;
  if (i >= o2 && i < o3) W2t[((i - o2) % kH) * kH + (i - o2) / kH] = bits;
  else if (i >= o3 && i < o3 + kH * kH) W3t[((i - o3) % kH) * kH + (i - o3) / kH] = bits;
}

// ------------------------------------------------------------------ host
static MlpArgs mlp_args(const pdmp_mlp* net) {
  MlpArgs a;
  const uint16_t* w = net->W_bf16;
  a.W1 = w;
  a.W2 = w + kEnc * kH;
  a.W3 = w + kEnc * kH + kH * kH;
  a.W4 = w + kEnc * kH + 2 * kH * kH;
  a.W2t = net->Wt_bf16;
  a.W3t = net->Wt_bf16 + kH * kH;
  a.b1 = net->b;
  a.b2 = net->b + kH;
  a.b3 = net->b + 2 * kH;
  a.b4 = net->b + 3 * kH;
  for (int i = 0; i < 3; ++i) {
    a.lo[i] = net->lo[i];
    a.in_scale[i] = net->in_scale[i];
    a.out_scale[i] = net->out_scale[i];
  }
  return a;
}

static int mlp_grid(int64_t tiles, const void* kernel) {
  int dev = 0, sms = 1, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 32 * kMlpWarps, sizeof(MlpSmem));
  if (per < 1) per = 1;
  int64_t want = (tiles + kMlpWarps - 1) / kMlpWarps;
  int64_t cap = (int64_t)sms * per;
  return (int)(want < cap ? (want < 1 ? 1 : want) : cap);
}

cudaError_t mlp_refresh(const pdmp_mlp* net, cudaStream_t st) {
  k_mlp_refresh<<<(unsigned)((kMlpNW + 255) / 256), 256, 0, st>>>(net->W, net->W_bf16, net->Wt_bf16,
                                                                  net->Wt_bf16 + kH * kH);
  return cudaGetLastError();
}

cudaError_t mlp_forward(const pdmp_mlp* net, const float* x0, int64_t N, float* y, bool fp32_act, cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  return mlp_forward_tc05(net, x0, N, y, fp32_act, st);
}

static size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

static int grad_parts(int B) { return (B + kGradKC - 1) / kGradKC; }

size_t mlp_train_workspace(int B) {
  return 2 * al256(sizeof(float) * 3 * (size_t)B * kH) + al256(sizeof(float) * kEnc * (size_t)B) +
         2 * al256(sizeof(float) * 3 * (size_t)B) + al256(sizeof(float) * kMlpNW) + al256(sizeof(float) * kMlpNB) +
         al256(sizeof(float) * (size_t)grad_parts(B) * (kMlpNW + kMlpNB));
}

template <bool EXACT>
static cudaError_t launch_gradient(const pdmp_mlp* net, const float* x0, const float* xT, int B, float* loss,
                                   float* gW, float* gb, char* p, cudaStream_t st) {
  auto take = [&](size_t b) { char* q = p; p += al256(b); return q; };
  float* Z = (float*)take(sizeof(float) * 3 * (size_t)B * kH);
  float* dZ = (float*)take(sizeof(float) * 3 * (size_t)B * kH);
  float* U = (float*)take(sizeof(float) * kEnc * (size_t)B);
  float* dY = (float*)take(sizeof(float) * 3 * (size_t)B);
  float* err = (float*)take(sizeof(float) * 3 * (size_t)B);
  take(sizeof(float) * kMlpNW);   // gW, gb of the training step
  take(sizeof(float) * kMlpNB);
  float* part = (float*)take(sizeof(float) * (size_t)grad_parts(B) * (kMlpNW + kMlpNB));
  const MlpArgs a = mlp_args(net);
  const size_t smem = sizeof(MlpSmem);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_mlp_train_forward<EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
    return e;
  if ((e = cudaFuncSetAttribute(k_mlp_train_backward<EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
    return e;
  constexpr size_t gsmem = grad_smem_bytes<EXACT>();
  if ((e = cudaFuncSetAttribute(k_mlp_weight_grads<EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsmem)))
    return e;
  const int64_t tiles = (B + 15) / 16;
  const int gf = mlp_grid(tiles, (const void*)k_mlp_train_forward<EXACT>);
  k_mlp_train_forward<EXACT><<<gf, 32 * kMlpWarps, smem, st>>>(a, x0, xT, B, Z, U, dY, err);
  if (loss) k_mlp_loss<<<1, 1024, 0, st>>>(err, B, loss);
  const int gbk = mlp_grid(tiles, (const void*)k_mlp_train_backward<EXACT>);
  k_mlp_train_backward<EXACT><<<gbk, 32 * kMlpWarps, smem, st>>>(a, B, dY, Z, dZ);
  k_mlp_weight_grads<EXACT><<<dim3((unsigned)grad_parts(B), 4), 128, gsmem, st>>>(B, U, Z, dZ, dY, part);
  k_mlp_grad_sum<<<(unsigned)((kMlpNW + kMlpNB + 255) / 256), 256, 0, st>>>(part, grad_parts(B), gW, gb);
  return cudaGetLastError();
}

cudaError_t mlp_gradient(const pdmp_mlp* net, const float* x0, const float* xT, int B, bool fp32_act, float* loss,
                         float* gW, float* gb, void* ws, cudaStream_t st) {
  return fp32_act ? launch_gradient<true>(net, x0, xT, B, loss, gW, gb, (char*)ws, st)
                  : launch_gradient<false>(net, x0, xT, B, loss, gW, gb, (char*)ws, st);
}

cudaError_t mlp_train_step(const pdmp_mlp* net, const float* x0, const float* xT, int B, float lr, float beta1,
                           float beta2, float eps, int step, float* loss, void* ws, cudaStream_t st) {
  char* p = (char*)ws + 2 * al256(sizeof(float) * 3 * (size_t)B * kH) + al256(sizeof(float) * kEnc * (size_t)B) +
            2 * al256(sizeof(float) * 3 * (size_t)B);
  float* gW = (float*)p;
  float* gb = (float*)(p + al256(sizeof(float) * kMlpNW));
  cudaError_t e = launch_gradient<false>(net, x0, xT, B, loss, gW, gb, (char*)ws, st);
  if (e != cudaSuccess) return e;
  float* mW = net->adam;
  float* vW = net->adam + kMlpNW;
  float* mb = net->adam + 2 * kMlpNW;
  float* vb = net->adam + 2 * kMlpNW + kMlpNB;
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  k_mlp_adam<<<(unsigned)((kMlpNW + kMlpNB + 255) / 256), 256, 0, st>>>(
      kMlpNW, kMlpNB, net->W, net->b, gW, gb, mW, vW, mb, vb, lr, beta1, beta2, eps, c1, c2, net->W_bf16,
      net->Wt_bf16, net->Wt_bf16 + kH * kH);
  return cudaGetLastError();
}

}  // namespace pdmp
