// Surrogate MLP inference on the fifth-generation tensor cores (tcgen05):
// y = x0 + out_scale * f(u(x0)) for the network of mlp.cu (39 -> 128 -> 128
// -> 128 -> 3, SiLU, BF16 weights), 128 samples a tile.
//
// Every layer is one tcgen05.mma chain, M = 128 samples, A = the layer's input
// activations and B = its weights, both BF16 in shared memory in the
// canonical K-major layout (tc05.cuh), D = FP32 in tensor memory:
//   layer 1: A = [enc_hi | enc_lo] (K = 2 x 48: the Fourier encoding split
//            into two BF16 pieces, 39 values and zero padding each), B =
//            [W1 | W1]: the product is enc W1^T to about 2^-16 of enc;
//   layers 2, 3: A = BF16(silu(z)) (K = 128), N = 128;
//   layer 4: N = 16 (3 outputs and zero rows).
// The epilogue of a layer reads D from TMEM (thread = sample row, sixteen
// warps: warps w, w + 4, w + 8 and w + 12 share the TMEM lanes 32 (w % 4) ..
// + 31 and take 32 columns each), adds the bias, applies SiLU and writes the
// next A.  (Sixteen warps ran 5 % faster than eight of 64 columns each:
// 0.438 against 0.462 ms for 2^20 samples.)
// Three tiles are in flight per CTA: while the epilogue warps run one tile's
// epilogue the tensor core runs another tile's next layer.  A warp of its own
// issues the MMAs; the two sides hand tiles over through mbarriers (the
// issuer's commit to "D ready", the epilogue warps' arrivals to "A ready"),
// so neither waits at a block barrier (2^20 samples: 0.324 ms against 0.438
// with block barriers and the MMAs issued by an epilogue thread).
//
// FP32-activation mode (diagnostic): one tile in flight, the activations as
// three BF16 pieces (three MMA chains over the same weights), the encoding as
// three pieces, CUDA's sinf / cosf / expf; the products are then those of FP32
// activations with the BF16 weights.
//
// Waits on the tensor core are bounded (about a second): past the limit the
// kernel raises PDMP_FLAG_MMA_TIMEOUT, waits (bounded again) for what it
// issued, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "mlp_common.cuh"
#include "tc05.cuh"

namespace pdmp {
namespace {

constexpr int kH = 128, kEnc = 39, kEncPad = 48;
constexpr int kRows = 128;                        // samples a tile (M)
constexpr int kCompute = 512;                     // 16 epilogue warps
constexpr int kThreads = kCompute + 32;           // and one warp that issues the MMAs
constexpr int kCWarps = kCompute / 32;
constexpr int kGroups = kCompute / 128;           // warps sharing a TMEM lane quarter (column groups)
constexpr int kGroupCols = kH / kGroups;          // hidden columns a thread takes in an epilogue
constexpr long long kWaitClocks = 1ll << 31;

// canonical K-major images (bytes)
constexpr uint32_t kW1Bytes = kH * 2 * kEncPad * 2;   // [W1 | W1], K = 96
constexpr uint32_t kWBytes = kH * kH * 2;             // W2, W3
constexpr uint32_t kW4Bytes = 16 * kH * 2;            // W4, N = 16
constexpr uint32_t kABytes = kRows * kH * 2;          // one A piece of one tile
constexpr uint32_t kSbo96 = (2 * kEncPad * 2 / 16) * 128;   // 1536
constexpr uint32_t kSbo128 = (kH * 2 / 16) * 128;           // 2048

template <bool EXACT>
struct Cfg {
  // tiles in flight: 3 (2^20 samples: 0.311 ms; 2 tiles 0.324, 4 tiles 0.332)
  static constexpr int kTiles = EXACT ? 1 : 3;
  static constexpr uint32_t kTmemCols = kTiles * kH <= 256 ? 256u : 512u;
  static constexpr int kPieces = EXACT ? 3 : 1;    // BF16 pieces of a hidden activation
  static constexpr int kEncBufs = EXACT ? 2 : 1;   // A buffers of layer 1 (K = 96 each)
  static constexpr int kABufs = kPieces > kEncBufs ? kPieces : kEncBufs;
  static constexpr uint32_t kOffW1 = 0;
  static constexpr uint32_t kOffW2 = kOffW1 + kW1Bytes;
  static constexpr uint32_t kOffW3 = kOffW2 + kWBytes;
  static constexpr uint32_t kOffW4 = kOffW3 + kWBytes;
  static constexpr uint32_t kOffA = kOffW4 + kW4Bytes;
  static constexpr uint32_t kOffBias = kOffA + (uint32_t)kTiles * kABufs * kABytes;
  static constexpr uint32_t kOffBar = kOffBias + (3 * kH + 4) * 4;
  static constexpr uint32_t kBytes = kOffBar + 64;
  static_assert(2 * kTiles * 8 <= 64, "two barriers a tile");
  static_assert(kBytes <= 227 * 1024, "shared memory of one CTA");
};

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// piece p of the BF16 split of x (x = p0 + p1 + p2 up to 2^-27 |x|)
__device__ __forceinline__ float piece(float x, int p) {
  const float h = __bfloat162float(__float2bfloat16_rn(x));
  if (p == 0) return h;
  const float r = x - h;
  const float m = __bfloat162float(__float2bfloat16_rn(r));
  return p == 1 ? m : r - m;
}

__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// SiLU: z sigma(z) = z (1 + tanh(z / 2)) / 2 on the special-function unit;
// the FP32-activation mode takes z / (1 + e^-z) with CUDA's expf
template <bool EXACT>
__device__ __forceinline__ float silu(float z) {
  if constexpr (EXACT) return z / (1.0f + expf(-z));
  const float h = 0.5f * z;
  return fmaf(h, tanh_approx(h), h);
}

struct MlpTcArgs {
  const uint16_t* W;   // BF16 weights: W1 (128 x 39), W2, W3 (128 x 128), W4 (3 x 128)
  const float* b;      // b1, b2, b3 (128 each), b4 (3)
  float lo[3], in_scale[3], out_scale[3];
};

template <bool EXACT>
__global__ void __launch_bounds__(kThreads, 1)
k_mlp_forward_tc05(MlpTcArgs a, const float* __restrict__ x0, int64_t N, float* __restrict__ y) {
  using C = Cfg<EXACT>;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3, cg = warp >> 2;     // lane quarter, column group
  const int row = 32 * q + lane;                  // this thread's sample within a tile (TMEM lane)
  const uint32_t sbase = tc05::smem_u32(sm);
  float* bias = reinterpret_cast<float*>(sm + C::kOffBias);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + C::kOffBar);

  // ---- weights into their canonical images, biases; barriers; tensor memory
  {
    const uint16_t* W1 = a.W;
    const uint16_t* W2 = a.W + kEnc * kH;
    const uint16_t* W3 = W2 + kH * kH;
    const uint16_t* W4 = W3 + kH * kH;
    for (int i = tid; i < kH * kEncPad; i += kThreads) {      // [W1 | W1]
      const int n = i / kEncPad, k = i % kEncPad;
      const uint16_t v = k < kEnc ? W1[n * kEnc + k] : (uint16_t)0;
      *reinterpret_cast<uint16_t*>(sm + C::kOffW1 + tc05::kmajor_offset(n, k, 12, 2)) = v;
      *reinterpret_cast<uint16_t*>(sm + C::kOffW1 + tc05::kmajor_offset(n, kEncPad + k, 12, 2)) = v;
    }
    for (int i = tid; i < kH * kH / 2; i += kThreads) {       // W2, W3: pairs along k
      const int n = i / (kH / 2), k = 2 * (i % (kH / 2));
      const uint32_t v2 = (uint32_t)W2[n * kH + k] | ((uint32_t)W2[n * kH + k + 1] << 16);
      const uint32_t v3 = (uint32_t)W3[n * kH + k] | ((uint32_t)W3[n * kH + k + 1] << 16);
      *reinterpret_cast<uint32_t*>(sm + C::kOffW2 + tc05::kmajor_offset(n, k, 16, 2)) = v2;
      *reinterpret_cast<uint32_t*>(sm + C::kOffW3 + tc05::kmajor_offset(n, k, 16, 2)) = v3;
    }
    for (int i = tid; i < 16 * kH / 2; i += kThreads) {       // W4, rows 3..15 zero
      const int n = i / (kH / 2), k = 2 * (i % (kH / 2));
      const uint32_t v = n < 3 ? ((uint32_t)W4[n * kH + k] | ((uint32_t)W4[n * kH + k + 1] << 16)) : 0u;
      *reinterpret_cast<uint32_t*>(sm + C::kOffW4 + tc05::kmajor_offset(n, k, 16, 2)) = v;
    }
    for (int i = tid; i < 3 * kH + 4; i += kThreads) bias[i] = i < 3 * kH + 3 ? a.b[i] : 0.0f;
    if (tid == 0) {
      for (int t = 0; t < C::kTiles; ++t) {
        tc05::mbar_init(&bar[t], 1);                    // tile t's MMAs done (commit)
        tc05::mbar_init(&bar[C::kTiles + t], kCWarps);  // tile t's A operand written (epilogue warps)
      }
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      abort_sh = 0;
    }
    if (warp == 0) tc05::tmem_alloc(&tmem_base_sh, C::kTmemCols);
    tc05::fence_async_smem();
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
  }
  const uint32_t tmem = tmem_base_sh;
  const uint32_t taddr_lane = tmem + ((uint32_t)(32 * q) << 16);
  constexpr uint32_t id_hidden = tc05::idesc(tc05::kBF16, tc05::kBF16, kRows, kH);
  constexpr uint32_t id_out = tc05::idesc(tc05::kBF16, tc05::kBF16, kRows, 16);
  auto a_buf = [&](int t, int p) -> uint32_t { return C::kOffA + (uint32_t)(t * C::kABufs + p) * kABytes; };
  uint64_t* bar_d = bar;                 // [kTiles] MMAs of the tile done
  uint64_t* bar_a = bar + C::kTiles;     // [kTiles] the tile's next A operand written
  auto fail = [&]() {
    if (!abort_sh) raise_flag(FLAG_MMA_TIMEOUT);
    abort_sh = 1;
  };
  const int64_t tiles = (N + kRows - 1) / kRows;
  const int64_t groups = (tiles + C::kTiles - 1) / C::kTiles;

  if (warp == kCWarps) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      uint32_t pa[C::kTiles], pd[C::kTiles];
      bool pending[C::kTiles];
#pragma unroll
      for (int t = 0; t < C::kTiles; ++t) {
        pa[t] = 0u;
        pd[t] = 0u;
        pending[t] = false;
      }
      bool ok = true;
      for (int64_t grp = blockIdx.x; grp < groups && ok; grp += gridDim.x)
#pragma unroll 1
        for (int layer = 1; layer <= 4 && ok; ++layer)
#pragma unroll
          for (int t = 0; t < C::kTiles; ++t) {
            if (abort_sh || !tc05::mbar_wait(&bar_a[t], pa[t], kWaitClocks)) {
              fail();
              ok = false;
              break;
            }
            pa[t] ^= 1u;
            tc05::fence_after_sync();
            const uint32_t d = tmem + (uint32_t)(t * kH);
            uint32_t acc = 0u;
            if (layer == 1) {
#pragma unroll 1
              for (int p = 0; p < C::kEncBufs; ++p)
                for (int s = 0; s < 2 * kEncPad / 16; ++s) {
                  const uint64_t ad = tc05::sdesc(sbase + a_buf(t, p) + s * 256, 128, kSbo96);
                  const uint64_t bd = tc05::sdesc(sbase + C::kOffW1 + s * 256, 128, kSbo96);
                  tc05::mma_ss(d, ad, bd, id_hidden, acc);
                  acc = 1u;
                }
            } else {
              const uint32_t w = layer == 2 ? C::kOffW2 : (layer == 3 ? C::kOffW3 : C::kOffW4);
              const uint32_t id = layer == 4 ? id_out : id_hidden;
#pragma unroll 1
              for (int p = 0; p < C::kPieces; ++p)
                for (int s = 0; s < kH / 16; ++s) {
                  const uint64_t ad = tc05::sdesc(sbase + a_buf(t, p) + s * 256, 128, kSbo128);
                  const uint64_t bd = tc05::sdesc(sbase + w + s * 256, 128, kSbo128);
                  tc05::mma_ss(d, ad, bd, id, acc);
                  acc = 1u;
                }
            }
            tc05::commit(&bar_d[t]);
            if (pending[t]) pd[t] ^= 1u;   // the previous commit of this tile has been waited for by the epilogue
            pending[t] = true;
          }
      // before the tensor memory is freed: this thread's last commit of each tile (bounded)
#pragma unroll
      for (int t = 0; t < C::kTiles; ++t)
        if (pending[t]) tc05::mbar_wait(&bar_d[t], pd[t], kWaitClocks);
    }
  } else {
    // ---------------------------------------------------------- epilogue warps
    uint32_t pd[C::kTiles];
#pragma unroll
    for (int t = 0; t < C::kTiles; ++t) pd[t] = 0u;
    // lane 0 waits for the warp (bounded); false after any failure
    auto wait_d = [&](int t) -> bool {
      int ok_ = 1;
      if (lane == 0) {
        ok_ = !abort_sh && tc05::mbar_wait(&bar_d[t], pd[t], kWaitClocks);
        if (!ok_) fail();
      }
      __syncwarp();
      ok_ = __shfl_sync(0xffffffffu, ok_, 0);
      if (ok_) pd[t] ^= 1u;
      tc05::fence_after_sync();
      return ok_ != 0;
    };
    // the warp's writes of tile t's A operand (and its reads of the tile's
    // accumulator) are done: hand the tile to the issuer
    auto ready = [&](int t) {
      tc05::fence_async_smem();
      tc05::fence_before_sync();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc05::smem_u32(&bar_a[t])) : "memory");
    };
    // the encoding of tile t's samples into its layer-1 A buffers: this thread
    // writes K pairs [6 cg, 6 cg + 6) of its row (pairs 0..23)
    auto encode = [&](int t, int64_t n0) {
      float xv[3] = {0.0f, 0.0f, 0.0f};
      const int64_t n = n0 + row;
      if (n < N)
#pragma unroll
        for (int j = 0; j < 3; ++j) xv[j] = x0[n * 3 + j];
      MlpEncIn u;
      mlp_enc_prepare(xv, a.lo, a.in_scale, u);
      constexpr int np = kEncPad / 2 / kGroups;
      static_assert(np * kGroups == kEncPad / 2, "the encoding's K pairs split evenly over the column groups");
#pragma unroll
      for (int i = 0; i < np; ++i) {
        const int kp = np * cg + i;
        const float v0 = mlp_enc_feature<EXACT>(2 * kp, u), v1 = mlp_enc_feature<EXACT>(2 * kp + 1, u);
        if constexpr (EXACT) {
          *reinterpret_cast<uint32_t*>(sm + a_buf(t, 0) + tc05::kmajor_offset(row, 2 * kp, 12, 2)) =
              pack2(piece(v0, 0), piece(v1, 0));
          *reinterpret_cast<uint32_t*>(sm + a_buf(t, 0) + tc05::kmajor_offset(row, kEncPad + 2 * kp, 12, 2)) =
              pack2(piece(v0, 1), piece(v1, 1));
          *reinterpret_cast<uint32_t*>(sm + a_buf(t, 1) + tc05::kmajor_offset(row, 2 * kp, 12, 2)) =
              pack2(piece(v0, 2), piece(v1, 2));
          *reinterpret_cast<uint32_t*>(sm + a_buf(t, 1) + tc05::kmajor_offset(row, kEncPad + 2 * kp, 12, 2)) = 0u;
        } else {
          *reinterpret_cast<uint32_t*>(sm + a_buf(t, 0) + tc05::kmajor_offset(row, 2 * kp, 12, 2)) =
              pack2(piece(v0, 0), piece(v1, 0));
          *reinterpret_cast<uint32_t*>(sm + a_buf(t, 0) + tc05::kmajor_offset(row, kEncPad + 2 * kp, 12, 2)) =
              pack2(piece(v0, 1), piece(v1, 1));
        }
      }
    };

    // epilogue of a hidden layer of tile t: D (this thread's row, its
    // kGroupCols columns) + bias, SiLU, into the next layer's A pieces
    auto hidden = [&](int t, const float* bl) {
#pragma unroll 1
      for (int c = 0; c < kGroupCols / 32; ++c) {
        const int col0 = kGroupCols * cg + 32 * c;
        float v[32];
        tc05::ld32(taddr_lane + (uint32_t)(t * kH + col0), v);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = silu<EXACT>(v[i] + bl[col0 + i]);
#pragma unroll
        for (int p = 0; p < C::kPieces; ++p)
#pragma unroll
          for (int kc = 0; kc < 4; ++kc) {
            uint4 w;
            w.x = pack2(piece(v[8 * kc + 0], p), piece(v[8 * kc + 1], p));
            w.y = pack2(piece(v[8 * kc + 2], p), piece(v[8 * kc + 3], p));
            w.z = pack2(piece(v[8 * kc + 4], p), piece(v[8 * kc + 5], p));
            w.w = pack2(piece(v[8 * kc + 6], p), piece(v[8 * kc + 7], p));
            *reinterpret_cast<uint4*>(sm + a_buf(t, p) + tc05::kmajor_offset(row, col0 + 8 * kc, 16, 2)) = w;
          }
      }
    };


    bool ok = true;
    for (int64_t grp = blockIdx.x; grp < groups && ok; grp += gridDim.x) {
      int64_t n0[C::kTiles];
#pragma unroll
      for (int t = 0; t < C::kTiles; ++t) {
        n0[t] = (grp * C::kTiles + t) * kRows;
        encode(t, n0[t]);
        ready(t);
      }
#pragma unroll 1
      for (int layer = 1; layer <= 3 && ok; ++layer)
#pragma unroll
        for (int t = 0; t < C::kTiles; ++t) {
          if (!(ok = wait_d(t))) break;
          hidden(t, bias + (layer - 1) * kH);
          ready(t);
        }
#pragma unroll
      for (int t = 0; t < C::kTiles && ok; ++t) {
        if (!(ok = wait_d(t))) break;
        if (cg == 0) {
          float o[16];
          tc05::ld16(taddr_lane + (uint32_t)(t * kH), o);
          const int64_t n = n0[t] + row;
          if (n < N)
#pragma unroll
            for (int j = 0; j < 3; ++j) y[n * 3 + j] = fmaf(o[j] + bias[3 * kH + j], a.out_scale[j], x0[n * 3 + j]);
        }
      }
    }
  }
  tc05::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc05::fence_after_sync();
    tc05::tmem_dealloc(tmem, C::kTmemCols);
  }
}

template <bool EXACT>
cudaError_t launch(const pdmp_mlp* net, const float* x0, int64_t N, float* y, cudaStream_t st) {
  using C = Cfg<EXACT>;
  MlpTcArgs a;
  a.W = net->W_bf16;
  a.b = net->b;
  for (int i = 0; i < 3; ++i) {
    a.lo[i] = net->lo[i];
    a.in_scale[i] = net->in_scale[i];
    a.out_scale[i] = net->out_scale[i];
  }
  cudaError_t e = cudaFuncSetAttribute(k_mlp_forward_tc05<EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)C::kBytes);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 1;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int64_t groups = ((N + kRows - 1) / kRows + C::kTiles - 1) / C::kTiles;
  const int grid = (int)(groups < sms ? groups : sms);
  k_mlp_forward_tc05<EXACT><<<grid, kThreads, C::kBytes, st>>>(a, x0, N, y);
  return cudaGetLastError();
}

}  // namespace

size_t mlp_forward_tc05_smem(bool fp32_act) { return fp32_act ? Cfg<true>::kBytes : Cfg<false>::kBytes; }

cudaError_t mlp_forward_tc05(const pdmp_mlp* net, const float* x0, int64_t N, float* y, bool fp32_act,
                             cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  return fp32_act ? launch<true>(net, x0, N, y, st) : launch<false>(net, x0, N, y, st);
}

}  // namespace pdmp
