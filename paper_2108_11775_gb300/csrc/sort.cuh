// Spatial sort of samples (see sort.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pdmp {

constexpr int kScanThreads = 1024;
constexpr int kScanChunk = 2 * kScanThreads;

// monotone map float -> uint32 (for atomicMin / atomicMax on floats)
__device__ __forceinline__ uint32_t ordered_bits(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_ordered(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// spreads the low 10 bits of v so that bit i lands at bit i * 2 (d = 2) or i * 3 (d = 3)
__device__ __forceinline__ uint32_t spread2(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 8)) & 0x00ff00ffu;
  v = (v | (v << 4)) & 0x0f0f0f0fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Hilbert index of the cell (c_0 .. c_{n-1}), each coordinate `bits` wide,
// by Skilling's method ("Programming the Hilbert curve", 2004): the
// coordinates are turned in place into the transposed index (undoing the
// curve's reflections and exchanges level by level, then Gray-decoding), whose
// bits interleaved with c_0 most significant give the index.  Consecutive
// indices are adjacent cells, so a run of sorted samples never jumps.
template <int n>
__device__ __forceinline__ uint32_t hilbert_key(uint32_t (&c)[n], int bits) {
  const uint32_t top = 1u << (bits - 1);
  for (uint32_t q = top; q > 1; q >>= 1) {
    const uint32_t p = q - 1;
#pragma unroll
    for (int i = 0; i < n; ++i) {
      if (c[i] & q) {
        c[0] ^= p;                        // reflect
      } else {
        const uint32_t t = (c[0] ^ c[i]) & p;   // exchange the low bits of c_0 and c_i
        c[0] ^= t;
        c[i] ^= t;
      }
    }
  }
#pragma unroll
  for (int i = 1; i < n; ++i) c[i] ^= c[i - 1];
  uint32_t t = 0;
  for (uint32_t q = top; q > 1; q >>= 1)
    if (c[n - 1] & q) t ^= q - 1;
#pragma unroll
  for (int i = 0; i < n; ++i) c[i] ^= t;
  uint32_t key = 0;
  if (n == 2) {
    key = (spread2(c[0]) << 1) | spread2(c[n - 1]);
  } else {
    key = (spread3(c[0]) << 2) | (spread3(c[1 % n]) << 1) | spread3(c[n - 1]);
  }
  return key;
}

// cell index in [0, cells) of v along one axis of the box [lo, hi]; NaN and
// values below lo give 0, values at or above hi give cells - 1
__device__ __forceinline__ uint32_t cell_coord(float v, float lo, float hi, float cells) {
  const float span = hi - lo;
  const float q = span > 0.0f ? (v - lo) * (cells / span) : 0.0f;
  return (q >= 0.0f) ? (uint32_t)fminf(q, cells - 1.0f) : 0u;
}

struct SortWs {
  int bits;           // grid cells per axis = 2^bits
  int64_t cells;      // 2^(d * bits)
  int64_t nchunks;    // scan chunks
  uint32_t* box;      // 2d ordered-float bounds
  uint32_t* keys;     // N cell keys
  int32_t* perm;      // N: sorted position -> original index
  uint32_t* counts;   // cells
  uint32_t* offs;     // cells
  uint32_t* cursor;   // cells
  uint32_t* chunk_tot;
  size_t bytes;       // total bytes of the layout
};

int sort_bits(int d, int64_t N);
SortWs sort_layout(void* ws, int d, int64_t N);
size_t sort_workspace(int d, int64_t N);
// bounding box of N points (d = 2, 3) as 2d ordered-float words: box[j] = min, box[d + j] = max
cudaError_t bounding_box(int d, const float* x, int64_t N, uint32_t* box, cudaStream_t st);
cudaError_t spatial_sort(int d, const float* x, int64_t N, const SortWs& s, cudaStream_t st);
// exclusive prefix sum of n uint32 values (chunk_tot: ceil(n / kScanChunk) scratch words)
cudaError_t exclusive_scan_u32(const uint32_t* in, int64_t n, uint32_t* out, uint32_t* chunk_tot, cudaStream_t st);
// counting sort of N items by keys[] < cells, given counts[] (item counts per
// key): perm receives the items in key order, each key's items by index when
// a key holds at most 64 items
cudaError_t sort_by_keys(const uint32_t* keys, int64_t N, const uint32_t* counts, uint32_t* offs, uint32_t* cursor,
                         uint32_t* chunk_tot, int64_t cells, int32_t* perm, cudaStream_t st);

}  // namespace pdmp
