// Spatial ordering of the samples for the fast RBF morph: a counting sort of
// the samples by the Hilbert index of their grid cell (over the samples'
// bounding box).  Consecutive samples of the resulting permutation are
// spatially close (the Hilbert order never jumps between distant cells),
// which keeps a tile's extent small.
//
// Determinism.  The scatter places a cell's samples in atomic arrival order;
// k_order_cells then orders every cell of 2 to 64 samples by original index.
// The grid is sized for about four samples per cell, so on inputs spread over
// their bounding box every cell is ordered and the permutation, the tiles and
// every result are reproducible bit for bit.  A cell of more than 64 samples
// (clustered inputs, or an outlier that stretches the bounding box) keeps the
// arrival order, which can change from run to run: the tiles, their origins
// and their choice between the expanded and the direct form can then differ,
// and so can the rounding of the results (within the kernels' accuracy: the
// tile a sample falls in changes only the rounding of its arithmetic).
#include "kernels.cuh"
#include "sort.cuh"

namespace pdmp {

template <int D>
__global__ void k_bbox(const float* __restrict__ x, int64_t N, uint32_t* __restrict__ box) {
  float lo[D], hi[D];
#pragma unroll
  for (int j = 0; j < D; ++j) { lo[j] = INFINITY; hi[j] = -INFINITY; }
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int j = 0; j < D; ++j) {
      float v = x[n * D + j];
      if (v == v) { lo[j] = fminf(lo[j], v); hi[j] = fmaxf(hi[j], v); }
    }
  }
#pragma unroll
  for (int j = 0; j < D; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[j] = fminf(lo[j], __shfl_xor_sync(0xffffffffu, lo[j], o));
      hi[j] = fmaxf(hi[j], __shfl_xor_sync(0xffffffffu, hi[j], o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&box[j], ordered_bits(lo[j]));
      atomicMax(&box[D + j], ordered_bits(hi[j]));
    }
  }
}

template <int D>
__global__ void k_cell_keys(const float* __restrict__ x, int64_t N, const uint32_t* __restrict__ box, int bits,
                            uint32_t* __restrict__ keys, uint32_t* __restrict__ counts) {
  int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const float cells = (float)(1u << bits);
  uint32_t c[D];
#pragma unroll
  for (int j = 0; j < D; ++j) c[j] = cell_coord(x[n * D + j], from_ordered(box[j]), from_ordered(box[D + j]), cells);
  const uint32_t key = hilbert_key<D>(c, bits);
  keys[n] = key;
  atomicAdd(&counts[key], 1u);
}

// exclusive scan of counts[0..C) into offs, in chunks of kScanChunk

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* sh, uint32_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    sh[lane] = wi - w;
    if (lane == 31) sh[32] = wi;
  }
  __syncthreads();
  uint32_t r = inc - v + sh[warp];
  total = sh[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_chunks(const uint32_t* __restrict__ counts, int64_t C,
                                                              uint32_t* __restrict__ offs,
                                                              uint32_t* __restrict__ chunk_tot) {
  __shared__ uint32_t sh[33];
  int64_t base = (int64_t)blockIdx.x * kScanChunk + 2 * threadIdx.x;
  uint32_t a = base < C ? counts[base] : 0u, b = base + 1 < C ? counts[base + 1] : 0u;
  uint32_t tot;
  uint32_t ex = block_exclusive_scan(a + b, sh, tot);
  if (base < C) offs[base] = ex;
  if (base + 1 < C) offs[base + 1] = ex + a;
  if (threadIdx.x == 0) chunk_tot[blockIdx.x] = tot;
}

// single block: exclusive scan of the chunk totals (any count), in place
__global__ void __launch_bounds__(kScanThreads) k_scan_totals(uint32_t* __restrict__ tot, int64_t nchunks) {
  __shared__ uint32_t sh[33];
  uint32_t carry = 0;
  for (int64_t b = 0; b < nchunks; b += kScanThreads) {
    int64_t i = b + threadIdx.x;
    uint32_t v = i < nchunks ? tot[i] : 0u, t;
    uint32_t ex = block_exclusive_scan(v, sh, t);
    if (i < nchunks) tot[i] = ex + carry;
    carry += t;
  }
}

__global__ void k_add_chunk_offsets(uint32_t* __restrict__ offs, int64_t C, const uint32_t* __restrict__ tot,
                                    uint32_t* __restrict__ cursor) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C) return;
  uint32_t v = offs[i] + tot[i / kScanChunk];
  offs[i] = v;
  if (cursor) cursor[i] = v;
}

__global__ void k_scatter(const uint32_t* __restrict__ keys, int64_t N, uint32_t* __restrict__ cursor,
                          int32_t* __restrict__ perm) {
  int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  uint32_t pos = atomicAdd(&cursor[keys[n]], 1u);
  perm[pos] = (int32_t)n;
}

// orders each cell's entries by original index (cells of up to 64 entries;
// larger cells keep the arrival order: see the note on determinism above)
__global__ void k_order_cells(const uint32_t* __restrict__ offs, const uint32_t* __restrict__ counts, int64_t C,
                              int32_t* __restrict__ perm) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  uint32_t n = counts[c];
  if (n < 2 || n > 64) return;
  int32_t* p = perm + offs[c];
  for (uint32_t i = 1; i < n; ++i) {
    int32_t v = p[i];
    uint32_t j = i;
    while (j > 0 && p[j - 1] > v) {
      p[j] = p[j - 1];
      --j;
    }
    p[j] = v;
  }
}

// ------------------------------------------------------------------ host
int sort_bits(int d, int64_t N) {
  // about four samples per cell: 2^(d * bits) ~ N / 4
  double target = N > 4 ? log2((double)N / 4.0) / d : 1.0;
  int bits = (int)floor(target + 0.5);
  int maxb = d == 2 ? 10 : 7;
  return bits < 1 ? 1 : (bits > maxb ? maxb : bits);
}

SortWs sort_layout(void* ws, int d, int64_t N) {
  SortWs s;
  s.bits = sort_bits(d, N);
  s.cells = (int64_t)1 << (d * s.bits);
  s.nchunks = (s.cells + kScanChunk - 1) / kScanChunk;
  char* p = (char*)ws;
  auto take = [&](size_t b) { char* q = p; p += (b + 255) & ~size_t(255); return q; };
  s.box = (uint32_t*)take(sizeof(uint32_t) * 6);
  s.keys = (uint32_t*)take(sizeof(uint32_t) * N);
  s.perm = (int32_t*)take(sizeof(int32_t) * N);
  s.counts = (uint32_t*)take(sizeof(uint32_t) * s.cells);
  s.offs = (uint32_t*)take(sizeof(uint32_t) * s.cells);
  s.cursor = (uint32_t*)take(sizeof(uint32_t) * s.cells);
  s.chunk_tot = (uint32_t*)take(sizeof(uint32_t) * s.nchunks);
  s.bytes = (size_t)(p - (char*)ws);
  return s;
}

size_t sort_workspace(int d, int64_t N) { return sort_layout(nullptr, d, N).bytes; }

cudaError_t spatial_sort(int d, const float* x, int64_t N, const SortWs& s, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(s.box, 0xff, sizeof(uint32_t) * d, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(s.box + d, 0x00, sizeof(uint32_t) * d, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(s.counts, 0, sizeof(uint32_t) * s.cells, st)) != cudaSuccess) return e;
  const unsigned nb = (unsigned)((N + 255) / 256);
  const unsigned bb = nb < 1024 ? nb : 1024;
  if (d == 2) {
    k_bbox<2><<<bb, 256, 0, st>>>(x, N, s.box);
    k_cell_keys<2><<<nb, 256, 0, st>>>(x, N, s.box, s.bits, s.keys, s.counts);
  } else {
    k_bbox<3><<<bb, 256, 0, st>>>(x, N, s.box);
    k_cell_keys<3><<<nb, 256, 0, st>>>(x, N, s.box, s.bits, s.keys, s.counts);
  }
  return sort_by_keys(s.keys, N, s.counts, s.offs, s.cursor, s.chunk_tot, s.cells, s.perm, st);
}

cudaError_t bounding_box(int d, const float* x, int64_t N, uint32_t* box, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(box, 0xff, sizeof(uint32_t) * d, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(box + d, 0x00, sizeof(uint32_t) * d, st)) != cudaSuccess) return e;
  if (N <= 0) return cudaSuccess;
  const unsigned nb = (unsigned)((N + 255) / 256);
  const unsigned bb = nb < 1024 ? nb : 1024;
  if (d == 2)
    k_bbox<2><<<bb, 256, 0, st>>>(x, N, box);
  else
    k_bbox<3><<<bb, 256, 0, st>>>(x, N, box);
  return cudaGetLastError();
}

cudaError_t exclusive_scan_u32(const uint32_t* in, int64_t n, uint32_t* out, uint32_t* chunk_tot, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t nchunks = (n + kScanChunk - 1) / kScanChunk;
  k_scan_chunks<<<(unsigned)nchunks, kScanThreads, 0, st>>>(in, n, out, chunk_tot);
  k_scan_totals<<<1, kScanThreads, 0, st>>>(chunk_tot, nchunks);
  k_add_chunk_offsets<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n, chunk_tot, nullptr);
  return cudaGetLastError();
}

cudaError_t sort_by_keys(const uint32_t* keys, int64_t N, const uint32_t* counts, uint32_t* offs, uint32_t* cursor,
                         uint32_t* chunk_tot, int64_t cells, int32_t* perm, cudaStream_t st) {
  const int64_t nchunks = (cells + kScanChunk - 1) / kScanChunk;
  k_scan_chunks<<<(unsigned)nchunks, kScanThreads, 0, st>>>(counts, cells, offs, chunk_tot);
  k_scan_totals<<<1, kScanThreads, 0, st>>>(chunk_tot, nchunks);
  k_add_chunk_offsets<<<(unsigned)((cells + 255) / 256), 256, 0, st>>>(offs, cells, chunk_tot, cursor);
  if (N > 0) k_scatter<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(keys, N, cursor, perm);
  k_order_cells<<<(unsigned)((cells + 255) / 256), 256, 0, st>>>(offs, counts, cells, perm);
  return cudaGetLastError();
}

}  // namespace pdmp
