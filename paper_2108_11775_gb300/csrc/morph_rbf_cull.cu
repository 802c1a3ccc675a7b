// Spatially culled RBF morph (d = 2, 3).  The same T Euler steps of Eq. (1) as
// the dense fast kernel, but each tile, at each step, sums only over centres
// that can lie within r_cut of one of its samples: the centres are sorted by
// the cells of a uniform grid, and for every grid row (fixed y, z cells) that
// meets the tile's bounding box grown by r_cut the tile visits the run of
// cells whose x-extent meets the disc (ball) section at that row.  A dropped
// centre is farther than r_cut from every sample of the tile, so with
// W = sum_m |w_m| and r_cut >= 1/sqrt(2 gamma) the dropped part of s is at most
// W exp(-gamma r_cut^2) and that of grad s at most W 2 gamma r_cut
// exp(-gamma r_cut^2) (pdmp_cull_radius picks r_cut from a bound eps on both).
#include "fast_tile.cuh"
#include "kernels.cuh"
#include "sort.cuh"

namespace pdmp {

constexpr int kCullRows = 64;                    // grid rows per batch (2 per lane)
constexpr int kCullRowWords = 2 * kCullRows + 2; // per warp: run starts, run offsets (+ total)

struct CullGrid {
  float lo[3], h[3], inv_h[3];
  int g[3];
  float r, margin;
};

template <int D>
__host__ __device__ constexpr int cull_cells_per_radius() { return D == 2 ? 8 : 4; }
template <int D>
__host__ __device__ constexpr int cull_max_cells_per_axis() { return D == 2 ? 512 : 64; }
template <int D>
__host__ __device__ constexpr int64_t cull_cell_capacity() {
  return D == 2 ? (int64_t)512 * 512 : (int64_t)64 * 64 * 64;
}

template <int D, int K>
__host__ __device__ constexpr size_t cull_smem_bytes() {
  return fast_smem_bytes<D, 4, K>() + (size_t)4 * kCullRowWords * sizeof(uint32_t);
}

// cell index of v along axis j (values outside the grid, and NaN, clamp to it)
__device__ __forceinline__ int cull_cell(const CullGrid& g, int j, float v) {
  const float q = fminf(fmaxf((v - g.lo[j]) * g.inv_h[j], 0.0f), (float)(g.g[j] - 1));
  return (int)q;
}

// distance from the interval [lo, hi] to the band [blo, bhi] (0 if they meet)
__device__ __forceinline__ float band_gap(float lo, float hi, float blo, float bhi) {
  return fmaxf(0.0f, fmaxf(blo - hi, lo - bhi));
}

// grid over the centres' bounding box: cells of side >= r / cells_per_radius
// and at most max_cells per axis
template <int D>
__global__ void k_cull_grid(const uint32_t* __restrict__ box, float r, CullGrid* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  CullGrid g;
  float scale = r;
  for (int j = 0; j < 3; ++j) {
    float lo = 0.0f, hi = 0.0f;
    if (j < D) {
      lo = from_ordered(box[j]);
      hi = from_ordered(box[D + j]);
      if (!(hi >= lo)) lo = hi = 0.0f;   // no finite centre on this axis
    }
    const float ext = hi - lo;
    float h = fmaxf(r / (float)cull_cells_per_radius<D>(), ext / (float)(cull_max_cells_per_axis<D>() - 1));
    h = fmaxf(h, 1e-30f);
    g.lo[j] = lo;
    g.h[j] = h;
    g.inv_h[j] = 1.0f / h;
    g.g[j] = j < D ? min((int)(ext / h) + 1, cull_max_cells_per_axis<D>()) : 1;
    scale = fmaxf(scale, fmaxf(fabsf(lo), fabsf(hi)));
  }
  g.r = r;
  g.margin = 1e-4f * (scale + r);   // covers the rounding of cell edges and of the disc section
  *out = g;
}

template <int D>
__global__ void k_centre_cells(const float* __restrict__ centres, int64_t M, const CullGrid* __restrict__ grid,
                               uint32_t* __restrict__ keys, uint32_t* __restrict__ counts) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const CullGrid g = *grid;
  int c[3] = {0, 0, 0};
#pragma unroll
  for (int j = 0; j < D; ++j) c[j] = cull_cell(g, j, centres[m * D + j]);
  const uint32_t key = (uint32_t)(c[0] + g.g[0] * (c[1] + g.g[1] * c[2]));
  keys[m] = key;
  atomicAdd(&counts[key], 1u);
}

// table entries in cell order: entry i is the record of centre perm[i]
template <int D>
__global__ void k_rbf_table_perm(const float* __restrict__ centres, const float* __restrict__ w,
                                 const int32_t* __restrict__ perm, int64_t M, float4* __restrict__ tab) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const int64_t m = perm[i];
  const float wm = w[m];
  const float lw = wm != 0.0f ? log2f(fabsf(wm)) : -INFINITY;
  const float sg = wm > 0.0f ? 1.0f : (wm < 0.0f ? -1.0f : 0.0f);
  if (D == 2) {
    tab[i] = make_float4(centres[m * 2], centres[m * 2 + 1], lw, sg);
  } else {
    tab[2 * i] = make_float4(centres[m * 3], centres[m * 3 + 1], centres[m * 3 + 2], lw);
    tab[2 * i + 1] = make_float4(sg, 0.0f, 0.0f, 0.0f);
  }
}

// Copies the table entries of virtual positions [v0, v0 + kWarpStage) of the
// batch's concatenated cell runs (run r starts at table entry rs[r] and at
// virtual position ro[r]) into the warp's raw buffer.
template <int D>
__device__ __forceinline__ void stage_prefetch_runs(const float4* __restrict__ tab, const uint32_t* rs,
                                                    const uint32_t* ro, int nr, int64_t v0, int64_t vend,
                                                    float4* raw, int lane) {
  constexpr int KT = FastRec<D>::kTab;
  for (int i = lane; i < kWarpStage; i += 32) {
    const int64_t v = v0 + i;
    if (v < vend) {
      int lo = 0, hi = nr - 1;   // the last run with ro[run] <= v
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int64_t)ro[mid] <= v)
          lo = mid;
        else
          hi = mid - 1;
      }
      const int64_t m = (int64_t)rs[lo] + (v - (int64_t)ro[lo]);
#pragma unroll
      for (int q = 0; q < KT; ++q) cp_async16(raw + i * KT + q, tab + KT * m + q);
    }
  }
  cp_async_commit();
}

template <int D, int W, int K>
__device__ __forceinline__ void cull_tile(const TileArgs& a, const CullGrid& g, const uint32_t* __restrict__ start,
                                          int64_t p0, int64_t p_end, unsigned char* smem,
                                          unsigned long long* work) {
  constexpr int RP = FastRec<D>::kPairs;
  constexpr int P = K / 2;
  constexpr int KT = FastRec<D>::kTab;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64* wbuf = reinterpret_cast<u64*>(smem) + (size_t)warp * 2 * kWarpStage * RP;
  float4* red = reinterpret_cast<float4*>(smem);
  float4* wraw = reinterpret_cast<float4*>(smem + fast_region0_bytes<D, W, K>()) + (size_t)warp * kWarpStage * KT;
  uint32_t* rs = reinterpret_cast<uint32_t*>(smem + fast_smem_bytes<D, W, K>()) + (size_t)warp * kCullRowWords;
  uint32_t* ro = rs + kCullRows;
  const float4* __restrict__ tab = a.tab;
  const float gl2e = a.gamma * kLog2e;
  const float r = g.r + g.margin;

  float x[K][D];
  bool act[K];
  tile_load<D, K>(a, p0, p_end, lane, x, act);
  unsigned nact = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) nact += __popc(__ballot_sync(0xffffffffu, act[k]));
  unsigned long long visited = 0;

  for (int t = 0; t < a.T; ++t) {
    float lo[D], hi[D], o[D];
    const bool expanded = tile_frame<D, K>(x, act, gl2e, lo, hi, o);
    u64 U[P][D], S[P], G[P][D];
#pragma unroll
    for (int i = 0; i < P; ++i) {
#pragma unroll
      for (int j = 0; j < D; ++j) {
        U[i][j] = pk(x[2 * i][j] - o[j], x[2 * i + 1][j] - o[j]);
        G[i][j] = 0ull;
      }
      S[i] = 0ull;
    }
    // grid rows (y, z cells) that meet the box grown by r
    const int y0 = cull_cell(g, 1, lo[1] - r), y1 = cull_cell(g, 1, hi[1] + r);
    const int z0 = D == 3 ? cull_cell(g, 2, lo[D - 1] - r) : 0, z1 = D == 3 ? cull_cell(g, 2, hi[D - 1] + r) : 0;
    const int ny = y1 - y0 + 1;
    const int nrows = ny * (z1 - z0 + 1);
    for (int rb = 0; rb < nrows; rb += kCullRows) {
      uint32_t beg[2], cnt[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int idx = rb + lane + 32 * q;
        beg[q] = 0;
        cnt[q] = 0;
        if (idx < nrows) {
          const int cy = y0 + idx % ny, cz = z0 + idx / ny;
          float rem = r * r;
          const float dy = band_gap(lo[1], hi[1], g.lo[1] + (float)cy * g.h[1] - g.margin,
                                    g.lo[1] + (float)(cy + 1) * g.h[1] + g.margin);
          rem -= dy * dy;
          if (D == 3) {
            const float dz = band_gap(lo[D - 1], hi[D - 1], g.lo[2] + (float)cz * g.h[2] - g.margin,
                                      g.lo[2] + (float)(cz + 1) * g.h[2] + g.margin);
            rem -= dz * dz;
          }
          if (rem >= 0.0f) {
            const float wx = sqrtf(rem) + g.margin;
            const int x0 = cull_cell(g, 0, lo[0] - wx), x1 = cull_cell(g, 0, hi[0] + wx);
            const int64_t base = ((int64_t)cz * g.g[1] + cy) * g.g[0];
            beg[q] = start[base + x0];
            cnt[q] = start[base + x1 + 1] - beg[q];
          }
        }
      }
      // offsets of the runs in the batch's concatenation (inclusive scans)
      uint32_t inc0 = cnt[0], inc1 = cnt[1];
#pragma unroll
      for (int s = 1; s < 32; s <<= 1) {
        const uint32_t u0 = __shfl_up_sync(0xffffffffu, inc0, s), u1 = __shfl_up_sync(0xffffffffu, inc1, s);
        if (lane >= s) {
          inc0 += u0;
          inc1 += u1;
        }
      }
      const uint32_t tot0 = __shfl_sync(0xffffffffu, inc0, 31);
      inc1 += tot0;
      const uint32_t Mt = __shfl_sync(0xffffffffu, inc1, 31);
      rs[lane] = beg[0];
      rs[lane + 32] = beg[1];
      ro[lane] = inc0 - cnt[0];
      ro[lane + 32] = inc1 - cnt[1];
      __syncwarp();
      visited += Mt;
      const int nr = min(kCullRows, nrows - rb);
      const int64_t Mw = (((int64_t)Mt + W - 1) / W + kWarpStage - 1) / kWarpStage * kWarpStage;
      const int64_t vbeg = (int64_t)warp * Mw;
      const int64_t vend = min64((int64_t)Mt, vbeg + Mw);
      const int nstage = vend > vbeg ? (int)((vend - vbeg + kWarpStage - 1) / kWarpStage) : 0;
      if (nstage > 0) {
        stage_prefetch_runs<D>(tab, rs, ro, nr, vbeg, vend, wraw, lane);
        stage_build<D>(vend, vbeg, expanded, o, gl2e, wraw, wbuf, lane);
        __syncwarp();
        for (int st = 0; st < nstage; ++st) {
          const int64_t vn = vbeg + (int64_t)(st + 1) * kWarpStage;
          if (st + 1 < nstage) stage_prefetch_runs<D>(tab, rs, ro, nr, vn, vend, wraw, lane);
          stage_accumulate<D, P>(wbuf + (size_t)(st & 1) * kWarpStage * RP, expanded, gl2e, U, S, G);
          if (st + 1 < nstage)
            stage_build<D>(vend, vn, expanded, o, gl2e, wraw, wbuf + (size_t)((st + 1) & 1) * kWarpStage * RP, lane);
          __syncwarp();
        }
      }
      __syncwarp();   // every lane is done with the run table before the next batch rewrites it
    }
    tile_finish_step<D, W, K, false>(a, t, p0, act, x, o, expanded, S, G, red, warp, lane);
  }
  if (work != nullptr && threadIdx.x == 0) atomicAdd(work, visited * nact);
  tile_store<D, K, false>(a, p0, act, x, warp, lane);
}

template <int D, int K>
__global__ void __launch_bounds__(Shape<4, K>::kThreads, Shape<4, K>::kMinBlocks)
k_morph_rbf_cull(TileArgs a, const CullGrid* __restrict__ grid, const uint32_t* __restrict__ start,
                 unsigned long long* work) {
  extern __shared__ __align__(16) unsigned char smem[];
  const CullGrid g = *grid;
  const int64_t p0 = (int64_t)blockIdx.x * Shape<4, K>::kTile;
  cull_tile<D, 4, K>(a, g, start, p0, a.N, smem, work);
}

// Samples per lane: 8 (256-sample tiles, 4 blocks per SM), and 4 (128-sample
// tiles) for launches of fewer than two waves of the larger ones.
template <int D, int K>
static cudaError_t launch_cull_shape(const TileArgs& a, const CullGrid* grid, const uint32_t* offs,
                                     unsigned long long* work, cudaStream_t st) {
  constexpr size_t smem = cull_smem_bytes<D, K>();
  cudaError_t e =
      cudaFuncSetAttribute(k_morph_rbf_cull<D, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((a.N + Shape<4, K>::kTile - 1) / Shape<4, K>::kTile);
  k_morph_rbf_cull<D, K><<<blocks, Shape<4, K>::kThreads, smem, st>>>(a, grid, offs, work);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ host
struct CullWs {
  CullGrid* grid;
  uint32_t* cbox;
  uint32_t* keys;
  int32_t* cperm;
  uint32_t *counts, *offs, *cursor, *chunk_tot;
  float4* tab;
  void* sort;
  size_t bytes;
};

static CullWs cull_layout(void* ws, int d, int64_t M, int64_t N) {
  CullWs s;
  const int64_t cells = (d == 2 ? cull_cell_capacity<2>() : cull_cell_capacity<3>()) + 1;
  const int64_t nchunks = (cells + kScanChunk - 1) / kScanChunk;
  char* p = (char*)ws;
  auto take = [&](size_t b) { char* q = p; p += (b + 255) & ~size_t(255); return q; };
  s.grid = (CullGrid*)take(sizeof(CullGrid));
  s.cbox = (uint32_t*)take(sizeof(uint32_t) * 6);
  s.keys = (uint32_t*)take(sizeof(uint32_t) * M);
  s.cperm = (int32_t*)take(sizeof(int32_t) * M);
  s.counts = (uint32_t*)take(sizeof(uint32_t) * cells);
  s.offs = (uint32_t*)take(sizeof(uint32_t) * cells);
  s.cursor = (uint32_t*)take(sizeof(uint32_t) * cells);
  s.chunk_tot = (uint32_t*)take(sizeof(uint32_t) * nchunks);
  s.tab = (float4*)take((size_t)M * 16 * (d == 2 ? 1 : 2));
  s.sort = take(sort_workspace(d, N));
  s.bytes = (size_t)(p - (char*)ws);
  return s;
}

size_t morph_rbf_cull_workspace(int d, int64_t M, int64_t N) { return cull_layout(nullptr, d, M, N).bytes; }

template <int D>
static cudaError_t launch_cull(const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float r_cut,
                               float* xT, float* ckpt, int k, void* ws, unsigned long long* work, cudaStream_t st,
                               float* s_out, float* g_out) {
  const CullWs c = cull_layout(ws, D, fa.M, N);
  const int64_t cells = cull_cell_capacity<D>() + 1;
  cudaError_t e;
  if ((e = bounding_box(D, fa.centres, fa.M, c.cbox, st)) != cudaSuccess) return e;
  k_cull_grid<D><<<1, 32, 0, st>>>(c.cbox, r_cut, c.grid);
  if ((e = cudaMemsetAsync(c.counts, 0, sizeof(uint32_t) * cells, st)) != cudaSuccess) return e;
  const unsigned mb = (unsigned)((fa.M + 255) / 256);
  k_centre_cells<D><<<mb, 256, 0, st>>>(fa.centres, fa.M, c.grid, c.keys, c.counts);
  if ((e = sort_by_keys(c.keys, fa.M, c.counts, c.offs, c.cursor, c.chunk_tot, cells, c.cperm, st)) != cudaSuccess)
    return e;
  k_rbf_table_perm<D><<<mb, 256, 0, st>>>(fa.centres, fa.w, c.cperm, fa.M, c.tab);
  const SortWs sw = sort_layout(c.sort, D, N);
  if ((e = spatial_sort(D, x0, N, sw, st)) != cudaSuccess) return e;
  TileArgs a{};
  a.tab = c.tab;
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
  a.s_out = s_out;
  a.g_out = g_out;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess || sms < 1)
    sms = 152;
  const int64_t tiles = (N + Shape<4, 8>::kTile - 1) / Shape<4, 8>::kTile;
  if (tiles < 2 * (int64_t)Shape<4, 8>::kMinBlocks * sms) return launch_cull_shape<D, 4>(a, c.grid, c.offs, work, st);
  return launch_cull_shape<D, 8>(a, c.grid, c.offs, work, st);
}

cudaError_t morph_rbf_cull(int d, const FieldArgs& fa, const float* x0, int64_t N, int T, float eta, float r_cut,
                           float* xT, float* ckpt, int k, void* ws, unsigned long long* work, cudaStream_t st,
                           float* s_out, float* g_out) {
  if (d == 2) return launch_cull<2>(fa, x0, N, T, eta, r_cut, xT, ckpt, k, ws, work, st, s_out, g_out);
  if (d == 3) return launch_cull<3>(fa, x0, N, T, eta, r_cut, xT, ckpt, k, ws, work, st, s_out, g_out);
  return cudaErrorInvalidValue;
}

// sum_m |w_m| in FP64 (one block, fixed order)
__global__ void __launch_bounds__(1024) k_abs_sum(const float* __restrict__ w, int64_t M, double* __restrict__ out) {
  __shared__ double sh[1024];
  double acc = 0.0;
  for (int64_t m = threadIdx.x; m < M; m += 1024) acc += fabs((double)w[m]);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

cudaError_t abs_weight_sum(const float* w, int64_t M, double* out, cudaStream_t st) {
  k_abs_sum<<<1, 1024, 0, st>>>(w, M, out);
  return cudaGetLastError();
}

}  // namespace pdmp
