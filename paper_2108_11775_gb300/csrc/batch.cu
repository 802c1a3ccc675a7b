// Batched morph of many environments (fields with their own samples, d = 2
// or 3, uneven M and N) in one persistent launch.
//
// Preparation (host, once per set of environments): the environment table and
// a list of (environment, tile) work units ordered longest first -- cost
// M_e * T_e per tile -- are copied into the caller's workspace.
// Run (launch-only, so a CUDA graph can capture it): every environment's
// centre table, one spatial sort over all environments' samples (cell keys
// are environment-major, so each environment's samples stay contiguous in
// sorted order), then one persistent kernel whose blocks claim work units from
// an atomic counter and run them with the same per-tile code as the
// single-field fast path.  Claiming is a single atomicAdd: no block ever
// waits on another.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "fast_tile.cuh"
#include "kernels.cuh"
#include "sort.cuh"

namespace pdmp {

struct BatchEnv {        // device table entry (64-bit aligned)
  const float* centres;
  const float* w;
  const float* x0;
  float* xT;
  float4* tab;
  int64_t N, M;
  int64_t sample_base;   // first global sample index (= first sorted position)
  int64_t centre_base;   // first global centre index
  int64_t cell_base;     // first global cell key
  int32_t d, T, bits, pad;
  float gamma, bias, eta, pad2;
};

struct BatchUnit {
  int32_t env;
  int32_t tile;
};

// ---------------------------------------------------------------- variants
// (warps per block, samples per lane)
// variant 0 is the single-field launch's shape (FastShape)
constexpr int kBatchVariants = 5;
static const int kVariantW[kBatchVariants] = {4, 2, 4, 8, 4};
static const int kVariantK[kBatchVariants] = {10, 8, 4, 8, 8};

static int variant_tile(int v) { return 32 * kVariantK[v]; }

// index of the environment whose [base[e], base[e+1]) holds g (base has n+1 entries)
__device__ __forceinline__ int find_env(const int64_t* __restrict__ base, int n, int64_t g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (base[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_batch_tables(const BatchEnv* __restrict__ envs, const int64_t* __restrict__ cbase, int n_envs,
                               int64_t total_M) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total_M) return;
  const int e = find_env(cbase, n_envs, g);
  const BatchEnv& E = envs[e];
  const int64_t m = g - E.centre_base;
  const float wm = E.w[m];
  const float lw = wm != 0.0f ? log2f(fabsf(wm)) : -INFINITY;
  const float sg = wm > 0.0f ? 1.0f : (wm < 0.0f ? -1.0f : 0.0f);
  if (E.d == 2) {
    E.tab[m] = make_float4(E.centres[m * 2], E.centres[m * 2 + 1], lw, sg);
  } else {
    E.tab[2 * m] = make_float4(E.centres[m * 3], E.centres[m * 3 + 1], E.centres[m * 3 + 2], lw);
    E.tab[2 * m + 1] = make_float4(sg, 0.0f, 0.0f, 0.0f);
  }
}

// per environment: minima to the largest ordered encoding, maxima to the smallest
__global__ void k_batch_init_boxes(uint32_t* __restrict__ boxes, int n_envs) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_envs) return;
  for (int j = 0; j < 3; ++j) {
    boxes[6 * e + j] = 0xffffffffu;
    boxes[6 * e + 3 + j] = 0u;
  }
}

// bounding box of every environment's samples; a warp whose lanes all belong
// to one environment reduces before its atomics
__global__ void k_batch_bbox(const BatchEnv* __restrict__ envs, const int64_t* __restrict__ sbase, int n_envs,
                             int64_t total_N, uint32_t* __restrict__ boxes) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = g < total_N;
  const int e = valid ? find_env(sbase, n_envs, g) : -1;
  const int e0 = __shfl_sync(0xffffffffu, e, 0);
  const bool uniform = __all_sync(0xffffffffu, e == e0) && e0 >= 0;
  if (uniform) {
    const BatchEnv& E = envs[e0];
    const int64_t n = g - E.sample_base;
    for (int j = 0; j < E.d; ++j) {
      const float v = E.x0[n * E.d + j];
      float lo = v == v ? v : INFINITY, hi = v == v ? v : -INFINITY;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      }
      if ((threadIdx.x & 31) == 0) {
        atomicMin(&boxes[6 * e0 + j], ordered_bits(lo));
        atomicMax(&boxes[6 * e0 + 3 + j], ordered_bits(hi));
      }
    }
  } else if (valid) {
    const BatchEnv& E = envs[e];
    const int64_t n = g - E.sample_base;
    for (int j = 0; j < E.d; ++j) {
      const float v = E.x0[n * E.d + j];
      if (v == v) {
        atomicMin(&boxes[6 * e + j], ordered_bits(v));
        atomicMax(&boxes[6 * e + 3 + j], ordered_bits(v));
      }
    }
  }
}

__global__ void k_batch_keys(const BatchEnv* __restrict__ envs, const int64_t* __restrict__ sbase, int n_envs,
                             int64_t total_N, const uint32_t* __restrict__ boxes, uint32_t* __restrict__ keys,
                             uint32_t* __restrict__ counts) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total_N) return;
  const int e = find_env(sbase, n_envs, g);
  const BatchEnv& E = envs[e];
  const int64_t n = g - E.sample_base;
  const float cells = (float)(1u << E.bits);
  const uint32_t* b = boxes + 6 * e;
  const float* x = E.x0 + n * E.d;
  // the Hilbert index is computed in a branch per dimension (one code path
  // with a dimension chosen at run time inside the loop assembled wrong keys)
  uint32_t key;
  if (E.d == 2) {
    uint32_t c[2] = {cell_coord(x[0], from_ordered(b[0]), from_ordered(b[3]), cells),
                     cell_coord(x[1], from_ordered(b[1]), from_ordered(b[4]), cells)};
    key = hilbert_key<2>(c, E.bits);
  } else {
    uint32_t c[3] = {cell_coord(x[0], from_ordered(b[0]), from_ordered(b[3]), cells),
                     cell_coord(x[1], from_ordered(b[1]), from_ordered(b[4]), cells),
                     cell_coord(x[2], from_ordered(b[2]), from_ordered(b[5]), cells)};
    key = hilbert_key<3>(c, E.bits);
  }
  key += (uint32_t)E.cell_base;
  keys[g] = key;
  atomicAdd(&counts[key], 1u);
}

template <int W, int K>
__global__ void __launch_bounds__(32 * W, Shape<W, K>::kMinBlocks)
k_morph_batched(const BatchEnv* __restrict__ envs, const BatchUnit* __restrict__ units, int64_t n_units,
                const int32_t* __restrict__ perm, unsigned int* __restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long s_unit;
  constexpr int kTile = Shape<W, K>::kTile;
  for (;;) {
    if (threadIdx.x == 0) s_unit = (long long)atomicAdd(counter, 1u);
    __syncthreads();
    const long long u = s_unit;
    __syncthreads();
    if (u >= n_units) break;
    const BatchUnit un = units[u];
    const BatchEnv& E = envs[un.env];
    TileArgs a;
    a.tab = E.tab;
    a.M = E.M;
    a.gamma = E.gamma;
    a.bias = E.bias;
    a.eta = E.eta;
    a.T = E.T;
    a.x0 = E.x0;
    a.perm = perm;
    a.perm_base = E.sample_base;
    a.N = E.N;
    a.xT = E.xT;
    a.ckpt = nullptr;
    a.kck = 1;
    a.traj = nullptr;
    a.steps = nullptr;
    a.s_out = nullptr;
    a.g_out = nullptr;
    const int64_t p0 = E.sample_base + (int64_t)un.tile * kTile;
    const int64_t pend = E.sample_base + E.N;
    if (E.d == 2)
      fast_tile<2, W, K, false, true>(a, p0, pend, smem);
    else
      fast_tile<3, W, K, false, true>(a, p0, pend, smem);
  }
}

template <int W, int K>
static size_t batched_smem() {
  const size_t a = fast_smem_bytes<2, W, K>(), b = fast_smem_bytes<3, W, K>();
  return a > b ? a : b;
}

// ---------------------------------------------------------------- layout
struct BatchLayout {
  size_t off_counter, off_envs, off_sbase, off_cbase, off_units, off_boxes, off_tabs, off_keys, off_perm, off_counts,
      off_offs, off_cursor, off_chunks, bytes;
  std::vector<size_t> tab_off;
  int64_t n_units, total_N, total_M, total_cells, nchunks;
};

static size_t al(size_t b) { return (b + 255) & ~size_t(255); }

static BatchLayout batch_layout(const pdmp_env* envs, int n, int variant) {
  BatchLayout L;
  const int tile = variant_tile(variant);
  L.n_units = 0;
  L.total_N = 0;
  L.total_M = 0;
  L.total_cells = 0;
  for (int e = 0; e < n; ++e) {
    L.n_units += (envs[e].N + tile - 1) / tile;
    L.total_N += envs[e].N;
    L.total_M += envs[e].field.M;
    L.total_cells += (int64_t)1 << (envs[e].field.d * sort_bits(envs[e].field.d, envs[e].N));
  }
  L.nchunks = (L.total_cells + kScanChunk - 1) / kScanChunk;
  size_t p = 0;
  auto take = [&](size_t b) { size_t q = p; p += al(b); return q; };
  L.off_counter = take(16);
  L.off_envs = take(sizeof(BatchEnv) * n);
  L.off_sbase = take(sizeof(int64_t) * (n + 1));
  L.off_cbase = take(sizeof(int64_t) * (n + 1));
  L.off_units = take(sizeof(BatchUnit) * L.n_units);
  L.off_boxes = take(sizeof(uint32_t) * 6 * n);
  L.tab_off.resize(n);
  L.off_tabs = p;
  for (int e = 0; e < n; ++e) L.tab_off[e] = take((size_t)envs[e].field.M * 16 * (envs[e].field.d == 2 ? 1 : 2));
  L.off_keys = take(sizeof(uint32_t) * L.total_N);
  L.off_perm = take(sizeof(int32_t) * L.total_N);
  L.off_counts = take(sizeof(uint32_t) * L.total_cells);
  L.off_offs = take(sizeof(uint32_t) * L.total_cells);
  L.off_cursor = take(sizeof(uint32_t) * L.total_cells);
  L.off_chunks = take(sizeof(uint32_t) * L.nchunks);
  L.bytes = p;
  return L;
}

int batch_variants() { return kBatchVariants; }

size_t batch_workspace(const pdmp_env* envs, int n, int variant) { return batch_layout(envs, n, variant).bytes; }

cudaError_t batch_prepare(const pdmp_env* envs, int n, int variant, void* ws, pdmp_batch_plan* plan,
                          cudaStream_t st) {
  BatchLayout L = batch_layout(envs, n, variant);
  const int tile = variant_tile(variant);
  char* base = (char*)ws;
  std::vector<BatchEnv> tab(n);
  std::vector<int64_t> sb(n + 1), cb(n + 1);
  int64_t s = 0, c = 0, cell = 0;
  for (int e = 0; e < n; ++e) {
    const pdmp_env& E = envs[e];
    BatchEnv& B = tab[e];
    memset(&B, 0, sizeof(B));
    B.centres = E.field.centres;
    B.w = E.field.w;
    B.x0 = E.x0;
    B.xT = E.xT;
    B.tab = (float4*)(base + L.tab_off[e]);
    B.N = E.N;
    B.M = E.field.M;
    B.sample_base = s;
    B.centre_base = c;
    B.cell_base = cell;
    B.d = E.field.d;
    B.T = E.T;
    B.bits = sort_bits(E.field.d, E.N);
    B.gamma = E.field.gamma;
    B.bias = E.field.bias;
    B.eta = E.eta;
    sb[e] = s;
    cb[e] = c;
    s += E.N;
    c += E.field.M;
    cell += (int64_t)1 << (B.d * B.bits);
  }
  sb[n] = s;
  cb[n] = c;
  // work units, longest first (cost M T per tile), then by environment and tile
  std::vector<BatchUnit> units;
  units.reserve(L.n_units);
  for (int e = 0; e < n; ++e)
    for (int64_t t = 0; t * tile < envs[e].N; ++t) units.push_back(BatchUnit{e, (int32_t)t});
  std::stable_sort(units.begin(), units.end(), [&](const BatchUnit& a, const BatchUnit& b) {
    const double ca = (double)envs[a.env].field.M * envs[a.env].T, cb2 = (double)envs[b.env].field.M * envs[b.env].T;
    return ca > cb2;
  });
  cudaError_t e;
  if ((e = cudaMemcpyAsync(base + L.off_envs, tab.data(), sizeof(BatchEnv) * n, cudaMemcpyHostToDevice, st)))
    return e;
  if ((e = cudaMemcpyAsync(base + L.off_sbase, sb.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st)))
    return e;
  if ((e = cudaMemcpyAsync(base + L.off_cbase, cb.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st)))
    return e;
  if (!units.empty() &&
      (e = cudaMemcpyAsync(base + L.off_units, units.data(), sizeof(BatchUnit) * units.size(),
                           cudaMemcpyHostToDevice, st)))
    return e;
  if ((e = cudaStreamSynchronize(st))) return e;

  // kernel attributes and the persistent grid (outside any capture)
  int dev = 0, sms = 1, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  size_t smem = 0;
  int block = 32 * kVariantW[variant];
#define PDMP_VARIANT(V, W_, K_)                                                                                      \
  if (variant == V) {                                                                                                \
    smem = batched_smem<W_, K_>();                                                                                   \
    if ((e = cudaFuncSetAttribute(k_morph_batched<W_, K_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) \
      return e;                                                                                                      \
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_morph_batched<W_, K_>, block, smem))) return e; \
  }
  PDMP_VARIANT(0, 4, 10) PDMP_VARIANT(1, 2, 8) PDMP_VARIANT(2, 4, 4) PDMP_VARIANT(3, 8, 8) PDMP_VARIANT(4, 4, 8)
#undef PDMP_VARIANT
  if (per_sm < 1) per_sm = 1;
  memset(plan, 0, sizeof(*plan));
  plan->n_envs = n;
  plan->variant = variant;
  plan->block = block;
  plan->grid = (int32_t)std::min<int64_t>((int64_t)sms * per_sm, std::max<int64_t>(L.n_units, 1));
  plan->smem_bytes = smem;
  plan->n_units = L.n_units;
  plan->total_N = L.total_N;
  plan->total_M = L.total_M;
  plan->total_cells = L.total_cells;
  plan->ws_bytes = L.bytes;
  plan->work = 0.0;
  for (int k = 0; k < n; ++k) plan->work += (double)envs[k].N * envs[k].field.M * envs[k].T;
  plan->off[0] = L.off_counter;
  plan->off[1] = L.off_envs;
  plan->off[2] = L.off_sbase;
  plan->off[3] = L.off_cbase;
  plan->off[4] = L.off_units;
  plan->off[5] = L.off_boxes;
  plan->off[6] = L.off_keys;
  plan->off[7] = L.off_perm;
  plan->off[8] = L.off_counts;
  plan->off[9] = L.off_offs;
  plan->off[10] = L.off_cursor;
  plan->off[11] = L.off_chunks;
  plan->nchunks = L.nchunks;
  return cudaSuccess;
}

cudaError_t batch_run(const pdmp_batch_plan* P, void* ws, cudaStream_t st) {
  char* base = (char*)ws;
  auto at = [&](int i) { return base + P->off[i]; };
  const BatchEnv* envs = (const BatchEnv*)at(1);
  const int64_t* sbase = (const int64_t*)at(2);
  const int64_t* cbase = (const int64_t*)at(3);
  const BatchUnit* units = (const BatchUnit*)at(4);
  uint32_t* boxes = (uint32_t*)at(5);
  uint32_t* keys = (uint32_t*)at(6);
  int32_t* perm = (int32_t*)at(7);
  uint32_t* counts = (uint32_t*)at(8);
  uint32_t* offs = (uint32_t*)at(9);
  uint32_t* cursor = (uint32_t*)at(10);
  uint32_t* chunks = (uint32_t*)at(11);
  unsigned int* counter = (unsigned int*)at(0);
  const int n = P->n_envs;
  cudaError_t e;
  if ((e = cudaMemsetAsync(counter, 0, 16, st))) return e;
  if (P->total_M > 0)
    k_batch_tables<<<(unsigned)((P->total_M + 255) / 256), 256, 0, st>>>(envs, cbase, n, P->total_M);
  if (P->total_N > 0) {
    k_batch_init_boxes<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(boxes, n);
    if ((e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * P->total_cells, st))) return e;
    const unsigned nb = (unsigned)((P->total_N + 255) / 256);
    k_batch_bbox<<<nb, 256, 0, st>>>(envs, sbase, n, P->total_N, boxes);
    k_batch_keys<<<nb, 256, 0, st>>>(envs, sbase, n, P->total_N, boxes, keys, counts);
    if ((e = sort_by_keys(keys, P->total_N, counts, offs, cursor, chunks, P->total_cells, perm, st))) return e;
  }
  if (P->n_units == 0) return cudaGetLastError();
#define PDMP_VARIANT(V, W_, K_)                                                                             \
  if (P->variant == V)                                                                                      \
    k_morph_batched<W_, K_><<<(unsigned)P->grid, 32 * W_, P->smem_bytes, st>>>(envs, units, P->n_units, perm, \
                                                                               counter);
  PDMP_VARIANT(0, 4, 10) PDMP_VARIANT(1, 2, 8) PDMP_VARIANT(2, 4, 4) PDMP_VARIANT(3, 8, 8) PDMP_VARIANT(4, 4, 8)
#undef PDMP_VARIANT
  return cudaGetLastError();
}

}  // namespace pdmp
