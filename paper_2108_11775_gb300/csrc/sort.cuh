// Spatial sort of samples (see sort.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pdmp {

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
cudaError_t spatial_sort(int d, const float* x, int64_t N, const SortWs& s, cudaStream_t st);

}  // namespace pdmp
