/* A C program on the library's boundary alone (no Python, no PyTorch): it
 * builds a small 2-D RBF occupancy field, asks for a certified Lipschitz
 * bound, morphs uniform samples with Eq. (1) through pdmp_morph on the fast
 * path, and prints a checksum and the largest displacement.
 *
 *   nvcc -o morph_c examples/morph_c.c -I include -L paper_2108_11775_gb300/_build -lpdmp \
 *        -Xlinker -rpath=$PWD/paper_2108_11775_gb300/_build
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "pdmp.h"

static unsigned long long state = 0x9E3779B97F4A7C15ull;
static float uniform01(void) {
  state ^= state << 13;
  state ^= state >> 7;
  state ^= state << 17;
  return (float)((state >> 40) * (1.0 / 16777216.0));
}

#define CHECK(call)                                                               \
  do {                                                                            \
    pdmp_status st_ = (call);                                                     \
    if (st_ != PDMP_OK) {                                                         \
      fprintf(stderr, "%s failed: %s\n", #call, pdmp_status_string(st_));         \
      return 1;                                                                   \
    }                                                                             \
  } while (0)

int main(void) {
  const int d = 2, M = 1024, N = 1 << 16, T = 20;
  float* hc = (float*)malloc(sizeof(float) * M * d);
  float* hw = (float*)malloc(sizeof(float) * M);
  float* hx = (float*)malloc(sizeof(float) * N * d);
  float* hy = (float*)malloc(sizeof(float) * N * d);
  for (int m = 0; m < M; ++m) {
    hc[2 * m] = 10.0f * uniform01();
    hc[2 * m + 1] = 10.0f * uniform01();
    hw[m] = 2.0f * uniform01() - 1.0f;
  }
  for (int i = 0; i < N * d; ++i) hx[i] = 10.0f * uniform01();

  float *dc, *dw, *dx, *dy;
  void* ws;
  cudaMalloc((void**)&dc, sizeof(float) * M * d);
  cudaMalloc((void**)&dw, sizeof(float) * M);
  cudaMalloc((void**)&dx, sizeof(float) * N * d);
  cudaMalloc((void**)&dy, sizeof(float) * N * d);
  cudaMemcpy(dc, hc, sizeof(float) * M * d, cudaMemcpyHostToDevice);
  cudaMemcpy(dw, hw, sizeof(float) * M, cudaMemcpyHostToDevice);
  cudaMemcpy(dx, hx, sizeof(float) * N * d, cudaMemcpyHostToDevice);

  pdmp_field f;
  f.kind = PDMP_KIND_RBF;
  f.d = d;
  f.M = M;
  f.centres = dc;
  f.phase = NULL;
  f.gamma = 4.0f;
  f.w = dw;
  f.bias = 0.0f;
  f.lipschitz = 0.0;

  double lo[2] = {-0.5, -0.5}, hi[2] = {10.5, 10.5}, L = 0.0, G = 0.0;
  CHECK(pdmp_lipschitz_bound(&f, lo, hi, 64, &L, &G, NULL));
  f.lipschitz = L;
  const float eta = (float)(0.5 / L);

  const size_t ws_bytes = pdmp_morph_workspace(&f, N);
  cudaMalloc(&ws, ws_bytes);
  CHECK(pdmp_morph(&f, dx, N, T, eta, dy, NULL, 0, ws, ws_bytes, NULL));
  int32_t detail = 0;
  CHECK(pdmp_stream_status(NULL, &detail));
  cudaMemcpy(hy, dy, sizeof(float) * N * d, cudaMemcpyDeviceToHost);

  double sum = 0.0, maxd = 0.0;
  for (int i = 0; i < N; ++i) {
    const double ddx = hy[2 * i] - hx[2 * i], ddy = hy[2 * i + 1] - hx[2 * i + 1];
    sum += hy[2 * i] + hy[2 * i + 1];
    const double dist = sqrt(ddx * ddx + ddy * ddy);
    if (dist > maxd) maxd = dist;
  }
  printf("pdmp %d: N=%d M=%d T=%d L=%.6g eta=%.6g checksum=%.6f max_displacement=%.6g\n", pdmp_version(), N, M, T, L,
         eta, sum, maxd);
  cudaFree(dc);
  cudaFree(dw);
  cudaFree(dx);
  cudaFree(dy);
  cudaFree(ws);
  free(hc);
  free(hw);
  free(hx);
  free(hy);
  return 0;
}
