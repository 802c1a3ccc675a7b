// Certified Lipschitz constant of grad c (Sec. 3.2: the IVP of Eq. (1) needs
// a Lipschitz gradient; the Euler step is kept below 1 / L), in FP64.
//
//   |Hess c|_2 <= |sigma'| |Hess s|_2 + |sigma''| |grad s|^2
//              <= |Hess s|_2 / 4 + |grad s|^2 / (6 sqrt 3)
// (max sigma(1-sigma) = 1/4 at s = 0; max |sigma(1-sigma)(1-2 sigma)| =
// sqrt(3)/18 where sigma = (3 +- sqrt 3)/6).
//
// RBF, r = |x - mu|:  |grad phi| = 2 g r e^{-g r^2} =: h1(r), maximal at
// r = 1/sqrt(2g);  |Hess phi|_2 = max(2g, |4 g^2 r^2 - 2g|) e^{-g r^2} =: h2(r),
// which in u = g r^2 decreases on [0, 1], increases on [1, 3/2] and decreases
// after, so its maximum over an interval is at an end or at u = 3/2.
#include "field.cuh"
#include "kernels.cuh"

namespace pdmp {

__device__ unsigned long long g_lip_bits[2];   // [0] bound on |Hess c|, [1] on |grad c|

constexpr int kLipThreads = 128;
constexpr int kLipTile = 512;

__device__ __forceinline__ double rbf_h1(double g, double r) { return 2.0 * g * r * exp(-g * r * r); }
__device__ __forceinline__ double rbf_h2(double g, double r) {
  double u = g * r * r;
  return 2.0 * g * fmax(1.0, fabs(2.0 * u - 1.0)) * exp(-u);
}
__device__ __forceinline__ double h1_sup(double g, double rmin, double rmax) {
  double rpk = rsqrt(2.0 * g);
  if (rmax <= rpk) return rbf_h1(g, rmax);
  if (rmin >= rpk) return rbf_h1(g, rmin);
  return rbf_h1(g, rpk);
}
__device__ __forceinline__ double h2_sup(double g, double rmin, double rmax) {
  double v = fmax(rbf_h2(g, rmin), rbf_h2(g, rmax));
  double rpk = sqrt(1.5 / g);
  if (rmin <= rpk && rpk <= rmax) v = fmax(v, rbf_h2(g, rpk));
  return v;
}

template <int D>
__global__ void __launch_bounds__(kLipThreads)
k_lip_rbf(const float* __restrict__ centres, const float* __restrict__ w, int64_t M, double gamma, double lo0,
          double lo1, double lo2, double wd0, double wd1, double wd2, int cells, int64_t ncells) {
  __shared__ double sm[kLipTile * (D + 1)];
  const int64_t cell = (int64_t)blockIdx.x * kLipThreads + threadIdx.x;
  double blo[D], bhi[D];
  {
    const double lo[3] = {lo0, lo1, lo2}, wd[3] = {wd0, wd1, wd2};
    int64_t rem = cell;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      int64_t k = rem % cells;
      rem /= cells;
      blo[j] = lo[j] + wd[j] * (double)k;
      bhi[j] = lo[j] + wd[j] * (double)(k + 1);
    }
  }
  double sum1 = 0.0, sum2 = 0.0;
  for (int64_t m0 = 0; m0 < M; m0 += kLipTile) {
    __syncthreads();
    const int cnt = (int)min64(kLipTile, M - m0);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
#pragma unroll
      for (int j = 0; j < D; ++j) sm[i * (D + 1) + j] = (double)centres[(m0 + i) * D + j];
      sm[i * (D + 1) + D] = fabs((double)w[m0 + i]);
    }
    __syncthreads();
    if (cell < ncells) {
      for (int i = 0; i < cnt; ++i) {
        const double* mu = sm + i * (D + 1);
        double dmin2 = 0.0, dmax2 = 0.0;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          double a = blo[j] - mu[j], b = mu[j] - bhi[j];
          double out = fmax(fmax(a, b), 0.0);           // distance outside the slab
          double far = fmax(fabs(a), fabs(b));          // distance to the far face
          dmin2 += out * out;
          dmax2 += far * far;
        }
        double rmin = sqrt(dmin2), rmax = sqrt(dmax2);
        sum1 += mu[D] * h1_sup(gamma, rmin, rmax);
        sum2 += mu[D] * h2_sup(gamma, rmin, rmax);
      }
    }
  }
  if (cell < ncells) {
    double L = 0.25 * sum2 + sum1 * sum1 / (6.0 * sqrt(3.0));
    double G = 0.25 * sum1;
    atomicMax(&g_lip_bits[0], (unsigned long long)__double_as_longlong(L));
    atomicMax(&g_lip_bits[1], (unsigned long long)__double_as_longlong(G));
  }
}

// RFF: single block; fixed-order tree sums of |w| |omega| and |w| |omega|^2.
__global__ void __launch_bounds__(1024) k_lip_rff(const float* __restrict__ omega, const float* __restrict__ w,
                                                  int64_t M, int d) {
  __shared__ double s1[1024], s2[1024];
  double a = 0.0, b = 0.0;
  for (int64_t m = threadIdx.x; m < M; m += blockDim.x) {
    double n2 = 0.0;
    for (int j = 0; j < d; ++j) {
      double o = (double)omega[m * d + j];
      n2 += o * o;
    }
    double aw = fabs((double)w[m]);
    a += aw * sqrt(n2);
    b += aw * n2;
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double L = 0.25 * s2[0] + s1[0] * s1[0] / (6.0 * sqrt(3.0));
    g_lip_bits[0] = (unsigned long long)__double_as_longlong(L);
    g_lip_bits[1] = (unsigned long long)__double_as_longlong(0.25 * s1[0]);
  }
}

cudaError_t lipschitz_bound(int kind, int d, const FieldArgs& fa, const double* lo, const double* hi, int cells,
                            double* L, double* G, cudaStream_t st) {
  unsigned long long zero[2] = {0ull, 0ull};
  cudaError_t e = cudaMemcpyToSymbolAsync(g_lip_bits, zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  if (kind == PDMP_KIND_RFF) {
    k_lip_rff<<<1, 1024, 0, st>>>(fa.centres, fa.w, fa.M, d);
  } else {
    double l[3] = {0, 0, 0}, wd[3] = {0, 0, 0};
    int64_t ncells = 1;
    for (int j = 0; j < d; ++j) {
      l[j] = lo[j];
      wd[j] = (hi[j] - lo[j]) / cells;
      ncells *= cells;
    }
    unsigned blocks = (unsigned)((ncells + kLipThreads - 1) / kLipThreads);
    double g = (double)fa.gamma;
    if (d == 1) k_lip_rbf<1><<<blocks, kLipThreads, 0, st>>>(fa.centres, fa.w, fa.M, g, l[0], l[1], l[2], wd[0], wd[1], wd[2], cells, ncells);
    if (d == 2) k_lip_rbf<2><<<blocks, kLipThreads, 0, st>>>(fa.centres, fa.w, fa.M, g, l[0], l[1], l[2], wd[0], wd[1], wd[2], cells, ncells);
    if (d == 3) k_lip_rbf<3><<<blocks, kLipThreads, 0, st>>>(fa.centres, fa.w, fa.M, g, l[0], l[1], l[2], wd[0], wd[1], wd[2], cells, ncells);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  unsigned long long bits[2];
  e = cudaMemcpyFromSymbolAsync(bits, g_lip_bits, sizeof(bits), 0, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  double v[2];
  memcpy(&v[0], &bits[0], 8);
  memcpy(&v[1], &bits[1], 8);
  *L = v[0];
  if (G) *G = v[1];
  return cudaSuccess;
}

}  // namespace pdmp
