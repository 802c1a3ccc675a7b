// Configuration space (Sec. 3.2, "Bringing Diffeomorphisms into Configuration
// Space", Eq. (3)).  A planar serial chain with n revolute joints carries p
// body points per link; the cost on them is the summed occupancy, and its
// joint-space gradient pulls the task-space gradients back through the
// kinematic Jacobians:  grad_q f_c = sum_i J_i^T grad_x c(psi_i(q)), where
// column j of J_i is z x (psi_i - o_j) for the joints j that move point i.
//
// One Euler step of Eq. (1) in joint space is three launches: the body points
// of every sample (forward kinematics), grad c at all N b points (the fast
// RBF tile kernel, spatially sorted, with its update discarded), and the
// pull-back fused with the update q <- q - eta grad_q f_c.
#include "kernels.cuh"

namespace pdmp {

struct ChainArgs {
  int n, p;
  float base[2];
  float len[kChainMax];
};

// absolute link angles, joint positions o[0..n] and the body points of one sample
__device__ __forceinline__ void chain_fk(const ChainArgs& ch, const float* q, float (*o)[2], float* cs, float* sn) {
  float th = 0.0f;
  o[0][0] = ch.base[0];
  o[0][1] = ch.base[1];
  for (int k = 0; k < ch.n; ++k) {
    th += q[k];
    sincosf(th, &sn[k], &cs[k]);
    o[k + 1][0] = fmaf(ch.len[k], cs[k], o[k][0]);
    o[k + 1][1] = fmaf(ch.len[k], sn[k], o[k][1]);
  }
}

__device__ __forceinline__ void body_point(const ChainArgs& ch, const float (*o)[2], const float* cs,
                                           const float* sn, int i, float& px, float& py) {
  const int k = i / ch.p, r = i % ch.p + 1;
  const float f = (float)r / (float)ch.p * ch.len[k];
  px = fmaf(f, cs[k], o[k][0]);
  py = fmaf(f, sn[k], o[k][1]);
}

__global__ void k_chain_points(ChainArgs ch, const float* __restrict__ q, int64_t N, float* __restrict__ P) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  float qs[kChainMax], o[kChainMax + 1][2], cs[kChainMax], sn[kChainMax];
  for (int k = 0; k < ch.n; ++k) qs[k] = q[s * ch.n + k];
  chain_fk(ch, qs, o, cs, sn);
  const int b = ch.n * ch.p;
  for (int i = 0; i < b; ++i) {
    float px, py;
    body_point(ch, o, cs, sn, i, px, py);
    P[(s * b + i) * 2] = px;
    P[(s * b + i) * 2 + 1] = py;
  }
}

// grad_q f_c by Eq. (3) from the body-point gradients G, then the Euler step
__global__ void k_chain_pullback(ChainArgs ch, const float* __restrict__ q, int64_t N, const float* __restrict__ G,
                                 float eta, float* __restrict__ q_out) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  float qs[kChainMax], o[kChainMax + 1][2], cs[kChainMax], sn[kChainMax], gq[kChainMax];
  for (int k = 0; k < ch.n; ++k) {
    qs[k] = q[s * ch.n + k];
    gq[k] = 0.0f;
  }
  chain_fk(ch, qs, o, cs, sn);
  const int b = ch.n * ch.p;
  for (int i = 0; i < b; ++i) {
    float px, py;
    body_point(ch, o, cs, sn, i, px, py);
    const float gx = G[(s * b + i) * 2], gy = G[(s * b + i) * 2 + 1];
    const int link = i / ch.p;
    for (int j = 0; j <= link; ++j) gq[j] = fmaf(px - o[j][0], gy, fmaf(-(py - o[j][1]), gx, gq[j]));
  }
  for (int k = 0; k < ch.n; ++k) q_out[s * ch.n + k] = fmaf(-eta, gq[k], qs[k]);
}

static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

size_t cspace_workspace(int d, int64_t M, int n, int p, int64_t N) {
  const int64_t pts = N * n * p;
  return 2 * align256(sizeof(float) * 2 * pts) + morph_rbf_fast_workspace(d, M, pts);
}

cudaError_t cspace_morph(const FieldArgs& fa, int kind, const int n, const int p, const float* base,
                         const float* len, const float* q0, int64_t N, int T, float eta, float* qT, void* ws,
                         cudaStream_t st) {
  ChainArgs ch{};
  ch.n = n;
  ch.p = p;
  ch.base[0] = base[0];
  ch.base[1] = base[1];
  for (int k = 0; k < n; ++k) ch.len[k] = len[k];
  const int64_t pts = N * n * p;
  float* P = (float*)ws;
  float* G = (float*)((char*)ws + align256(sizeof(float) * 2 * pts));
  void* fws = (char*)ws + 2 * align256(sizeof(float) * 2 * pts);
  const unsigned nb = (unsigned)((N + 127) / 128);
  cudaError_t e;
  for (int t = 0; t < T; ++t) {
    const float* q = t == 0 ? q0 : qT;
    k_chain_points<<<nb, 128, 0, st>>>(ch, q, N, P);
    if (kind == PDMP_KIND_RBF)
      e = grad_rbf_fast(2, fa, P, pts, G, fws, st);
    else
      e = occupancy_query(kind, 2, fa, P, pts, nullptr, nullptr, G, st);
    if (e != cudaSuccess) return e;
    k_chain_pullback<<<nb, 128, 0, st>>>(ch, q, N, G, eta, qT);
  }
  return cudaGetLastError();
}

}  // namespace pdmp
