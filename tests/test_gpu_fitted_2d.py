"""Parity on the benchmarked workload itself: the 2-D fitted field (16,384
RBF centres, gamma = 8) with the occupancy weights the oracle fitted alone
(tests/golden/fit_rbf2d_fitted.txt, written by make_golden.py --fit-rbf2d;
Sec. 3.1), N = 2^20 samples and T = 50 steps at eta = 0.5 / L, L the
oracle's certified bound stored with the fit -- the field, samples, step and
launch configuration that bench.py times.

* the GPU fit (pdmp_fit_occupancy, the same algorithm on the same data)
  reaches the oracle's loss to 1e-4 relative, and the GPU's certified bound
  on the stored field equals the oracle's;
* every one of the 50 steps of 200 sampled samples (per-step tolerance, the
  oracle at the GPU's own state), and their final positions against the
  oracle's own 50-step chain (1e-4); the trace twin equals the timed kernel
  bit for bit on all 2^20 samples;
* the VJP (k = 5, from the forward's checkpoints): the correction g0 - gT to
  1e-4 of its norm against the oracle's VJP taken segment by segment from the
  GPU's checkpointed states, and g0 to 1e-4 against the oracle's full chain;
* the log-det and the inverse on sampled samples.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2108_11775_gb300 as pdmp
import workloads as wl
from gpu_util import max_abs, per_step_check, setup_oracle_threads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fitted():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    setup_oracle_threads()
    wk, params = wl.config2_fitted()
    L = params["L"]
    eta = float(np.float32(0.5 / L))
    fld = pdmp.DeviceField.from_host(wk.field, lipschitz=L)
    yield wk, params, eta, fld
    st, detail = pdmp.stream_status()
    assert st == 0, (st, detail)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def sample_idx(N, n, seed):
    return np.unique(np.concatenate([wl.rng(seed, 1).choice(N, n, replace=False), [0, N - 1]]))


def test_gpu_fit_reaches_the_oracle_fit(fitted):
    """The same fit (lambda = 1e-4, 20 power iterations, 200 Nesterov
    iterations) on the same 200k labelled points: the GPU's final loss equals
    the oracle's to 1e-4 relative (Sec. 3.1 with the fit's parity rule); the
    GPU's certified bound on the stored field equals the oracle's."""
    wk, params, eta, fld = fitted
    w, b, loss, alpha = pdmp.fit_occupancy(fld, dev(wk.fit_X), dev(wk.fit_y), params["l2"],
                                           params["power_iters"], params["iters"])
    assert abs(alpha - params["alpha"]) <= 1e-4 * params["alpha"]
    assert abs(loss - params["loss_f64"]) <= 1e-4 * params["loss_f64"]
    L, G = pdmp.lipschitz_bound(fld, wk.lo - 0.5, wk.hi + 0.5, cells=128)
    assert abs(L - params["L"]) <= 1e-9 * params["L"] and abs(G - params["G"]) <= 1e-9 * params["G"]


def test_morph_per_step_and_final_at_full_size(fitted):
    """The full trace (N = 2^20, T = 50) through pdmp_morph_trace, the same
    kernels and tiles as the timed pdmp_morph (bit-identical final state on
    every sample); each step of 200 sampled samples at the per-step tolerance,
    and their x_T against the oracle's own chain from the same float32 x0."""
    wk, params, eta, fld = fitted
    N, T = wk.x0.shape[0], wk.T
    x0 = dev(wk.x0)
    traj, steps = pdmp.morph_trace(fld, x0, T, eta)
    xT = pdmp.morph(fld, x0, T, eta)
    assert torch.equal(traj[-1], xT), "the trace twin and the timed kernel disagree"
    idx = sample_idx(N, 200, 21)
    it = torch.from_numpy(idx).cuda()
    tr = traj[:, it].cpu().numpy()
    st = steps[:, it].cpu().numpy()
    del traj, steps
    assert np.array_equal(tr[0], wk.x0[idx])
    worst = per_step_check(wk.field, tr, st, eta)
    assert worst <= 1.0
    ref = oracle.morph(wk.field, wk.x0[idx], T, eta)
    assert max_abs(tr[-1], ref) <= 1e-4
    assert np.abs(ref - wk.x0[idx]).max() > 1e-2          # the samples moved
    assert bool(torch.isfinite(xT).all())


def test_vjp_segmentwise_against_the_oracle_at_full_size(fitted):
    """The VJP as the benchmark's extra runs it (N = 2^20, T = 50, k = 5,
    sorted tiles, from the forward's checkpoints).  The oracle takes each
    segment's VJP from the GPU's checkpointed state (promoted to FP64) and
    chains the cotangent back: the 50-step FP32 trajectory then cannot
    separate the two sides, and the correction g0 - gT must agree to 1e-4 of
    its norm.  g0 also agrees with the oracle's own full FP64 chain to 1e-4."""
    wk, params, eta, fld = fitted
    N, T, k = wk.x0.shape[0], wk.T, 5
    x0 = dev(wk.x0)
    gT = wl.f32(wl.rng(2, wl.S_COTANGENT).standard_normal((N, 2)))
    ck = torch.empty(T // k, N, 2, device="cuda")
    pdmp.morph(fld, x0, T, eta, ckpt=ck, k=k)
    g0 = pdmp.morph_vjp(fld, x0, T, eta, k, dev(gT), ckpt=ck).cpu().numpy()
    assert np.isfinite(g0).all()
    idx = sample_idx(N, 48, 22)
    cks = ck[:, torch.from_numpy(idx).cuda()].cpu().numpy()
    g = gT[idx].astype(np.float64)
    for j in reversed(range(T // k)):
        start = wk.x0[idx] if j == 0 else cks[j - 1]
        g = oracle.morph_vjp(wk.field, start, k, eta, g)
    corr = g - gT[idx]
    assert np.linalg.norm(corr) > 1e-3 * np.linalg.norm(gT[idx])     # the chain is not the identity
    assert np.linalg.norm((g0[idx] - gT[idx]) - corr) <= 1e-4 * np.linalg.norm(corr)
    r0 = oracle.morph_vjp(wk.field, wk.x0[idx], T, eta, gT[idx])
    assert np.linalg.norm(g0[idx] - r0) <= 1e-4 * np.linalg.norm(r0)


def test_logdet_sampled_at_full_size(fitted):
    """sum_t log det(I - eta Hess c(x_t)) on all 2^20 samples (sorted tiles)
    against the oracle on sampled samples (abs 1e-4 T); det > 0 at every step."""
    wk, params, eta, fld = fitted
    N, T = wk.x0.shape[0], wk.T
    ld = pdmp.logdet(fld, dev(wk.x0), T, eta).cpu().numpy()
    assert np.isfinite(ld).all()
    idx = sample_idx(N, 48, 23)
    rl, _, mindet = oracle.logdet(wk.field, wk.x0[idx], T, eta)
    assert np.all(mindet > 0)
    assert max_abs(ld[idx], rl) <= 1e-4 * T
    assert np.abs(rl).max() > 1e-3                          # the Jacobian is not the identity


def test_inverse_sampled_at_the_bench_size(fitted):
    """Eq. (2) as the benchmark's extra runs it: the first 2^18 samples
    morphed through T = 50 steps, then inverted on sorted tiles; sampled
    samples against the oracle's inverse, and the round trip on all."""
    wk, params, eta, fld = fitted
    n = 1 << 18
    x0 = np.ascontiguousarray(wk.x0[:n])
    z = pdmp.morph(fld, dev(x0), wk.T, eta)
    work = torch.zeros(1, dtype=torch.int64, device="cuda")
    y = pdmp.morph_inverse(fld, z, wk.T, eta, tol=1e-6, maxit=60, work=work).cpu().numpy()
    assert np.isfinite(y).all()
    assert max_abs(y, x0) <= 1e-4
    idx = sample_idx(n, 24, 24)
    ref, _ = oracle.morph_inverse(wk.field, z.cpu().numpy()[idx], wk.T, eta, tol=1e-13, maxit=200)
    assert max_abs(y[idx], ref) <= 1e-4
    assert int(work.item()) >= n * wk.T * wk.field.M


def test_log_density_in_one_kernel_at_the_bench_size(fitted):
    """The log-density (Eq. 2 and the change of variables of Sec. 3.2) as the
    benchmark's extra runs it: the first 2^18 samples morphed through T = 50
    steps, then inverted with every step's log-det taken from the inverse's
    last fixed-point sweep.  Against the two-kernel path (the inverse, then
    the forward log-det from the recovered points) on every sample and the
    oracle's log-det at the recovered points on sampled ones, both at abs
    1e-4 T; the recovered points equal x0 to 1e-4."""
    wk, params, eta, fld = fitted
    n, T = 1 << 18, wk.T
    lo, hi = np.asarray(wk.lo, np.float64), np.asarray(wk.hi, np.float64)
    x0 = np.ascontiguousarray(wk.x0[:n])
    z = pdmp.morph(fld, dev(x0), T, eta)
    lp, y = pdmp.log_density(fld, z, T, eta, lo, hi, tol=1e-6, maxit=60)
    lp, yh = lp.cpu().numpy(), y.cpu().numpy()
    assert max_abs(yh, x0) <= 1e-4
    inside = np.all((yh > lo + 1e-3) & (yh < hi - 1e-3), axis=1)
    assert inside.mean() > 0.99 and np.isfinite(lp[inside]).all()
    log_vol = float(np.log(np.prod(hi - lo)))
    ld2 = pdmp.logdet(fld, y, T, eta).cpu().numpy()
    assert np.abs(lp[inside] - (-log_vol - ld2[inside])).max() <= 1e-4 * T
    idx = sample_idx(n, 24, 25)
    idx = idx[inside[idx]]
    rl, _, _ = oracle.logdet(wk.field, yh[idx], T, eta)
    assert np.abs(lp[idx] - (-log_vol - rl)).max() <= 1e-4 * T
    assert np.abs(rl).max() > 1e-3


def test_tensor_core_morph_per_step_and_final_at_full_size(fitted, monkeypatch):
    """The opt-in tensor-core form (PDMP_RBF_TC05=1: the exponent on tcgen05)
    on the benchmarked field at full size: each of the 50 steps of 200
    sampled samples at the per-step tolerance, their x_T against the oracle's
    chain (1e-4), and every x_T within 1e-4 of the default FP32 kernel's."""
    wk, params, eta, fld = fitted
    N, T = wk.x0.shape[0], wk.T
    x0 = dev(wk.x0)
    monkeypatch.setenv("PDMP_RBF_TC05", "0")
    xT_fp32 = pdmp.morph(fld, x0, T, eta)
    monkeypatch.setenv("PDMP_RBF_TC05", "1")
    traj, steps = pdmp.morph_trace(fld, x0, T, eta)
    xT = pdmp.morph(fld, x0, T, eta)
    assert torch.equal(traj[-1], xT), "the trace twin and the timed kernel disagree"
    assert (xT - xT_fp32).abs().max().item() <= 1e-4
    idx = sample_idx(N, 200, 23)
    it = torch.from_numpy(idx).cuda()
    tr = traj[:, it].cpu().numpy()
    st = steps[:, it].cpu().numpy()
    del traj, steps
    assert per_step_check(wk.field, tr, st, eta) <= 1.0
    ref = oracle.morph(wk.field, wk.x0[idx], T, eta)
    assert max_abs(tr[-1], ref) <= 1e-4
