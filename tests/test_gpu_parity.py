"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (from the stated accuracy targets):
* per step:  |step_gpu - step_ref|_inf <= 1e-5 eta sigma'(s) sum_m |w_m| |grad phi_m|
             + 1e-5 |step_ref|_inf, with step_gpu the kernel's FP32 increment
             at the GPU's own state x_t (promoted to FP64 for the oracle);
* final:     |x_T gpu - x_T ref|_inf <= 1e-4, oracle started from the same
             float32 x_0;
* VJP:       normwise relative 1e-4 (on g0 - gT when the chain is near the
             identity);
* log-det:   absolute 1e-4 T;
* labels:    bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2108_11775_gb300 as pdmp
import workloads as wl
from gpu_util import max_abs, per_step_check, rbf_eta, rff_eta_certified, rff_eta_sampled, setup_oracle_threads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    setup_oracle_threads()
    pdmp.lib()
    yield
    st, detail = pdmp.stream_status()
    assert st == 0, (st, detail)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# --------------------------------------------------------------------------
# morph: 2-D grid field, 4096 samples, 10 steps
@pytest.mark.parametrize("fast", [True, False])
def test_morph_config1_per_step_and_final(fast):
    w1 = wl.config1()
    eta, L = rbf_eta(w1.field, w1.lo, w1.hi)
    fld = pdmp.DeviceField.from_host(w1.field, lipschitz=L)
    x0 = dev(w1.x0)
    traj, steps = pdmp.morph_trace(fld, x0, w1.T, eta, fast=fast)
    traj, steps = traj.cpu().numpy(), steps.cpu().numpy()
    assert np.array_equal(traj[0], w1.x0)
    per_step_check(w1.field, traj, steps, eta)
    xT = pdmp.morph(fld, x0, w1.T, eta, fast=fast).cpu().numpy()
    assert np.array_equal(xT, traj[-1]), "morph and its trace twin disagree"
    ref = oracle.morph(w1.field, w1.x0, w1.T, eta)
    assert max_abs(xT, ref) <= 1e-4
    assert np.abs(ref - w1.x0).max() > 1e-2          # the samples moved


@pytest.mark.parametrize("kind,d,M,N,T", [
    (wl.RBF, 1, 7, 37, 5), (wl.RBF, 2, 1, 1, 4), (wl.RBF, 2, 300, 1000, 6), (wl.RBF, 3, 513, 777, 5),
    (wl.RBF, 2, 257, 513, 3), (wl.RFF, 1, 33, 100, 5), (wl.RFF, 3, 129, 301, 4), (wl.RFF, 7, 300, 257, 5),
    (wl.RFF, 8, 64, 65, 3), (wl.RFF, 4, 17, 130, 3), (wl.RFF, 5, 1000, 700, 4), (wl.RFF, 6, 129, 128, 4),
    (wl.RFF, 7, 2048, 1, 3),
])
def test_morph_ragged_shapes(kind, d, M, N, T):
    if kind == wl.RBF:
        f = wl.random_field(50 + d + M, kind, d, M, lo=0, hi=3, gamma=3.0, wscale=2.0, bias=0.25)
        lo, hi = np.full(d, -1.0), np.full(d, 4.0)
        eta, _ = rbf_eta(f, lo, hi, cells=32 if d < 3 else 12)
        x0 = wl.uniform_box(60 + N, 3, N, np.zeros(d), np.full(d, 3.0))
    else:
        f = wl.random_field(50 + d + M, kind, d, M, wscale=4.0, bias=-0.1)
        lo, hi = np.full(d, -np.pi), np.full(d, np.pi)
        eta, _ = rff_eta_sampled(f, lo, hi, n=500)
        x0 = wl.uniform_box(60 + N, 3, N, lo, hi)
    fld = pdmp.DeviceField.from_host(f)
    traj, steps = pdmp.morph_trace(fld, dev(x0), T, eta)
    per_step_check(f, traj.cpu().numpy(), steps.cpu().numpy(), eta)
    xT = pdmp.morph(fld, dev(x0), T, eta).cpu().numpy()
    assert max_abs(xT, oracle.morph(f, x0, T, eta)) <= 1e-4


@pytest.mark.parametrize("d", [2, 3])
def test_fast_path_dense_tiles_per_step_and_final(d):
    """Enough samples that the sorted 320-sample tiles are compact, so the
    fast kernel runs its expanded form; checked on a subset of the samples."""
    if d == 2:
        f = wl.config1().field
        lo, hi, N, T = np.zeros(2), np.full(2, 10.0), 1 << 16, 10
        eta, L = rbf_eta(f, lo, hi)
    else:
        f = wl.random_field(77, wl.RBF, 3, 8192, lo=0, hi=5, gamma=8.0, wscale=2.0, bias=-0.2)
        lo, hi, N, T = np.zeros(3), np.full(3, 5.0), 1 << 18, 8
        eta, L = rbf_eta(f, lo - 0.5, hi + 0.5, cells=16)
    x0 = wl.uniform_box(80 + d, 3, N, lo, hi)
    fld = pdmp.DeviceField.from_host(f, lipschitz=L)
    traj, steps = pdmp.morph_trace(fld, dev(x0), T, eta)
    xT = pdmp.morph(fld, dev(x0), T, eta).cpu().numpy()
    xT2 = pdmp.morph(fld, dev(x0), T, eta).cpu().numpy()
    traj, steps = traj.cpu().numpy(), steps.cpu().numpy()
    assert np.array_equal(xT, xT2), "the fast path is not deterministic"
    assert np.array_equal(xT, traj[-1])
    idx = np.sort(wl.rng(d, 9).choice(N, 160, replace=False))
    per_step_check(f, traj[:, idx], steps[:, idx], eta)
    assert max_abs(xT[idx], oracle.morph(f, x0[idx], T, eta)) <= 1e-4
    direct = pdmp.morph(fld, dev(x0), T, eta, fast=False).cpu().numpy()
    assert max_abs(xT, direct) <= 1e-4


def test_morph_in_place_zero_steps_and_empty():
    w1 = wl.config1(N=300)
    eta, _ = rbf_eta(w1.field, w1.lo, w1.hi)
    fld = pdmp.DeviceField.from_host(w1.field)
    x = dev(w1.x0)
    ref = pdmp.morph(fld, x, 4, eta).cpu().numpy()
    pdmp.morph(fld, x, 4, eta, out=x)                 # in place
    assert np.array_equal(x.cpu().numpy(), ref)
    y = dev(w1.x0)
    out = pdmp.morph(fld, y, 0, eta)
    assert np.array_equal(out.cpu().numpy(), w1.x0)
    empty = torch.empty(0, 2, device="cuda")
    assert pdmp.morph(fld, empty, 4, eta).shape == (0, 2)


def test_morph_zero_weights_is_identity():
    f = wl.random_field(3, wl.RBF, 2, 100).with_weights(np.zeros(100), bias=0.3)
    x0 = wl.uniform_box(3, 3, 1000, [0, 0], [10, 10])
    out = pdmp.morph(pdmp.DeviceField.from_host(f), dev(x0), 20, 0.5).cpu().numpy()
    assert np.array_equal(out, x0)


def test_checkpoints_are_the_trajectory():
    w1 = wl.config1(N=700)
    eta, _ = rbf_eta(w1.field, w1.lo, w1.hi)
    fld = pdmp.DeviceField.from_host(w1.field)
    ck = torch.empty(5, 700, 2, device="cuda")
    xT = pdmp.morph(fld, dev(w1.x0), 10, eta, ckpt=ck, k=2)
    traj, _ = pdmp.morph_trace(fld, dev(w1.x0), 10, eta)
    traj = traj.cpu().numpy()
    ck = ck.cpu().numpy()
    for j in range(5):
        assert np.array_equal(ck[j], traj[2 * (j + 1)])
    assert np.array_equal(xT.cpu().numpy(), traj[-1])


def test_step_size_checked_against_the_field_bound():
    w1 = wl.config1(N=16)
    _, L = rbf_eta(w1.field, w1.lo, w1.hi)
    fld = pdmp.DeviceField.from_host(w1.field, lipschitz=L)
    with pytest.raises(pdmp.PdmpError) as e:
        pdmp.morph(fld, dev(w1.x0), 3, 1.5 / L)
    assert e.value.status == 2


# --------------------------------------------------------------------------
# full-size workloads, sampled
def test_morph_rff_7d_full_size_sampled():
    wk = wl.config3()
    eta, L = rff_eta_certified(wk.field)
    fld = pdmp.DeviceField.from_host(wk.field, lipschitz=L)
    k = wk.extra["k"]
    ck = torch.empty(wk.T // k, wk.x0.shape[0], 7, device="cuda")
    xT = pdmp.morph(fld, dev(wk.x0), wk.T, eta, ckpt=ck, k=k).cpu().numpy()
    idx = np.concatenate([np.sort(wl.rng(8, 1).choice(wk.x0.shape[0], 24, replace=False)), [wk.x0.shape[0] - 1]])
    ref = oracle.morph(wk.field, wk.x0[idx], wk.T, eta)
    assert max_abs(xT[idx], ref) <= 1e-4
    assert np.abs(ref - wk.x0[idx]).max() > 1e-5


# --------------------------------------------------------------------------
# VJP and log-det
def _vjp_case(kind):
    if kind == wl.RBF:
        w1 = wl.config1(N=256)
        eta, _ = rbf_eta(w1.field, w1.lo, w1.hi)
        return w1.field, w1.x0, 10, 5, eta
    f = wl.random_field(21, wl.RFF, 7, 256, wscale=6.0, bias=0.1)
    lo, hi = np.full(7, -np.pi), np.full(7, np.pi)
    eta, _ = rff_eta_sampled(f, lo, hi, n=800)
    return f, wl.uniform_box(21, 3, 128, lo, hi), 20, 5, eta


@pytest.mark.parametrize("kind", [wl.RBF, wl.RFF])
@pytest.mark.parametrize("use_ckpt", [True, False])
def test_vjp_matches_oracle(kind, use_ckpt):
    f, x0, T, k, eta = _vjp_case(kind)
    fld = pdmp.DeviceField.from_host(f)
    N, d = x0.shape
    gT = wl.f32(wl.rng(5, wl.S_COTANGENT).standard_normal((N, d)))
    ck = None
    if use_ckpt:
        ck = torch.empty(T // k, N, d, device="cuda")
        pdmp.morph(fld, dev(x0), T, eta, ckpt=ck, k=k)
    g0, gw, gb = pdmp.morph_vjp(fld, dev(x0), T, eta, k, dev(gT), ckpt=ck, want_param_grad=True)
    g0, gw, gb = g0.cpu().numpy(), gw.cpu().numpy(), float(gb.cpu().numpy()[0])
    r0, rw, rb = oracle.morph_vjp(f, x0, T, eta, gT, want_gw=True)
    corr_ref = r0 - gT
    assert np.linalg.norm(g0 - r0) <= 1e-4 * np.linalg.norm(r0)
    assert np.linalg.norm((g0 - gT) - corr_ref) <= 1e-4 * np.linalg.norm(corr_ref) + 1e-6
    assert np.linalg.norm(gw - rw) <= 1e-4 * np.linalg.norm(rw)
    assert abs(gb - rb) <= 1e-4 * max(abs(rb), 1e-3)


@pytest.mark.parametrize("d,N,T,k,use_ckpt", [(7, 300, 12, 4, True), (7, 129, 12, 12, False), (3, 97, 6, 1, True),
                                              (5, 1, 4, 2, False)])
def test_vjp_tensor_core_path(d, N, T, k, use_ckpt):
    """RFF, d <= 7, no parameter gradient: the tensor-core VJP (ragged
    blocks, with and without checkpoints, segments of 1 .. T steps, g0
    written over gT) against the oracle and the direct kernel."""
    f = wl.random_field(30 + d, wl.RFF, d, 300, wscale=6.0, bias=0.1)
    lo, hi = np.full(d, -np.pi), np.full(d, np.pi)
    eta, _ = rff_eta_sampled(f, lo, hi, n=600)
    x0 = wl.uniform_box(31 + d, 3, N, lo, hi)
    gT = wl.f32(wl.rng(32 + d, wl.S_COTANGENT).standard_normal((N, d)))
    fld = pdmp.DeviceField.from_host(f)
    assert pdmp.morph_vjp_workspace(fld, N, T, k, False) > 0
    ck = None
    if use_ckpt:
        ck = torch.empty(T // k, N, d, device="cuda")
        pdmp.morph(fld, dev(x0), T, eta, ckpt=ck, k=k)
    g = dev(gT)
    out = pdmp.morph_vjp(fld, dev(x0), T, eta, k, g, ckpt=ck, g0=g)
    assert out.data_ptr() == g.data_ptr()
    g0 = out.cpu().numpy()
    r0 = oracle.morph_vjp(f, x0, T, eta, gT)
    corr = r0 - gT
    assert np.linalg.norm(g0 - r0) <= 1e-4 * np.linalg.norm(r0)
    assert np.linalg.norm((g0 - gT) - corr) <= 1e-4 * np.linalg.norm(corr) + 1e-6
    direct = pdmp.morph_vjp(fld, dev(x0), T, eta, k, dev(gT), ckpt=ck, fast=False).cpu().numpy()
    assert np.linalg.norm(g0 - direct) <= 1e-4 * np.linalg.norm(direct)


@pytest.mark.parametrize("d,N,M,T,k,use_ckpt", [(7, 300, 300, 12, 4, True), (3, 129, 77, 6, 6, False),
                                                (5, 1, 130, 4, 2, True)])
def test_vjp_param_grad_tensor_core_path(d, N, M, T, k, use_ckpt):
    """RFF, d <= 7, with the weight and bias gradient: the tensor-core VJP's
    second pass per step (ragged sample blocks, M past one stage of 128
    features and below it) against the oracle's d/dw, d/dbias and the direct
    kernel's."""
    f = wl.random_field(40 + d, wl.RFF, d, M, wscale=6.0, bias=0.1)
    lo, hi = np.full(d, -np.pi), np.full(d, np.pi)
    eta, _ = rff_eta_sampled(f, lo, hi, n=600)
    x0 = wl.uniform_box(41 + d, 3, N, lo, hi)
    gT = wl.f32(wl.rng(42 + d, wl.S_COTANGENT).standard_normal((N, d)))
    fld = pdmp.DeviceField.from_host(f)
    assert pdmp.morph_vjp_workspace(fld, N, T, k, 1) > pdmp.morph_vjp_workspace(fld, N, T, k, 2) > 0
    ck = None
    if use_ckpt:
        ck = torch.empty(T // k, N, d, device="cuda")
        pdmp.morph(fld, dev(x0), T, eta, ckpt=ck, k=k)
    g0, gw, gb = pdmp.morph_vjp(fld, dev(x0), T, eta, k, dev(gT), ckpt=ck, want_param_grad=True)
    g0, gw, gb = g0.cpu().numpy(), gw.cpu().numpy(), float(gb.cpu().numpy()[0])
    r0, rw, rb = oracle.morph_vjp(f, x0, T, eta, gT, want_gw=True)
    assert np.linalg.norm(g0 - r0) <= 1e-4 * np.linalg.norm(r0)
    assert np.linalg.norm(gw - rw) <= 1e-4 * np.linalg.norm(rw)
    assert abs(gb - rb) <= 1e-4 * max(abs(rb), 1e-3)
    d0, dw, db = pdmp.morph_vjp(fld, dev(x0), T, eta, k, dev(gT), ckpt=ck, want_param_grad=True, fast=False)
    assert np.linalg.norm(gw - dw.cpu().numpy()) <= 1e-4 * np.linalg.norm(rw)
    assert np.array_equal(g0, pdmp.morph_vjp(fld, dev(x0), T, eta, k, dev(gT), ckpt=ck).cpu().numpy())


def test_vjp_and_logdet_rff_7d_full_size_sampled():
    """The differentiation workload as the benchmark runs it (N = 2^20,
    M = 4096, T = 20, k = 5, tensor-core kernels): the VJP from the forward's
    checkpoints and the log-det, on sampled samples against the oracle."""
    wk = wl.config3()
    eta, L = rff_eta_certified(wk.field)
    fld = pdmp.DeviceField.from_host(wk.field, lipschitz=L)
    N, T, k = wk.x0.shape[0], wk.T, wk.extra["k"]
    x0 = dev(wk.x0)
    gT = wk.extra["gT"]
    ck = torch.empty(T // k, N, 7, device="cuda")
    pdmp.morph(fld, x0, T, eta, ckpt=ck, k=k)
    g0 = pdmp.morph_vjp(fld, x0, T, eta, k, dev(gT), ckpt=ck).cpu().numpy()
    ld = pdmp.logdet(fld, x0, T, eta).cpu().numpy()
    assert np.isfinite(g0).all() and np.isfinite(ld).all()
    idx = np.concatenate([np.sort(wl.rng(10, 1).choice(N, 20, replace=False)), [0, N - 1]])
    r0 = oracle.morph_vjp(wk.field, wk.x0[idx], T, eta, gT[idx])
    corr = r0 - gT[idx]
    assert np.linalg.norm((g0[idx] - gT[idx]) - corr) <= 1e-4 * np.linalg.norm(corr)
    rl, _, mindet = oracle.logdet(wk.field, wk.x0[idx], T, eta)
    assert np.all(mindet > 0)
    assert max_abs(ld[idx], rl) <= 1e-4 * T


def test_rff_7d_full_size_with_a_visible_step():
    """The 7-D workload's field and shape (N = 2^20, M = 4096, T = 20, k = 5)
    at a step from the sampled Hessian (reading 6) rather than the loose
    certified bound, so that the chain moves visibly, through the
    tensor-core kernels: every step of sampled samples at the per-step
    tolerance (the oracle at the GPU's own state), the VJP correction with the
    oracle chained segment by segment from the GPU's checkpoints (1e-4 of its
    norm), and the log-det (abs 1e-4 T, det > 0 at every step)."""
    wk = wl.config3()
    f = wk.field
    lo, hi = np.full(7, -np.pi), np.full(7, np.pi)
    eta, _ = rff_eta_sampled(f, lo, hi, n=800)
    fld = pdmp.DeviceField.from_host(f)
    N, T, k = wk.x0.shape[0], wk.T, wk.extra["k"]
    x0 = dev(wk.x0)
    idx = np.concatenate([np.sort(wl.rng(12, 1).choice(N, 40, replace=False)), [0, N - 1]])
    it = torch.from_numpy(idx).cuda()
    traj, steps = pdmp.morph_trace(fld, x0, T, eta)
    tr, st = traj[:, it].cpu().numpy(), steps[:, it].cpu().numpy()
    del traj, steps
    assert per_step_check(f, tr, st, eta) <= 1.0
    assert np.abs(tr[-1] - wk.x0[idx]).max() > 1e-2             # the chain moves visibly
    ck = torch.empty(T // k, N, 7, device="cuda")
    xT = pdmp.morph(fld, x0, T, eta, ckpt=ck, k=k)
    assert np.array_equal(xT[it].cpu().numpy(), tr[-1])
    gT = wk.extra["gT"]
    g0 = pdmp.morph_vjp(fld, x0, T, eta, k, dev(gT), ckpt=ck).cpu().numpy()
    cks = ck[:, it].cpu().numpy()
    g = gT[idx].astype(np.float64)
    for j in reversed(range(T // k)):
        start = wk.x0[idx] if j == 0 else cks[j - 1]
        g = oracle.morph_vjp(f, start, k, eta, g)
    corr = g - gT[idx]
    assert np.linalg.norm(corr) > 1e-2 * np.linalg.norm(gT[idx])
    assert np.linalg.norm((g0[idx] - gT[idx]) - corr) <= 1e-4 * np.linalg.norm(corr)
    ld = pdmp.logdet(fld, x0, T, eta).cpu().numpy()
    assert np.isfinite(ld).all()
    rl, _, mindet = oracle.logdet(f, wk.x0[idx], T, eta)
    assert np.all(mindet > 0)
    assert max_abs(ld[idx], rl) <= 1e-4 * T
    assert np.abs(rl).max() > 1e-2
    assert pdmp.stream_status()[0] == 0


@pytest.mark.parametrize("d,N,T,k,use_ckpt", [(2, 1000, 10, 5, True), (2, 700, 6, 6, False), (3, 451, 6, 2, True),
                                              (3, 193, 4, 1, False)])
def test_vjp_sorted_tiles_rbf(d, N, T, k, use_ckpt):
    """RBF, d = 2, 3, no parameter gradient: the sorted-tile VJP (ragged
    tiles, with and without checkpoints, g0 written over gT) against the
    oracle and the direct kernel."""
    f = wl.random_field(70 + d, wl.RBF, d, 500, lo=0.0, hi=4.0, gamma=4.0, wscale=2.0, bias=0.2)
    lo, hi = np.zeros(d), np.full(d, 4.0)
    eta, _ = rbf_eta(f, lo - 0.5, hi + 0.5, cells=32 if d == 2 else 12)
    x0 = wl.uniform_box(71 + d, 3, N, lo, hi)
    gT = wl.f32(wl.rng(72 + d, wl.S_COTANGENT).standard_normal((N, d)))
    fld = pdmp.DeviceField.from_host(f)
    assert pdmp.morph_vjp_workspace(fld, N, T, k, False) > 0
    ck = None
    if use_ckpt:
        ck = torch.empty(T // k, N, d, device="cuda")
        pdmp.morph(fld, dev(x0), T, eta, ckpt=ck, k=k)
    g = dev(gT)
    g0 = pdmp.morph_vjp(fld, dev(x0), T, eta, k, g, ckpt=ck, g0=g).cpu().numpy()
    r0 = oracle.morph_vjp(f, x0, T, eta, gT)
    corr = r0 - gT
    assert np.linalg.norm(g0 - r0) <= 1e-4 * np.linalg.norm(r0)
    assert np.linalg.norm((g0 - gT) - corr) <= 1e-4 * np.linalg.norm(corr) + 1e-6
    direct = pdmp.morph_vjp(fld, dev(x0), T, eta, k, dev(gT), ckpt=ck, fast=False).cpu().numpy()
    assert np.linalg.norm(g0 - direct) <= 1e-4 * np.linalg.norm(direct)


@pytest.mark.parametrize("d,N,M,T,k,use_ckpt,hi", [(2, 4096, 500, 6, 3, True, 1.0), (3, 4096, 300, 4, 2, False, 1.0),
                                                   (2, 300, 500, 6, 3, True, 4.0), (3, 257, 77, 4, 4, False, 4.0),
                                                   (2, 1, 130, 4, 2, True, 4.0)])
def test_vjp_param_grad_sorted_tiles_rbf(d, N, M, T, k, use_ckpt, hi):
    """RBF, d = 2, 3, with the weight and bias gradient: the sorted-tile VJP's
    transposed pass (4096 samples in the unit box: compact tiles, expanded
    form; a few hundred in [0, 4]^d: wide tiles, direct form; ragged tiles,
    M below and past a warp's slice) against the oracle's d/dw, d/dbias and
    the direct kernel's; g0 is the same, bit for bit, as without the
    parameter gradient."""
    f = wl.random_field(90 + d, wl.RBF, d, M, lo=0.0, hi=hi, gamma=4.0, wscale=2.0, bias=0.2)
    lo, hb = np.zeros(d), np.full(d, hi)
    eta, _ = rbf_eta(f, lo - 0.5, hb + 0.5, cells=32 if d == 2 else 12)
    x0 = wl.uniform_box(91 + d, 3, N, lo, hb)
    gT = wl.f32(wl.rng(92 + d, wl.S_COTANGENT).standard_normal((N, d)))
    fld = pdmp.DeviceField.from_host(f)
    assert pdmp.morph_vjp_workspace(fld, N, T, k, 1) > pdmp.morph_vjp_workspace(fld, N, T, k, 2) > 0
    ck = None
    if use_ckpt:
        ck = torch.empty(T // k, N, d, device="cuda")
        pdmp.morph(fld, dev(x0), T, eta, ckpt=ck, k=k)
    g0, gw, gb = pdmp.morph_vjp(fld, dev(x0), T, eta, k, dev(gT), ckpt=ck, want_param_grad=True)
    g0, gw, gb = g0.cpu().numpy(), gw.cpu().numpy(), float(gb.cpu().numpy()[0])
    assert pdmp.stream_status()[0] == 0
    r0, rw, rb = oracle.morph_vjp(f, x0, T, eta, gT, want_gw=True)
    assert np.linalg.norm(g0 - r0) <= 1e-4 * np.linalg.norm(r0)
    assert np.linalg.norm(gw - rw) <= 1e-4 * np.linalg.norm(rw)
    assert abs(gb - rb) <= 1e-4 * max(abs(rb), 1e-3)
    _, dw, db = pdmp.morph_vjp(fld, dev(x0), T, eta, k, dev(gT), ckpt=ck, want_param_grad=True, fast=False)
    assert np.linalg.norm(gw - dw.cpu().numpy()) <= 1e-4 * np.linalg.norm(rw)
    assert np.array_equal(g0, pdmp.morph_vjp(fld, dev(x0), T, eta, k, dev(gT), ckpt=ck).cpu().numpy())


def test_vjp_and_inverse_sorted_tiles_dense_3d():
    """3-D samples dense enough (2^17 in [0,5]^3, gamma = 8: tiles of 192 or
    320 samples span g' R^2 of about 3 to 4) that the sorted tiles take the
    expanded form: the VJP and the inverse on sampled samples against the
    oracle, and against the direct kernels on all."""
    f = wl.random_field(79, wl.RBF, 3, 2048, lo=0, hi=5, gamma=8.0, wscale=2.0, bias=-0.2)
    lo, hi = np.zeros(3), np.full(3, 5.0)
    eta, L = rbf_eta(f, lo - 0.5, hi + 0.5, cells=16)
    fld = pdmp.DeviceField.from_host(f, lipschitz=L)
    N, T, k = 1 << 17, 4, 2
    x0 = wl.uniform_box(80, 3, N, lo, hi)
    gT = wl.f32(wl.rng(81, wl.S_COTANGENT).standard_normal((N, 3)))
    ck = torch.empty(T // k, N, 3, device="cuda")
    z = pdmp.morph(fld, dev(x0), T, eta, ckpt=ck, k=k)
    g0 = pdmp.morph_vjp(fld, dev(x0), T, eta, k, dev(gT), ckpt=ck).cpu().numpy()
    y = pdmp.morph_inverse(fld, z, T, eta, tol=1e-6, maxit=60).cpu().numpy()
    idx = np.concatenate([np.sort(wl.rng(82, 1).choice(N, 48, replace=False)), [N - 1]])
    r0 = oracle.morph_vjp(f, x0[idx], T, eta, gT[idx])
    assert np.linalg.norm(g0[idx] - r0) <= 1e-4 * np.linalg.norm(r0)
    corr = r0 - gT[idx]
    assert np.linalg.norm((g0[idx] - gT[idx]) - corr) <= 1e-4 * np.linalg.norm(corr) + 1e-6
    ry, _ = oracle.morph_inverse(f, z.cpu().numpy()[idx], T, eta, tol=1e-13, maxit=200)
    assert max_abs(y[idx], ry) <= 1e-4
    assert max_abs(y, x0) <= 1e-4
    gd = pdmp.morph_vjp(fld, dev(x0), T, eta, k, dev(gT), ckpt=ck, fast=False).cpu().numpy()
    assert np.linalg.norm(g0 - gd) <= 1e-4 * np.linalg.norm(gd)
    yd = pdmp.morph_inverse(fld, z, T, eta, tol=1e-6, maxit=60, fast=False).cpu().numpy()
    assert max_abs(y, yd) <= 1e-4


def test_vjp_rff_7d_certified_step_full_chain():
    wk = wl.config3(N=4096)
    eta, _ = rff_eta_certified(wk.field)
    fld = pdmp.DeviceField.from_host(wk.field)
    gT = wk.extra["gT"]
    ck = torch.empty(4, 4096, 7, device="cuda")
    pdmp.morph(fld, dev(wk.x0), 20, eta, ckpt=ck, k=5)
    g0 = pdmp.morph_vjp(fld, dev(wk.x0), 20, eta, 5, dev(gT), ckpt=ck).cpu().numpy()
    idx = np.arange(0, 4096, 128)
    r0 = oracle.morph_vjp(wk.field, wk.x0[idx], 20, eta, gT[idx])
    corr = r0 - gT[idx]
    assert np.linalg.norm((g0[idx] - gT[idx]) - corr) <= 1e-4 * np.linalg.norm(corr)


@pytest.mark.parametrize("kind", [wl.RBF, wl.RFF])
def test_logdet_matches_oracle_and_is_diffeomorphic(kind):
    f, x0, T, _, eta = _vjp_case(kind)
    fld = pdmp.DeviceField.from_host(f)
    ld, xT = pdmp.logdet(fld, dev(x0), T, eta, want_xT=True)
    ld, xT = ld.cpu().numpy(), xT.cpu().numpy()
    ref, xref, mindet = oracle.logdet(f, x0, T, eta)
    assert np.all(mindet > 0)
    assert max_abs(ld, ref) <= 1e-4 * T
    assert max_abs(xT, xref) <= 1e-4
    assert pdmp.stream_status()[0] == 0


@pytest.mark.parametrize("d,N,T,M", [(7, 300, 6, 300), (3, 131, 5, 1000), (1, 64, 4, 17), (5, 129, 3, 260)])
def test_logdet_tensor_core_path(d, N, T, M):
    """RFF, d <= 7, with the workspace: the tensor-core log-det (ragged blocks,
    several stages, the Hessian's d(d+1)/2 entries) against the oracle and
    the direct kernel."""
    f = wl.random_field(60 + d, wl.RFF, d, M, wscale=6.0, bias=0.1)
    lo, hi = np.full(d, -np.pi), np.full(d, np.pi)
    eta, _ = rff_eta_sampled(f, lo, hi, n=600)
    x0 = wl.uniform_box(61 + d, 3, N, lo, hi)
    fld = pdmp.DeviceField.from_host(f)
    ld, xT = pdmp.logdet(fld, dev(x0), T, eta, want_xT=True)
    ld, xT = ld.cpu().numpy(), xT.cpu().numpy()
    ref, xref, mindet = oracle.logdet(f, x0, T, eta)
    assert np.all(mindet > 0)
    assert max_abs(ld, ref) <= 1e-4 * T
    assert max_abs(xT, xref) <= 1e-4
    assert np.abs(ref).max() > 1e-3                       # the steps change volume measurably
    direct = pdmp.logdet(fld, dev(x0), T, eta, fast=False).cpu().numpy()
    assert max_abs(ld, direct) <= 1e-4 * T
    assert pdmp.stream_status()[0] == 0


@pytest.mark.parametrize("d", [2, 3])
def test_logdet_sorted_tiles_rbf(d):
    """RBF, d = 2, 3 with the workspace: the log-det on the morph's sorted
    tiles (enough samples that tiles are compact and take the expanded form,
    plus a ragged last tile) against the oracle on sampled samples and the
    direct kernel on all."""
    if d == 2:
        f = wl.config1().field
        lo, hi, N, T = np.zeros(2), np.full(2, 10.0), (1 << 15) + 77, 6
        eta, L = rbf_eta(f, lo, hi)
    else:
        f = wl.random_field(78, wl.RBF, 3, 4096, lo=0, hi=5, gamma=8.0, wscale=2.0, bias=-0.2)
        lo, hi, N, T = np.zeros(3), np.full(3, 5.0), (1 << 15) + 5, 5
        eta, L = rbf_eta(f, lo - 0.5, hi + 0.5, cells=16)
    x0 = wl.uniform_box(90 + d, 3, N, lo, hi)
    fld = pdmp.DeviceField.from_host(f, lipschitz=L)
    ld, xT = pdmp.logdet(fld, dev(x0), T, eta, want_xT=True)
    ld, xT = ld.cpu().numpy(), xT.cpu().numpy()
    idx = np.concatenate([np.sort(wl.rng(d, 11).choice(N, 64, replace=False)), [N - 1]])
    ref, xref, mindet = oracle.logdet(f, x0[idx], T, eta)
    assert np.all(mindet > 0)
    assert max_abs(ld[idx], ref) <= 1e-4 * T
    assert max_abs(xT[idx], xref) <= 1e-4
    assert np.abs(ref).max() > 1e-3
    direct = pdmp.logdet(fld, dev(x0), T, eta, fast=False).cpu().numpy()
    assert max_abs(ld, direct) <= 1e-4 * T
    assert pdmp.stream_status()[0] == 0


def test_logdet_flags_a_non_diffeomorphic_step_on_the_tensor_cores():
    f = wl.random_field(66, wl.RFF, 7, 256, wscale=6.0, bias=0.1)
    lo, hi = np.full(7, -np.pi), np.full(7, np.pi)
    eta, _ = rff_eta_sampled(f, lo, hi, n=600)
    fld = pdmp.DeviceField.from_host(f)                   # carries no bound: the call is accepted
    ld = pdmp.logdet(fld, dev(wl.uniform_box(67, 3, 256, lo, hi)), 3, 400.0 * eta).cpu().numpy()
    st, detail = pdmp.stream_status()
    assert st == 7 and detail & 1
    assert np.isnan(ld).any()
    assert pdmp.stream_status()[0] == 0


def test_logdet_flags_a_non_diffeomorphic_step():
    w1 = wl.config1(N=128)
    _, L = rbf_eta(w1.field, w1.lo, w1.hi)
    fld = pdmp.DeviceField.from_host(w1.field)           # carries no bound: the call is accepted
    ld = pdmp.logdet(fld, dev(w1.x0), 3, 40.0 / L).cpu().numpy()
    st, detail = pdmp.stream_status()
    assert st == 7 and detail & 1
    assert np.isnan(ld).any()
    assert pdmp.stream_status()[0] == 0                   # the flag was cleared


# --------------------------------------------------------------------------
# queries, labels, Lipschitz bound
def test_occupancy_query_matches_oracle():
    w1 = wl.config1()
    fld = pdmp.DeviceField.from_host(w1.field)
    q = pdmp.occupancy_query(fld, dev(w1.x0))
    ev = oracle.evaluate(w1.field, w1.x0)
    abs_s = oracle.evaluate(w1.field.with_weights(np.abs(w1.field.w)), w1.x0)["s"]   # sum |w| phi
    assert np.all(np.abs(q["s"].cpu().numpy() - ev["s"]) <= 1e-5 * abs_s + 1e-6)
    assert np.all(np.abs(q["c"].cpu().numpy() - ev["c"]) <= 1e-5 * abs_s + 1e-6)
    g = q["grad"].cpu().numpy()
    assert np.all(np.abs(g - ev["grad"]).max(axis=1) <= 1e-5 * ev["scale"] + 1e-5 * np.abs(ev["grad"]).max(axis=1))


def _grid(lo, hi, n, d):
    axes = [lo + (hi - lo) * (np.arange(n) + 0.5) / n for _ in range(d)]
    mesh = np.meshgrid(*axes, indexing="ij")
    return wl.f32(np.stack([m.ravel() for m in mesh], axis=1))


@pytest.mark.parametrize("d", [2, 3])
def test_collision_labels_bit_exact_on_grid(d):
    if d == 2:
        wk = wl.config2(N=16)
        pts = _grid(0.0, 10.0, 256, 2)
    else:
        wk = wl.config5(N=16, n_train=16)
        pts = _grid(0.0, 5.0, 64, 3)
    # add points exactly on box faces and one ulp outside them
    b = wk.boxes
    face = np.concatenate([b[:, :d], b[:, d:], np.nextafter(b[:, d:], np.float32(np.inf)),
                           np.nextafter(b[:, :d], np.float32(-np.inf))])
    pts = np.concatenate([pts, wl.f32(face)])
    lab = pdmp.box_labels(dev(b), dev(pts)).cpu().numpy()
    ref = oracle.box_labels(b, pts)
    assert np.array_equal(lab, ref)
    assert 0 < ref.sum() < len(ref)
    assert np.array_equal(pdmp.box_labels(dev(np.zeros((0, 2 * d), np.float32)), dev(pts)).cpu().numpy(),
                          np.zeros(len(pts), np.uint8))


def test_learned_labels_on_grid_match_outside_the_margin():
    wk = wl.config2(N=16)
    f = wk.field.with_weights(wl.proxy_fitted_weights(2, wk.field.centres, wk.boxes), bias=-0.5)
    pts = _grid(0.0, 10.0, 128, 2)
    s_gpu = pdmp.occupancy_query(pdmp.DeviceField.from_host(f), dev(pts), want=("s",))["s"].cpu().numpy()
    ev = oracle.evaluate(f, pts)
    margin = 1e-5 * (oracle.evaluate(f.with_weights(np.abs(f.w), bias=0.0), pts)["s"] + abs(f.bias))
    sure = np.abs(ev["s"]) > margin
    assert sure.mean() > 0.999
    assert np.array_equal(s_gpu[sure] >= 0, ev["s"][sure] >= 0)


def test_lipschitz_bound_matches_oracle():
    w1 = wl.config1()
    L, G = pdmp.lipschitz_bound(pdmp.DeviceField.from_host(w1.field), w1.lo, w1.hi, cells=64)
    Lr, Gr = oracle.lipschitz(w1.field, w1.lo, w1.hi, cells=64)
    assert abs(L - Lr) <= 1e-9 * Lr and abs(G - Gr) <= 1e-9 * Gr
    f3 = wl.config3(N=8).field
    L, G = pdmp.lipschitz_bound(pdmp.DeviceField.from_host(f3))
    Lr, Gr = oracle.lipschitz(f3)
    assert abs(L - Lr) <= 1e-9 * Lr and abs(G - Gr) <= 1e-9 * Gr
    f3d = wl.random_field(4, wl.RBF, 3, 500, lo=0, hi=5, gamma=8.0)
    L, G = pdmp.lipschitz_bound(pdmp.DeviceField.from_host(f3d), [0, 0, 0], [5, 5, 5], cells=12)
    Lr, Gr = oracle.lipschitz(f3d, [0, 0, 0], [5, 5, 5], cells=12)
    assert abs(L - Lr) <= 1e-9 * Lr and abs(G - Gr) <= 1e-9 * Gr


# --------------------------------------------------------------------------
# occupancy fit
def test_fit_matches_oracle_same_algorithm():
    wk = wl.config2(N=16, M=256, n_fit=4096)
    f = wk.field
    w, b, loss, alpha = pdmp.fit_occupancy(pdmp.DeviceField.from_host(f), dev(wk.fit_X), dev(wk.fit_y), 1e-4, 30, 100)
    rw, rb, rloss, ralpha = oracle.fit(f, wk.fit_X, wk.fit_y, 1e-4, 30, 100)
    assert abs(alpha - ralpha) <= 1e-4 * ralpha
    assert abs(loss - rloss) <= 1e-4 * rloss
    w = w.cpu().numpy()
    assert np.linalg.norm(w - rw) <= 1e-3 * np.linalg.norm(rw)
    assert abs(b - rb) <= 1e-3 * max(1.0, abs(rb))


def test_fit_full_size_2d_learns_the_boxes():
    wk = wl.config2(N=16)
    fld = pdmp.DeviceField.from_host(wk.field)
    X, y = dev(wk.fit_X), dev(wk.fit_y)
    w, b, loss, _ = pdmp.fit_occupancy(fld, X, y, 1e-4, 20, 200)
    assert np.isfinite(loss) and loss < 0.35
    fitted = fld.with_weights(w, bias=b)
    s = pdmp.occupancy_query(fitted, X, want=("s",))["s"].cpu().numpy()
    acc = np.mean((s >= 0) == (wk.fit_y == 1))
    assert acc > 0.93
    # the oracle's objective at the GPU's weights agrees with the reported loss
    sub = slice(0, 20000)
    lo_, _, _ = oracle.fit_objective(wk.field, wk.fit_X[sub], wk.fit_y[sub], 1e-4, w.cpu().numpy(), b)
    assert abs(lo_ - loss) < 0.05


# --------------------------------------------------------------------------
# Eq. (2): the inverse map
@pytest.mark.parametrize("kind", [wl.RBF, wl.RFF])
@pytest.mark.parametrize("fast", [True, False])
def test_inverse_matches_oracle_and_round_trips(kind, fast):
    f, x0, T, _, eta = _vjp_case(kind)
    fld = pdmp.DeviceField.from_host(f)
    z = pdmp.morph(fld, dev(x0), T, eta)
    y, its = pdmp.morph_inverse(fld, z, T, eta, tol=1e-6, maxit=80, want_iters=True, fast=fast)
    y, its, z = y.cpu().numpy(), its.cpu().numpy(), z.cpu().numpy()
    ref, _ = oracle.morph_inverse(f, z, T, eta, tol=1e-13, maxit=200)
    assert max_abs(y, ref) <= 1e-4
    assert max_abs(y, x0) <= 1e-4                      # round trip through the forward map
    assert its.max() < 80
    assert np.abs(z - x0).max() > 1e-3


@pytest.mark.parametrize("d,N", [(2, 1000), (3, 1000), (3, 321)])
def test_inverse_sorted_tiles_ragged_in_place_and_work(d, N):
    """The sorted-tile inverse (RBF, d = 2, 3): ragged tiles, in place, the
    work counter, and agreement with the direct kernel and the oracle."""
    f = wl.random_field(40 + d, wl.RBF, d, 700, lo=0.0, hi=5.0, gamma=4.0, wscale=1.5)
    lo, hi = np.zeros(d), np.full(d, 5.0)
    eta, _ = rbf_eta(f, lo - 0.5, hi + 0.5, cells=32 if d == 2 else 12)
    T = 8
    x0 = wl.uniform_box(41 + d, 3, N, lo, hi)
    fld = pdmp.DeviceField.from_host(f)
    z = pdmp.morph(fld, dev(x0), T, eta)
    zc = z.clone()
    work = torch.zeros(1, dtype=torch.int64, device="cuda")
    y, its = pdmp.morph_inverse(fld, z, T, eta, tol=1e-6, maxit=60, want_iters=True, out=z, work=work)
    assert y.data_ptr() == z.data_ptr()
    y, its = y.cpu().numpy(), its.cpu().numpy()
    ref, _ = oracle.morph_inverse(f, zc.cpu().numpy(), T, eta, tol=1e-13, maxit=200)
    assert max_abs(y, ref) <= 1e-4
    assert max_abs(y, x0) <= 1e-4
    assert 1 <= its.min() and its.max() < 60
    wv = int(work.item())
    assert wv % f.M == 0 and T * N * f.M <= wv <= T * 60 * N * f.M
    yd = pdmp.morph_inverse(fld, zc, T, eta, tol=1e-6, maxit=60, fast=False).cpu().numpy()
    assert max_abs(y, yd) <= 1e-4
    assert np.abs(zc.cpu().numpy() - x0).max() > 1e-3


@pytest.mark.parametrize("d", [2, 3])
def test_inverse_and_log_density_large_launch_tiles(d):
    """2^19 samples: enough tiles that the sorted-tile inverse (320-sample
    tiles) and the one-kernel log-density (256 / 192) keep their larger tiles
    (smaller launches take 128-sample tiles). Sampled points against the
    oracle's inverse (1e-4) and its log-det at the recovered points (abs
    1e-4 T); the inverse also against the direct kernel on those points."""
    lo, hi = np.zeros(d), np.full(d, 10.0)
    fld_h = wl.random_field(60 + d, wl.RBF, d, 500, gamma=2.0, wscale=2.0, bias=-0.5)
    eta, _ = rbf_eta(fld_h, lo - 1.0, hi + 1.0, cells=32 if d == 2 else 10)
    T, N = 6, 1 << 19
    fld = pdmp.DeviceField.from_host(fld_h)
    x0 = wl.uniform_box(61 + d, 3, N, lo, hi)
    z = pdmp.morph(fld, dev(x0), T, eta)
    y = pdmp.morph_inverse(fld, z, T, eta, tol=1e-6, maxit=60).cpu().numpy()
    lp, yl = pdmp.log_density(fld, z, T, eta, lo, hi, tol=1e-6, maxit=60)
    lp, yl = lp.cpu().numpy(), yl.cpu().numpy()
    idx = np.sort(wl.rng(62 + d, 1).choice(N, 48, replace=False))
    zs = z.cpu().numpy()[idx]
    ry, _ = oracle.morph_inverse(fld_h, zs, T, eta, tol=1e-13, maxit=200)
    assert max_abs(y[idx], ry) <= 1e-4 and max_abs(yl[idx], ry) <= 1e-4
    yd = pdmp.morph_inverse(fld, dev(zs), T, eta, tol=1e-6, maxit=60, fast=False).cpu().numpy()
    assert max_abs(y[idx], yd) <= 1e-4
    inside = np.all((yl[idx] > lo + 1e-3) & (yl[idx] < hi - 1e-3), axis=1)
    sel = idx[inside]
    rl, _, mindet = oracle.logdet(fld_h, yl[sel], T, eta)
    assert np.all(mindet > 0) and sel.size > 30
    log_vol = float(np.log(np.prod(hi - lo)))
    assert np.abs(lp[sel] - (-log_vol - rl)).max() <= 1e-4 * T
    assert pdmp.stream_status()[0] == 0


@pytest.mark.parametrize("d,N", [(7, 257), (3, 300)])
def test_inverse_tensor_cores_rff(d, N):
    """RFF, d <= 7, with the workspace: the inverse on the tensor cores
    (ragged blocks, in place, the work counter) against the oracle, the round
    trip and the direct kernel."""
    f = wl.random_field(44 + d, wl.RFF, d, 300, wscale=6.0, bias=0.1)
    lo, hi = np.full(d, -np.pi), np.full(d, np.pi)
    eta, _ = rff_eta_sampled(f, lo, hi, n=600)
    T = 10
    x0 = wl.uniform_box(45 + d, 3, N, lo, hi)
    fld = pdmp.DeviceField.from_host(f)
    z = pdmp.morph(fld, dev(x0), T, eta)
    zc = z.clone()
    work = torch.zeros(1, dtype=torch.int64, device="cuda")
    y, its = pdmp.morph_inverse(fld, z, T, eta, tol=1e-6, maxit=60, want_iters=True, out=z, work=work)
    assert y.data_ptr() == z.data_ptr()
    y, its = y.cpu().numpy(), its.cpu().numpy()
    ref, _ = oracle.morph_inverse(f, zc.cpu().numpy(), T, eta, tol=1e-13, maxit=200)
    assert max_abs(y, ref) <= 1e-4
    assert max_abs(y, x0) <= 1e-4
    assert 1 <= its.min() and its.max() < 60
    wv = int(work.item())
    assert wv % f.M == 0 and T * N * f.M <= wv <= T * 60 * N * f.M
    yd = pdmp.morph_inverse(fld, zc, T, eta, tol=1e-6, maxit=60, fast=False).cpu().numpy()
    assert max_abs(y, yd) <= 1e-4
    assert np.abs(zc.cpu().numpy() - x0).max() > 1e-3


@pytest.mark.parametrize("kind,fast", [(wl.RBF, True), (wl.RBF, False), (wl.RFF, True)])
def test_inverse_reports_non_convergence(kind, fast):
    """An iteration cap too small for the tolerance raises the not-converged
    bit of the device flag (and the result is still the capped iterate);
    enough iterations leave the flag clear."""
    if kind == wl.RBF:
        f, x0, T, _, eta = _vjp_case(wl.RBF)
        x0 = np.tile(x0, (4, 1))[:1000]                    # several sorted tiles
    else:
        f, x0, T, _, eta = _vjp_case(wl.RFF)
    fld = pdmp.DeviceField.from_host(f)
    z = pdmp.morph(fld, dev(x0), T, eta)
    assert pdmp.stream_status()[0] == 0
    pdmp.morph_inverse(fld, z, T, eta, tol=0.0, maxit=1, fast=fast)
    st, detail = pdmp.stream_status()
    assert st == 7 and detail & 4
    pdmp.morph_inverse(fld, z, T, eta, tol=1e-6, maxit=80, fast=fast)
    assert pdmp.stream_status()[0] == 0


def test_log_density_matches_oracle_and_integrates_to_one():
    """log p_z = log p_0(phi^{-1}(z)) - log det J: against the oracle's inverse
    and log-det on sampled points, and normalised (Monte Carlo over a box that
    contains the support of p_z)."""
    w1 = wl.config1(N=256)
    eta, _ = rbf_eta(w1.field, w1.lo, w1.hi)
    T = 10
    fld = pdmp.DeviceField.from_host(w1.field)
    lo, hi = np.asarray(w1.lo, np.float64), np.asarray(w1.hi, np.float64)
    # points of the base box pushed forward: log p_z(z) = -log vol - log det J(y)
    y0 = wl.uniform_box(31, 3, 4096, lo, hi)
    z = pdmp.morph(fld, dev(y0), T, eta)
    lp, y = pdmp.log_density(fld, z, T, eta, lo, hi)
    lp, y = lp.cpu().numpy(), y.cpu().numpy()
    ref_ld, _, _ = oracle.logdet(w1.field, y0, T, eta)
    inside = np.all((y0 > lo + 1e-3) & (y0 < hi - 1e-3), axis=1)
    assert inside.mean() > 0.99
    assert np.abs(lp[inside] - (-np.log(np.prod(hi - lo)) - ref_ld[inside])).max() <= 1e-4 * T
    # arbitrary points, including outside the image of the box: the oracle's inverse decides
    zq = wl.uniform_box(32, 3, 512, lo - 1.0, hi + 1.0)
    lq, yq = pdmp.log_density(fld, dev(zq), T, eta, lo, hi)
    lq, yq = lq.cpu().numpy(), yq.cpu().numpy()
    ry, _ = oracle.morph_inverse(w1.field, zq, T, eta)
    assert max_abs(yq, ry) <= 1e-4
    rin = np.all((ry >= lo) & (ry <= hi), axis=1)
    clear = np.all(np.minimum(np.abs(ry - lo), np.abs(ry - hi)) > 1e-3, axis=1)
    assert np.array_equal(np.isfinite(lq)[clear], rin[clear])
    rld, _, _ = oracle.logdet(w1.field, ry[rin & clear], T, eta)
    assert np.abs(lq[rin & clear] + np.log(np.prod(hi - lo)) + rld).max() <= 1e-4 * T
    # normalisation
    n = 1 << 20
    zb_lo, zb_hi = lo - 1.0, hi + 1.0
    zs = wl.uniform_box(33, 3, n, zb_lo, zb_hi)
    ls, _ = pdmp.log_density(fld, dev(zs), T, eta, lo, hi)
    mass = float(torch.exp(ls.double()).mean()) * np.prod(zb_hi - zb_lo)
    assert abs(mass - 1.0) <= 5e-3


@pytest.mark.parametrize("d", [2, 3])
def test_log_density_one_kernel_matches_two_kernels_and_oracle(d):
    """With a workspace, RBF fields in d = 2, 3 take the log-density in one
    kernel (each step's log-det from the inverse's last fixed-point sweep).
    Ragged tiles (256 samples for d = 2, 192 for d = 3) and points outside
    the image of the box: the recovered points against the oracle's inverse
    (1e-4), the log-density against the two-kernel path (the inverse, then
    the forward log-det from the recovered points) and against the oracle's
    log-det at the recovered points, both abs 1e-4 T."""
    lo, hi = np.zeros(d), np.full(d, 10.0)
    fld_h = wl.random_field(40 + d, wl.RBF, d, 600 if d == 2 else 900, gamma=2.0, wscale=2.0, bias=-0.5)
    eta, _ = rbf_eta(fld_h, lo - 1.0, hi + 1.0, cells=32 if d == 2 else 10)
    T = 8
    fld = pdmp.DeviceField.from_host(fld_h)
    n = 4096 + 77
    x0 = wl.uniform_box(41 + d, 3, n, lo - 0.5, hi + 0.5)
    z = pdmp.morph(fld, dev(x0), T, eta)
    lp, y = pdmp.log_density(fld, z, T, eta, lo, hi, tol=1e-6, maxit=60)
    lp, yh = lp.cpu().numpy(), y.cpu().numpy()
    assert max_abs(yh, x0) <= 1e-4
    clear = np.all(np.minimum(np.abs(yh - lo), np.abs(yh - hi)) > 1e-3, axis=1)
    rin = np.all((yh >= lo) & (yh <= hi), axis=1)
    assert np.array_equal(np.isfinite(lp)[clear], rin[clear])
    assert (clear & ~rin).sum() > 0 and (clear & rin).sum() > n // 2
    log_vol = float(np.log(np.prod(hi - lo)))
    yin = np.ascontiguousarray(yh[clear & rin])
    ld2 = pdmp.logdet(fld, dev(yin), T, eta).cpu().numpy()
    assert np.abs(lp[clear & rin] - (-log_vol - ld2)).max() <= 1e-4 * T
    idx = np.flatnonzero(clear & rin)[:: max(1, (clear & rin).sum() // 40)]
    ry, _ = oracle.morph_inverse(fld_h, z.cpu().numpy()[idx], T, eta, tol=1e-13, maxit=200)
    assert max_abs(yh[idx], ry) <= 1e-4
    rl, _, mindet = oracle.logdet(fld_h, yh[idx], T, eta)
    assert np.all(mindet > 0)
    assert np.abs(lp[idx] - (-log_vol - rl)).max() <= 1e-4 * T
    assert np.abs(rl).max() > 1e-3
    assert pdmp.stream_status()[0] == 0
