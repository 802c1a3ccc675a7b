"""Configuration space (Sec. 3.2, Eq. (3)): the occupancy on a planar chain's
body points pulled back to joint space and the morph there, against the FP64
oracle; RBF (fast sorted gradient path) and RFF (direct query path) fields."""
import numpy as np
import pytest
import torch

import oracle
import paper_2108_11775_gb300 as pdmp
import workloads as wl
from gpu_util import max_abs, setup_oracle_threads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available()
    setup_oracle_threads()
    yield
    assert pdmp.stream_status()[0] == 0


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def sampled_eta(f, ch, n=40, seed=47, safety=2.0):
    """eta = 0.5 / (safety x the largest sampled |Hess_q f_c|_2), the Hessians by
    central differences of the oracle's joint-space gradient (the certified
    bound is loose by orders of magnitude; it is checked separately)."""
    lo, hi = wl.joint_box(ch.n)
    Q = wl.uniform_box(seed, 3, n, lo, hi).astype(np.float64)
    h, worst = 1e-5, 0.0
    for q in Q:
        H = np.zeros((ch.n, ch.n))
        for j in range(ch.n):
            e = np.zeros(ch.n)
            e[j] = h
            H[j] = (oracle.cspace_evaluate(f, ch, (q + e)[None])[1][0]
                    - oracle.cspace_evaluate(f, ch, (q - e)[None])[1][0]) / (2 * h)
        worst = max(worst, np.linalg.norm(0.5 * (H + H.T), 2))
    return float(np.float32(0.5 / (safety * worst)))


def case(kind=wl.RBF, n=7, p=4, M=2048, seed=41):
    if kind == wl.RBF:
        f = wl.random_field(seed, wl.RBF, 2, M, lo=0, hi=10, gamma=4.0, wscale=1.0, bias=-0.5)
    else:
        f = wl.random_field(seed, wl.RFF, 2, M, wscale=3.0, bias=-0.5)
    ch = wl.planar_arm(n, 4.5, (5.0, 5.0), p)
    return f, ch, sampled_eta(f, ch)


@pytest.mark.parametrize("kind", [wl.RBF, wl.RFF])
def test_one_step_and_T_steps_match_oracle(kind):
    f, ch, eta = case(kind)
    lo, hi = wl.joint_box(ch.n)
    N = 3001
    q0 = wl.uniform_box(42, 3, N, lo, hi)
    fld = pdmp.DeviceField.from_host(f)
    q1 = pdmp.cspace_morph(fld, ch, dev(q0), 1, eta).cpu().numpy()
    ref1 = oracle.cspace_morph(f, ch, q0, 1, eta)
    inc, rinc = q1 - q0, ref1 - q0
    err = np.linalg.norm(inc - rinc, axis=1)
    assert (err <= 1e-5 * np.linalg.norm(rinc, axis=1) + 4 * np.pi * 2.0 ** -23).all()
    T = 20
    qT = pdmp.cspace_morph(fld, ch, dev(q0), T, eta).cpu().numpy()
    idx = np.arange(0, N, 11)
    ref = oracle.cspace_morph(f, ch, q0[idx], T, eta)
    assert max_abs(qT[idx], ref) <= 1e-4
    assert np.abs(qT - q0).max() > 1e-3


def test_in_place_ragged_and_empty():
    f, ch, eta = case(n=3, p=2, M=512, seed=43)
    fld = pdmp.DeviceField.from_host(f)
    lo, hi = wl.joint_box(ch.n)
    for N in (1, 5, 129):
        q0 = wl.uniform_box(44 + N, 3, N, lo, hi)
        q = dev(q0)
        out = pdmp.cspace_morph(fld, ch, q, 6, eta, out=q)
        assert out.data_ptr() == q.data_ptr()
        assert max_abs(q.cpu().numpy(), oracle.cspace_morph(f, ch, q0, 6, eta)) <= 1e-4
    q = dev(wl.uniform_box(45, 3, 4, lo, hi))
    assert torch.equal(pdmp.cspace_morph(fld, ch, q, 0, eta), q)
    assert pdmp.cspace_morph(fld, ch, torch.empty(0, ch.n, device="cuda"), 3, eta).shape == (0, ch.n)


def test_bound_matches_oracle_and_morph_lowers_the_cost():
    """The fitted-like 2-D field under a 7-link arm: the library's certified
    joint-space bound equals the oracle's, and the morph lowers the summed
    body-point occupancy (the purpose of Eq. (3)) for most samples."""
    lo2, hi2 = np.zeros(2), np.full(2, 10.0)
    centres = wl.uniform_box(2, wl.S_CENTRES, 4096, lo2, hi2)
    boxes = wl.random_boxes(2, 24, lo2, hi2, 0.3, 1.5)
    f = wl.Field(wl.RBF, centres, wl.proxy_fitted_weights(2, centres, boxes, scale=2.0), gamma=8.0)
    ch = wl.planar_arm(7, 4.5, (5.0, 5.0), 4)
    Lx, Gx = oracle.lipschitz(f, lo2 - 0.5, hi2 + 0.5, cells=64)
    Lq = oracle.cspace_lipschitz(ch, Lx, Gx)
    assert abs(pdmp.cspace_lipschitz(ch, Lx, Gx) - Lq) <= 1e-12 * Lq
    eta = sampled_eta(f, ch, n=20)
    lo, hi = wl.joint_box(ch.n)
    q0 = wl.uniform_box(46, 3, 512, lo, hi)
    fld = pdmp.DeviceField.from_host(f)
    qT = pdmp.cspace_morph(fld, ch, dev(q0), 40, eta).cpu().numpy()
    f0, _ = oracle.cspace_evaluate(f, ch, q0)
    fT, _ = oracle.cspace_evaluate(f, ch, qT)
    assert (fT <= f0 + 1e-9).mean() > 0.95
    assert fT.sum() < f0.sum()
