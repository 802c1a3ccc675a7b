"""Edge cases of the morph at the limits: very many centres, very many
samples (sampled against the oracle), and non-finite samples, which must not
disturb the other samples of their tile."""
import numpy as np
import pytest
import torch

import oracle
import paper_2108_11775_gb300 as pdmp
import workloads as wl
from gpu_util import max_abs, rbf_eta, setup_oracle_threads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available()
    setup_oracle_threads()
    yield


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_a_million_centres():
    """M = 2^20 centres on [0,10]^2 (gamma = 64, so a feature is narrow),
    4096 samples, T = 2: fast and direct paths against the oracle on 48 samples."""
    M = 1 << 20
    f = wl.random_field(61, wl.RBF, 2, M, lo=0, hi=10, gamma=64.0, wscale=0.05, bias=-0.5)
    fld = pdmp.DeviceField.from_host(f)
    lo, hi = np.zeros(2), np.full(2, 10.0)
    x0 = wl.uniform_box(61, 3, 4096, lo, hi)
    eta = 1e-4
    idx = np.arange(0, 4096, 85)
    ref = oracle.morph(f, x0[idx], 2, eta)
    for fast in (True, False):
        out = pdmp.morph(fld, dev(x0), 2, eta, fast=fast).cpu().numpy()
        assert max_abs(out[idx], ref) <= 1e-4
    assert pdmp.stream_status()[0] == 0


def test_sixteen_million_samples():
    """N = 2^24 samples (the largest configuration's sample count), M = 256,
    T = 3, on the fast path: sampled against the oracle, every output finite."""
    N = 1 << 24
    f = wl.random_field(62, wl.RBF, 2, 256, lo=0, hi=10, gamma=4.0, wscale=1.0)
    eta, L = rbf_eta(f, np.full(2, -0.5), np.full(2, 10.5), cells=32)
    fld = pdmp.DeviceField.from_host(f, lipschitz=L)
    x0 = wl.uniform_box(62, 3, N, np.zeros(2), np.full(2, 10.0))
    out = pdmp.morph(fld, dev(x0), 3, eta)
    assert bool(torch.isfinite(out).all())
    idx = np.sort(wl.rng(62, 9).choice(N, 256, replace=False))
    ref = oracle.morph(f, x0[idx], 3, eta)
    assert max_abs(out.cpu().numpy()[idx], ref) <= 1e-4


def test_non_finite_samples_stay_local():
    """NaN and infinite samples give non-finite outputs and leave every other
    sample (also those in their tiles) within the tolerance of the oracle."""
    w1 = wl.config1(N=4096)
    eta, L = rbf_eta(w1.field, w1.lo, w1.hi)
    fld = pdmp.DeviceField.from_host(w1.field, lipschitz=L)
    x0 = w1.x0.copy()
    bad = np.array([5, 700, 701, 3000])
    x0[bad[0], 0] = np.nan
    x0[bad[1], 1] = np.inf
    x0[bad[2]] = -np.inf
    x0[bad[3], 0] = np.nan
    good = np.setdiff1d(np.arange(4096), bad)
    for fast in (True, False):
        out = pdmp.morph(fld, dev(x0), w1.T, eta, fast=fast).cpu().numpy()
        assert not np.isfinite(out[bad]).all(axis=1).any()
        idx = good[::41]
        ref = oracle.morph(w1.field, x0[idx], w1.T, eta)
        assert max_abs(out[idx], ref) <= 1e-4
        assert np.isfinite(out[good]).all()


def test_rff_tensor_cores_many_features():
    """7-D random Fourier field with M = 2^17 features on the tensor-core
    kernels (a 50 MB fragment table, 1024 stages): the morph, the log-det and
    the VJP on sampled samples against the oracle."""
    M = 1 << 17
    f = wl.random_field(63, wl.RFF, 7, M, wscale=6.0, bias=0.1)
    lo, hi = np.full(7, -np.pi), np.full(7, np.pi)
    L, _ = oracle.lipschitz(f)
    eta = float(np.float32(0.5 / L))
    fld = pdmp.DeviceField.from_host(f, lipschitz=L)
    N, T = 4096, 2
    x0 = wl.uniform_box(63, 3, N, lo, hi)
    gT = wl.f32(wl.rng(63, wl.S_COTANGENT).standard_normal((N, 7)))
    idx = np.arange(0, N, 171)
    xT = pdmp.morph(fld, dev(x0), T, eta).cpu().numpy()
    assert max_abs(xT[idx], oracle.morph(f, x0[idx], T, eta)) <= 1e-4
    ld = pdmp.logdet(fld, dev(x0), T, eta).cpu().numpy()
    ref_ld, _, _ = oracle.logdet(f, x0[idx], T, eta)
    assert max_abs(ld[idx], ref_ld) <= 1e-4 * T
    g0 = pdmp.morph_vjp(fld, dev(x0), T, eta, T, dev(gT)).cpu().numpy()
    r0 = oracle.morph_vjp(f, x0[idx], T, eta, gT[idx])
    assert np.linalg.norm(g0[idx] - r0) <= 1e-4 * np.linalg.norm(r0)
    assert pdmp.stream_status()[0] == 0


def test_rff_non_finite_samples_stay_local():
    """On the tensor-core kernels a NaN or infinite sample sits in one row of
    its 16 x 8 tiles: its own outputs are non-finite, every other sample's
    (also in its tiles and quads) match the oracle."""
    f = wl.random_field(64, wl.RFF, 7, 300, wscale=6.0, bias=0.1)
    lo, hi = np.full(7, -np.pi), np.full(7, np.pi)
    L, _ = oracle.lipschitz(f)
    eta = float(np.float32(0.5 / L))
    fld = pdmp.DeviceField.from_host(f, lipschitz=L)
    N, T = 512, 4
    x0 = wl.uniform_box(64, 3, N, lo, hi)
    bad = np.array([3, 11, 200, 511])
    x0[bad[0], 0] = np.nan
    x0[bad[1], 6] = np.inf
    x0[bad[2]] = -np.inf
    x0[bad[3], 3] = np.nan
    good = np.setdiff1d(np.arange(N), bad)
    out = pdmp.morph(fld, dev(x0), T, eta).cpu().numpy()
    assert not np.isfinite(out[bad]).all(axis=1).any()
    assert np.isfinite(out[good]).all()
    idx = good[::29]
    assert max_abs(out[idx], oracle.morph(f, x0[idx], T, eta)) <= 1e-4
    gT = np.ones((N, 7), np.float32)
    g0 = pdmp.morph_vjp(fld, dev(x0), T, eta, 2, dev(gT)).cpu().numpy()
    assert np.isfinite(g0[good]).all()
    r0 = oracle.morph_vjp(f, x0[idx], T, eta, gT[idx])
    assert np.linalg.norm(g0[idx] - r0) <= 1e-4 * np.linalg.norm(r0)
    assert pdmp.stream_status()[0] == 0


def test_clustered_samples_with_an_outlier():
    """Most samples in a tight blob and one far outlier that stretches the
    sort's bounding box, so many grid cells hold more than 64 samples and keep
    the scatter's arrival order: the tiles may then differ between runs, and the
    results are held only to the oracle's tolerance (two runs agree within it)."""
    f = wl.config1().field
    eta, L = rbf_eta(f, np.zeros(2), np.full(2, 10.0))
    fld = pdmp.DeviceField.from_host(f, lipschitz=L)
    N = 1 << 16
    g = wl.rng(63, 3)
    x0 = wl.f32(np.clip(5.0 + 0.05 * g.standard_normal((N, 2)), 0.0, 10.0))
    x0[N // 2] = (0.0, 10.0)                   # the outlier: the blob covers a few cells of the 2^14
    runs = [pdmp.morph(fld, dev(x0), 10, eta).cpu().numpy() for _ in range(2)]
    idx = np.r_[np.arange(0, N, 331), N // 2]
    ref = oracle.morph(f, x0[idx], 10, eta)
    for out in runs:
        assert np.isfinite(out).all()
        assert max_abs(out[idx], ref) <= 1e-4
    assert max_abs(runs[0], runs[1]) <= 1e-4
