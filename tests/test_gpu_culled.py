"""The spatially culled RBF morph: features farther than r_cut from a sample
tile are dropped, with r_cut from a certified truncation bound.  Checked
against the FP64 oracle (dense), the dense GPU morph, the work counter and the
edge cases of the grid (samples outside the centres' box, ragged tiles)."""
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
    assert pdmp.stream_status()[0] == 0


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def fitted_like_2d(M=16384, seed=2):
    lo, hi = np.zeros(2), np.full(2, 10.0)
    centres = wl.uniform_box(seed, wl.S_CENTRES, M, lo, hi)
    boxes = wl.random_boxes(seed, 64, lo, hi, 0.3, 1.5)
    f = wl.Field(wl.RBF, centres, wl.proxy_fitted_weights(seed, centres, boxes), gamma=8.0)
    return f, lo, hi


def test_cull_radius_bound():
    f, lo, hi = fitted_like_2d(M=4096)
    fld = pdmp.DeviceField.from_host(f)
    for eps in (1e-3, 1e-6, 1e-9):
        r, W = pdmp.cull_radius(fld, eps)
        assert abs(W - np.abs(f.w.astype(np.float64)).sum()) <= 1e-9 * W
        g = f.gamma
        assert r >= 1.0 / np.sqrt(2.0 * g)
        bound = lambda r: W * max(1.0, 2.0 * g * r) * np.exp(-g * r * r)
        assert bound(r) <= eps * (1 + 1e-9)
        assert bound(r * (1 - 1e-4)) > eps          # the smallest such radius


@pytest.mark.parametrize("d", [2, 3])
def test_culled_matches_oracle_and_dense(d):
    if d == 2:
        f, lo, hi = fitted_like_2d(M=8192)
        N, T = 20_000, 20
        eta, L = rbf_eta(f, lo - 0.5, hi + 0.5, cells=64)
    else:
        f = wl.random_field(78, wl.RBF, 3, 8192, lo=0, hi=8, gamma=8.0, wscale=1.0, bias=-0.2)
        lo, hi = np.zeros(3), np.full(3, 8.0)
        N, T = 20_000, 8
        eta, L = rbf_eta(f, lo - 0.5, hi + 0.5, cells=16)
    fld = pdmp.DeviceField.from_host(f, lipschitz=L)
    x0 = wl.uniform_box(90 + d, 3, N, lo, hi)
    r, _ = pdmp.cull_radius(fld, 1e-7)
    work = torch.zeros(1, dtype=torch.int64, device="cuda")
    xc = pdmp.morph_culled(fld, dev(x0), T, eta, r, work=work).cpu().numpy()
    xd = pdmp.morph(fld, dev(x0), T, eta).cpu().numpy()
    assert max_abs(xc, xd) <= 5e-5                # summation order differs from the dense kernel
    idx = np.sort(wl.rng(d, 11).choice(N, 200, replace=False))
    ref = oracle.morph(f, x0[idx], T, eta)
    assert max_abs(xc[idx], ref) <= 1e-4
    frac = int(work.item()) / (N * T * f.M)
    assert 0.0 < frac < 0.8                       # the grid does drop most far features
    # deterministic
    xc2 = pdmp.morph_culled(fld, dev(x0), T, eta, r).cpu().numpy()
    assert np.array_equal(xc, xc2)


def test_culled_radius_covering_everything_is_the_dense_sum():
    f, lo, hi = fitted_like_2d(M=2048)
    eta, L = rbf_eta(f, lo - 0.5, hi + 0.5, cells=64)
    fld = pdmp.DeviceField.from_host(f, lipschitz=L)
    N, T = 5000, 6
    x0 = wl.uniform_box(95, 3, N, lo, hi)
    work = torch.zeros(1, dtype=torch.int64, device="cuda")
    xc = pdmp.morph_culled(fld, dev(x0), T, eta, 100.0, work=work).cpu().numpy()
    assert int(work.item()) == N * T * f.M
    xd = pdmp.morph(fld, dev(x0), T, eta).cpu().numpy()
    assert max_abs(xc, xd) <= 1e-5


def test_culled_edges_outside_box_ragged_in_place_and_checkpoints():
    f, lo, hi = fitted_like_2d(M=4096, seed=5)
    eta, L = rbf_eta(f, lo - 6.0, hi + 6.0, cells=64)
    fld = pdmp.DeviceField.from_host(f, lipschitz=L)
    r, _ = pdmp.cull_radius(fld, 1e-7)
    T, k = 10, 5
    for N in (1, 255, 257, 3001):
        x0 = wl.uniform_box(100 + N, 3, N, lo - 5.0, hi + 5.0)   # many samples far outside the centres
        ck = torch.empty(T // k, N, 2, device="cuda")
        xin = dev(x0)
        out = pdmp.morph_culled(fld, xin, T, eta, r, out=xin, ckpt=ck, k=k)   # in place
        assert out.data_ptr() == xin.data_ptr()
        xc = xin.cpu().numpy()
        ref = oracle.morph(f, x0, T, eta)
        assert max_abs(xc, ref) <= 1e-4
        assert np.array_equal(ck[-1].cpu().numpy(), xc)
        refk = oracle.morph(f, x0, k, eta)
        assert max_abs(ck[0].cpu().numpy(), refk) <= 1e-4


@pytest.mark.parametrize("N", [1 << 18, 1 << 19])
def test_culled_fitted_shape_sampled_at_scale(N):
    """The fitted-like 2-D field (16,384 centres, T = 50) on sampled outputs:
    2^18 samples (the throughput measurement's size; under two waves of
    256-sample tiles, so the kernel takes 128-sample tiles) and 2^19 (256)."""
    f, lo, hi = fitted_like_2d()
    eta, L = rbf_eta(f, lo - 0.5, hi + 0.5, cells=128)
    fld = pdmp.DeviceField.from_host(f, lipschitz=L)
    T = 50
    x0 = wl.uniform_box(7, 3, N, lo, hi)
    r, _ = pdmp.cull_radius(fld, 1e-6)
    xc = pdmp.morph_culled(fld, dev(x0), T, eta, r).cpu().numpy()
    idx = np.sort(wl.rng(7, 12).choice(N, 96, replace=False))
    ref = oracle.morph(f, x0[idx], T, eta)
    assert max_abs(xc[idx], ref) <= 1e-4
