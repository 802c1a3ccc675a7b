"""The paper's own occupancy model (Sec. 3.1: tanh hidden layers, sigmoid
output) as the morph cost: queries, one Euler step (relative error of the
increment), the T-step morph against the FP64 oracle, ragged and in-place
launches, checkpoints and the certified Lipschitz bound."""
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


SHAPES = [(2, 64), (3, 64), (2, 32), (3, 32)]


def make(d, H, seed=3, gain=2.0):
    lo, hi = np.zeros(d), np.full(d, 10.0)
    net = wl.tanh_net(seed * 10 + d + H, d, H, lo=0.0, hi=10.0, gain=gain)
    L, G = oracle.tnet_lipschitz(net)
    eta = float(np.float32(0.5 / L))
    return net, lo, hi, L, eta


@pytest.mark.parametrize("d,H", SHAPES)
def test_query_matches_oracle(d, H):
    net, lo, hi, L, _ = make(d, H)
    dn = pdmp.DeviceTanhNet.from_host(net, lipschitz=L)
    x = wl.uniform_box(31, 3, 3000, lo - 1, hi + 1)
    c, s, g = (t.cpu().numpy() for t in pdmp.tanh_net_query(dn, dev(x)))
    r = oracle.tnet_evaluate(net, x)
    assert np.abs(s - r["s"]).max() <= 1e-5 * (1 + np.abs(r["s"]).max())
    assert np.abs(c - r["c"]).max() <= 1e-6
    scale = np.linalg.norm(r["grad"], axis=1).max()
    assert np.abs(g - r["grad"]).max() <= 1e-5 * scale


@pytest.mark.parametrize("d,H", SHAPES)
def test_one_step_relative_error_and_T_steps(d, H):
    net, lo, hi, L, eta = make(d, H)
    dn = pdmp.DeviceTanhNet.from_host(net, lipschitz=L)
    N = 4099                                                  # ragged: 64 tiles + 3
    x0 = wl.uniform_box(32, 3, N, lo, hi)
    x1 = pdmp.tanh_net_morph(dn, dev(x0), 1, eta).cpu().numpy()
    ref1 = oracle.tnet_morph(net, x0, 1, eta)
    inc, rinc = x1 - x0, ref1 - x0
    # relative error of the step's increment, per sample (FP32 rounding of x0 + inc aside)
    err = np.linalg.norm(inc - rinc, axis=1)
    ulp = np.abs(x0).max(axis=1) * 2.0 ** -23
    assert (err <= 1e-5 * np.linalg.norm(rinc, axis=1) + 2 * ulp).all()
    T = 30
    xT = pdmp.tanh_net_morph(dn, dev(x0), T, eta).cpu().numpy()
    idx = np.arange(0, N, 7)
    ref = oracle.tnet_morph(net, x0[idx], T, eta)
    assert max_abs(xT[idx], ref) <= 1e-4
    assert np.abs(xT - x0).max() > 1e-3                        # the samples do move
    again = pdmp.tanh_net_morph(dn, dev(x0), T, eta).cpu().numpy()
    assert np.array_equal(xT, again)


def test_edges_in_place_checkpoints_and_empty():
    net, lo, hi, L, eta = make(2, 64, seed=4)
    dn = pdmp.DeviceTanhNet.from_host(net, lipschitz=L)
    T, k = 12, 4
    for N in (1, 63, 64, 65):
        x0 = wl.uniform_box(40 + N, 3, N, lo, hi)
        xin = dev(x0)
        ck = torch.empty(T // k, N, 2, device="cuda")
        out = pdmp.tanh_net_morph(dn, xin, T, eta, out=xin, ckpt=ck, k=k)
        assert out.data_ptr() == xin.data_ptr()
        ref = oracle.tnet_morph(net, x0, T, eta)
        assert max_abs(xin.cpu().numpy(), ref) <= 1e-4
        assert np.array_equal(ck[-1].cpu().numpy(), xin.cpu().numpy())
        assert max_abs(ck[0].cpu().numpy(), oracle.tnet_morph(net, x0, k, eta)) <= 1e-4
    x0 = dev(wl.uniform_box(50, 3, 10, lo, hi))
    assert torch.equal(pdmp.tanh_net_morph(dn, x0, 0, eta), x0)
    empty = torch.empty(0, 2, device="cuda")
    assert pdmp.tanh_net_morph(dn, empty, 5, eta).shape == (0, 2)
    with pytest.raises(pdmp.PdmpError):
        pdmp.tanh_net_morph(dn, x0, 5, float(np.float32(1.5 / L)))     # eta L >= 1


@pytest.mark.parametrize("d,H", SHAPES)
def test_lipschitz_matches_oracle(d, H):
    net, _, _, L, _ = make(d, H, seed=5, gain=3.0)
    Lg, Gg = pdmp.tanh_net_lipschitz(pdmp.DeviceTanhNet.from_host(net))
    Lo, Go = oracle.tnet_lipschitz(net)
    assert abs(Lg - Lo) <= 1e-9 * Lo and abs(Gg - Go) <= 1e-9 * Go


def test_morph_at_scale_sampled():
    """2^18 samples, T = 50, the 2-D width-64 network: sampled against the oracle."""
    net, lo, hi, L, eta = make(2, 64, seed=6)
    dn = pdmp.DeviceTanhNet.from_host(net, lipschitz=L)
    N, T = 1 << 18, 50
    x0 = wl.uniform_box(60, 3, N, lo, hi)
    xT = pdmp.tanh_net_morph(dn, dev(x0), T, eta).cpu().numpy()
    idx = np.sort(wl.rng(60, 7).choice(N, 256, replace=False))
    ref = oracle.tnet_morph(net, x0[idx], T, eta)
    assert max_abs(xT[idx], ref) <= 1e-4
