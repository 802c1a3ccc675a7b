"""The learned surrogate: BF16 MLP forward and gradients against the FP64
oracle (same BF16 weights upcast), training on pairs the plain morph
generates, and inference with the plain morph as fallback and judge."""
import numpy as np
import pytest
import torch

import oracle
import paper_2108_11775_gb300 as pdmp
import workloads as wl
from gpu_util import rbf_eta, setup_oracle_threads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available()
    setup_oracle_threads()
    yield
    assert pdmp.stream_status()[0] == 0


LO, HI = np.zeros(3), np.full(3, 5.0)


def normalised(net, x):
    """The network's input: the oracle's Fourier encoding of the normalised coordinates."""
    u = (np.asarray(x, np.float64) - np.asarray(net.lo)) * np.asarray(net.in_scale) - 1.0
    return oracle.mlp_encode(u, 6)


def test_mlp_forward_matches_oracle():
    net = pdmp.Surrogate(LO, HI, [0.05, 0.07, 0.03], seed=3)
    x = wl.uniform_box(3, 3, 1000, LO, HI)
    y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    Ws = net.bf16_weights()
    _, bs = net.weights()
    f = oracle.mlp_forward(Ws, [b.astype(np.float64) for b in bs], normalised(net, x))
    ref = x.astype(np.float64) + f * np.asarray(net.out_scale)
    pred = (y - x) / np.asarray(net.out_scale)
    assert np.linalg.norm(pred - f) <= 2e-2 * np.linalg.norm(f)
    assert np.abs(y - ref).max() <= 2e-2 * np.abs(ref - x).max() + 1e-6


def test_mlp_train_step_gradient_matches_oracle():
    net = pdmp.Surrogate(LO, HI, [0.05, 0.07, 0.03], seed=4)
    B = 512
    x0 = wl.uniform_box(4, 3, B, LO, HI)
    xT = (x0 + 0.05 * wl.rng(4, 9).standard_normal((B, 3))).astype(np.float32)
    Ws = net.bf16_weights()
    _, bs = net.weights()
    target = (xT.astype(np.float64) - x0) / np.asarray(net.out_scale)
    loss_ref, dW, db = oracle.mlp_loss_backward(Ws, [b.astype(np.float64) for b in bs], normalised(net, x0), target)
    loss = torch.zeros(1, device="cuda")
    net.train_step(torch.from_numpy(x0).cuda(), torch.from_numpy(xT).cuda(), loss=loss)
    assert abs(float(loss.item()) - loss_ref) <= 2e-2 * loss_ref
    # after the first Adam step the first moment is (1 - beta1) * gradient
    m = net.adam[:pdmp.MLP_NW].cpu().numpy().astype(np.float64) / 0.1
    g_ref = np.concatenate([d.ravel() for d in dW])
    assert np.linalg.norm(m - g_ref) <= 2e-2 * np.linalg.norm(g_ref)
    mb = net.adam[2 * pdmp.MLP_NW:2 * pdmp.MLP_NW + pdmp.MLP_NB].cpu().numpy().astype(np.float64) / 0.1
    gb_ref = np.concatenate([d.ravel() for d in db])
    assert np.linalg.norm(mb - gb_ref) <= 2e-2 * np.linalg.norm(gb_ref)


def _small_world(M=1024, N_train=1 << 15, T=20, seed=5):
    wk = wl.config5(seed=seed, N=16, M=M, n_fit=20_000, n_train=N_train)
    fld = pdmp.DeviceField.from_host(wk.field)
    w, b, _, _ = pdmp.fit_occupancy(fld, torch.from_numpy(wk.fit_X).cuda(), torch.from_numpy(wk.fit_y).cuda(),
                                    1e-4, 20, 150)
    fitted = fld.with_weights(w, bias=b)
    L, _ = pdmp.lipschitz_bound(fitted, LO - 0.5, HI + 0.5, cells=24)
    eta = float(np.float32(0.5 / L))
    fitted.lipschitz = L
    return wk, fitted, eta, T


def test_surrogate_learns_the_displacement_and_beats_the_identity():
    wk, fld, eta, T = _small_world()
    x0 = torch.from_numpy(wk.extra["x_train"]).cuda()
    xT = pdmp.morph(fld, x0, T, eta)
    scale = pdmp.displacement_rms(x0, xT).cpu().numpy()
    net = pdmp.Surrogate(LO, HI, scale, seed=1)
    loss = torch.zeros(1, device="cuda")
    B = 4096
    first = None
    for step in range(600):
        i = (step * B) % (x0.shape[0] - B)
        net.train_step(x0[i:i + B].contiguous(), xT[i:i + B].contiguous(), lr=2e-3, loss=loss)
        if first is None:
            first = float(loss.item())
    last = float(loss.item())
    assert np.isfinite(last) and last < 0.5 * first
    xv = torch.from_numpy(wl.uniform_box(77, 3, 8192, LO, HI)).cuda()
    plain = pdmp.morph(fld, xv, T, eta)
    pred = net.forward(xv)
    err_net = float((pred - plain).norm())
    err_identity = float((xv - plain).norm())          # the method without the network: x_T ~ x_0
    assert err_net < 0.7 * err_identity


def test_surrogate_inference_fallback_is_the_plain_morph():
    wk, fld, eta, T = _small_world(M=768)
    x0 = torch.from_numpy(wl.uniform_box(21, 3, 5000, LO, HI)).cuda()
    net = pdmp.Surrogate(LO, HI, [0.02, 0.02, 0.02], seed=2)
    plain = pdmp.morph(fld, x0, T, eta)
    # tau_r = 0: every sample fails the check and comes from the plain morph
    out, nf = net.infer(fld, x0, T, eta, tau_r=0.0)
    assert nf == x0.shape[0]
    assert torch.equal(out, plain)
    # a generous tau_r: only predictions in predicted-occupied space fall back
    out, nf = net.infer(fld, x0, T, eta, tau_r=1e9)
    pred = net.forward(x0)
    s = pdmp.occupancy_query(fld, pred, want=("s",))["s"]
    fell = (s >= 0).cpu().numpy()
    assert nf == int(fell.sum())
    o, p, q = out.cpu().numpy(), plain.cpu().numpy(), pred.cpu().numpy()
    assert np.array_equal(o[fell], p[fell])
    assert np.array_equal(o[~fell], q[~fell])
    # the oracle judges a few fallen-back samples
    idx = np.flatnonzero(fell)[:8]
    if idx.size:
        ref = oracle.morph(wk.field.with_weights(fld.w.cpu().numpy(), bias=fld.bias), x0.cpu().numpy()[idx], T, eta)
        assert np.abs(o[idx] - ref).max() <= 1e-4


def test_save_and_load_round_trip(tmp_path):
    net = pdmp.Surrogate(LO, HI, [0.05, 0.07, 0.03], seed=9)
    x0 = torch.from_numpy(wl.uniform_box(9, 3, 4096, LO, HI)).cuda()
    xT = x0 + 0.01
    for _ in range(3):
        net.train_step(x0, xT)
    path = str(tmp_path / "net.bin")
    net.save(path)
    other = pdmp.Surrogate.load(path)
    assert torch.equal(net.forward(x0), other.forward(x0))
    net.train_step(x0, xT)
    other.train_step(x0, xT)                 # Adam moments and step restored: the next step agrees
    assert torch.equal(net.W, other.W) and torch.equal(net.adam, other.adam)
