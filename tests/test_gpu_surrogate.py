"""The learned surrogate: BF16 MLP forward and gradients against the FP64
oracle (same BF16 weights upcast), training on pairs the plain morph
generates, and inference with the plain morph as fallback and judge."""
import ctypes

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
    """The network's input: the oracle's Fourier encoding of the normalised
    coordinates u = (x - lo) s - 1, in FP64 with the network's own float32
    lo and s (pdmp_mlp carries them as float)."""
    lo = np.asarray(net.lo, np.float32).astype(np.float64)
    sc = np.asarray(net.in_scale, np.float32).astype(np.float64)
    u = (np.asarray(x, np.float64) - lo) * sc - 1.0
    return oracle.mlp_encode(u, 6)


def fp32_output_excess(net, x, y, f):
    """|y - (x + out_scale f)| beyond one unit in the last place of the
    float32 output y = x_T_hat (the interface returns x_0 + displacement in
    float32, whose rounding alone is about 5e-4 of a 5e-4 displacement)."""
    ref = np.asarray(x, np.float64) + f * np.asarray(net.out_scale)
    ulp = np.spacing(np.abs(np.asarray(y, np.float32))).astype(np.float64)
    return np.maximum(np.abs(np.asarray(y, np.float64) - ref) - ulp, 0.0)


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


def test_mlp_forward_fp32_activations_matches_oracle_to_1e4():
    """The FP32-activation mode: the same kernel and fragment layouts, every
    activation fed to the tensor cores as three BF16 pieces; the output equals
    the FP64 oracle's on the same BF16 weights to 1e-4 normwise (and on every
    sample to 1e-4 of the output's scale)."""
    net = pdmp.Surrogate(LO, HI, [0.05, 0.07, 0.03], seed=3)
    x = wl.uniform_box(13, 3, 1001, LO, HI)
    y = net.forward(torch.from_numpy(x).cuda(), fp32_act=True).cpu().numpy()
    _, bs = net.weights()
    f = oracle.mlp_forward(net.bf16_weights(), [b.astype(np.float64) for b in bs], normalised(net, x))
    excess = fp32_output_excess(net, x, y, f)
    disp = f * np.asarray(net.out_scale)
    assert np.linalg.norm(excess) <= 1e-4 * np.linalg.norm(disp)
    assert excess.max() <= 1e-4 * np.abs(disp).max()
    yb = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.linalg.norm(fp32_output_excess(net, x, yb, f)) > np.linalg.norm(excess)   # BF16 activations: coarser


@pytest.mark.parametrize("N", [1, 127, 129, 256 * 152 * 3 + 77])
def test_mlp_forward_ragged_and_many_tiles(N):
    """The tensor-core inference kernel over ragged sample counts (a partial
    128-sample tile, a partial pair of tiles) and over more tile pairs than
    CTAs (each CTA loops): sampled rows against the oracle in both modes, and
    every output finite."""
    net = pdmp.Surrogate(LO, HI, [0.05, 0.07, 0.03], seed=8)
    x = wl.uniform_box(18, 3, N, LO, HI)
    xd = torch.from_numpy(x).cuda()
    idx = np.unique(np.concatenate([wl.rng(18, 1).choice(N, min(N, 300), replace=False), [0, N - 1]]))
    _, bs = net.weights()
    f = oracle.mlp_forward(net.bf16_weights(), [b.astype(np.float64) for b in bs], normalised(net, x[idx]))
    for fp32_act, tol in ((False, 2e-2), (True, 1e-4)):
        y = net.forward(xd, fp32_act=fp32_act).cpu().numpy()
        assert np.isfinite(y).all()
        excess = fp32_output_excess(net, x[idx], y[idx], f)
        assert np.linalg.norm(excess) <= tol * np.linalg.norm(f * np.asarray(net.out_scale))
    assert pdmp.stream_status()[0] == 0


@pytest.mark.parametrize("fp32_act,tol", [(True, 1e-4), (False, 2e-2)])
@pytest.mark.parametrize("B", [1000, 4096])
def test_mlp_gradient_every_layer_matches_oracle(fp32_act, tol, B):
    """d loss / d(W_l, b_l) of every layer (the backward pass through each
    layer, and the tensor-core weight-gradient contraction of each) against
    the FP64 oracle on the same BF16 weights: 1e-4 relative per layer in the
    FP32-activation mode, 2e-2 with the BF16 activations of training.  B = 1000
    leaves a ragged last block of the weight-gradient kernel."""
    net = pdmp.Surrogate(LO, HI, [0.05, 0.07, 0.03], seed=6)
    x0 = wl.uniform_box(6, 3, B, LO, HI)
    xT = (x0 + 0.05 * wl.rng(6, 9).standard_normal((B, 3))).astype(np.float32)
    _, bs = net.weights()
    target = (xT.astype(np.float64) - x0) / np.asarray(net.out_scale)
    loss_ref, dW, db = oracle.mlp_loss_backward(net.bf16_weights(), [b.astype(np.float64) for b in bs],
                                                normalised(net, x0), target)
    loss, gW, gb = net.gradient(torch.from_numpy(x0).cuda(), torch.from_numpy(xT).cuda(), fp32_act=fp32_act)
    assert abs(float(loss.item()) - loss_ref) <= tol * loss_ref
    gW, gb = gW.cpu().numpy().astype(np.float64), gb.cpu().numpy().astype(np.float64)
    ow = ob = 0
    for layer, (rw, rb) in enumerate(zip(dW, db)):
        w = gW[ow:ow + rw.size].reshape(rw.shape)
        b = gb[ob:ob + rb.size]
        ow += rw.size
        ob += rb.size
        assert np.linalg.norm(w - rw) <= tol * np.linalg.norm(rw), f"layer {layer} weights"
        assert np.linalg.norm(b - rb) <= tol * np.linalg.norm(rb), f"layer {layer} biases"


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
    """A reduced 3-D world: config5's centres and boxes with M centres and
    weights of a fitted occupancy's sign structure (from the seeded generators,
    so that the oracle and the GPU take the same field); eta = 0.5 / L with L
    the oracle's certified bound."""
    wk = wl.config5(seed=seed, N=16, M=M, n_fit=16, n_train=N_train)
    f = wk.field.with_weights(wl.proxy_fitted_weights(seed, wk.field.centres, wk.boxes), bias=-0.5)
    wk.field = f
    eta, L = rbf_eta(f, LO - 0.5, HI + 0.5, cells=24)
    fld = pdmp.DeviceField.from_host(f, lipschitz=L)
    return wk, fld, eta, T


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
        ref = oracle.morph(wk.field, x0.cpu().numpy()[idx], T, eta)
        assert np.abs(o[idx] - ref).max() <= 1e-4


def test_culled_residual_check_matches_the_dense_check():
    """pdmp_surrogate_infer_culled: the residual check on the culled kernel
    (r_cut from cull_radius(f, 1e-6)) decides like the dense check except for
    samples within the culling margin of a threshold (s = 0 or step length =
    tau_r); accepted samples are the network's predictions and fallen-back
    ones the culled morph (bit for bit when every sample falls back), within
    the culled kernel's 1e-4 of the dense plain morph."""
    wk, fld, eta, T = _small_world(M=768)
    N = 20000
    x0 = torch.from_numpy(wl.uniform_box(23, 3, N, LO, HI)).cuda()
    net = pdmp.Surrogate(LO, HI, [0.02, 0.02, 0.02], seed=2)
    r_cut, _ = pdmp.cull_radius(fld, 1e-6)
    assert 0.0 < r_cut < 5.0                                   # the check really is culled
    pred = net.forward(x0)
    q = pdmp.occupancy_query(fld, pred, want=("s", "grad"))
    s = q["s"].cpu().numpy()
    slen = (eta * q["grad"]).norm(dim=1).cpu().numpy()
    plain = pdmp.morph(fld, x0, T, eta)
    culled = pdmp.morph_culled(fld, x0, T, eta, r_cut)
    # tau_r = 0: every sample falls back under both checks
    oc, nc = net.infer(fld, x0, T, eta, 0.0, r_cut=r_cut)
    od, nd = net.infer(fld, x0, T, eta, 0.0)
    assert nc == nd == N and torch.equal(od, plain) and torch.equal(oc, culled)
    assert (oc - od).abs().max().item() <= 1e-4
    for tau in (1e9, float(np.median(slen[s < 0]))):
        od, nd = net.infer(fld, x0, T, eta, tau)
        oc, nc = net.infer(fld, x0, T, eta, tau, r_cut=r_cut)
        fd = ~(od == pred).all(dim=1).cpu().numpy()
        fc = ~(oc == pred).all(dim=1).cpu().numpy()
        assert fd.sum() == nd and fc.sum() == nc
        assert 0 < nc < N
        differ = fd != fc
        near = (np.abs(s) <= 1e-4) | (np.abs(slen / tau - 1.0) <= 1e-3)
        assert np.all(near[differ]) and differ.sum() <= 5
        o_c, o_d, p_ = oc.cpu().numpy(), od.cpu().numpy(), plain.cpu().numpy()
        same = ~differ
        assert np.array_equal(o_c[same & ~fc], pred.cpu().numpy()[same & ~fc])
        # the fallback morphs its own subset (other tiles), on the culled kernel
        assert np.abs(o_c[same & fc] - p_[same & fc]).max() <= 1e-4
        assert np.abs(o_c[same] - o_d[same]).max() <= 1e-4
    L = pdmp._mlp_sigs()
    m, f = net.struct(), fld.struct()
    ws = torch.empty(int(L.pdmp_surrogate_workspace(ctypes.byref(f), N)), dtype=torch.uint8, device="cuda")
    out, nf = torch.empty_like(x0), ctypes.c_int64(0)
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        st = L.pdmp_surrogate_infer_culled(ctypes.byref(m), ctypes.byref(f), x0.data_ptr(), N, T, eta, 1.0, bad,
                                           out.data_ptr(), ctypes.byref(nf), ws.data_ptr(), ws.numel(), None)
        assert st == 1                                          # PDMP_ERR_INVALID_ARG
    assert pdmp.stream_status()[0] == 0


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


def test_residual_threshold_matches_oracle():
    """tau_r (pdmp_residual_threshold): the nearest-rank q-quantile of the last
    step's length over the training samples, against the oracle's from its own
    FP64 chain.  A k-th order statistic moves by at most the largest change of
    any one value; a length changes by at most eta L |dx| <= 0.5 sqrt(3) 1e-4
    when x_{T-1} moves by the final-position tolerance 1e-4 per coordinate,
    plus the per-step error of the increment (1e-5 of its scale), so the two
    thresholds agree to 1e-4.  x_T agrees with the plain morph's to 1e-5 (its
    last step runs on tiles re-sorted at x_{T-1}, whose frames change only the
    rounding) and with the oracle's to the final-position tolerance 1e-4."""
    wk, fld, eta, T = _small_world(N_train=1 << 14)
    x0 = wk.extra["x_train"]
    xd = torch.from_numpy(x0).cuda()
    taus = {q: pdmp.residual_threshold(fld, xd, T, eta, q) for q in (0.5, 0.99, 1.0)}
    tau, xT = taus[0.99]
    xm = pdmp.morph(fld, xd, T, eta)
    assert float((xT - xm).abs().max()) <= 1e-5
    xprev = oracle.morph(wk.field, x0, T - 1, eta)
    rT = oracle.morph(wk.field, xprev, 1, eta)
    assert np.abs(xT.cpu().numpy() - rT).max() <= 1e-4
    lengths = np.linalg.norm(eta * oracle.evaluate(wk.field, xprev)["grad"], axis=1)
    srt = np.sort(lengths)
    n = len(srt)
    for q, (t, _) in taus.items():
        ref = srt[int(np.ceil(q * n)) - 1]
        assert abs(t - ref) <= 1e-4, (q, t, ref)
    assert taus[0.5][0] <= taus[0.99][0] <= taus[1.0][0]
    assert srt[-1] > 10 * 1e-4                       # the tolerance is small against the lengths


def test_surrogate_gains_over_the_plain_morph_at_equal_collision_rate():
    """What the trained network gains over the method without it, at a
    reduced size (3-D, M = 2048 centres, T = 40; 2^16 training pairs from the
    plain morph; inference on 2^20 samples): the surrogate with its residual
    check and plain-morph fallback is several times faster than the plain
    morph, and its ground-truth collision rate (samples inside an obstacle box)
    is at most the plain morph's + 0.1 percentage points."""
    wk, fld, eta, _ = _small_world(M=2048, N_train=1 << 16)
    T = 40
    xtr = torch.from_numpy(wk.extra["x_train"]).cuda()
    tau_r, xTtr = pdmp.residual_threshold(fld, xtr, T, eta, 0.99)
    net = pdmp.Surrogate(LO, HI, pdmp.displacement_rms(xtr, xTtr).cpu().numpy(), seed=5)
    B, steps = 4096, 800
    for s in range(steps):
        lr = 2e-3 * 0.5 * (1.0 + np.cos(np.pi * s / steps)) + 1e-5
        i = (s * B) % (xtr.shape[0] - B)
        net.train_step(xtr[i:i + B], xTtr[i:i + B], lr=lr)
    x0 = torch.from_numpy(wl.uniform_box(55, 3, 1 << 20, LO, HI)).cuda()
    boxes = torch.from_numpy(wk.boxes).cuda()
    ws = torch.empty(pdmp.morph_workspace(fld, x0.shape[0]), dtype=torch.uint8, device="cuda")
    plain = torch.empty_like(x0)
    sur = torch.empty_like(x0)
    run_plain = lambda: pdmp.morph(fld, x0, T, eta, out=plain, ws=ws)
    res = {}

    def run_sur():
        res["nf"] = net.infer(fld, x0, T, eta, tau_r, out=sur)[1]

    def best(fn, reps=3):
        fn()
        times = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        return min(times)
    t_plain, t_sur = best(run_plain), best(run_sur)
    col = lambda x: float(pdmp.box_labels(boxes, x).float().mean().item())
    c_prior, c_plain, c_sur = col(x0), col(plain), col(sur)
    assert c_plain < c_prior                            # the morph moves samples out of the obstacles
    assert c_sur <= c_plain + 1e-3, (c_sur, c_plain)
    assert res["nf"] < 0.1 * x0.shape[0]
    assert t_plain / t_sur >= 4.0, (t_plain, t_sur)
