"""Pins the FP64 oracle to things other than itself (no GPU needed).

Each test checks the oracle against something it does not share code with:
symbolic derivatives (sympy), central finite differences of the oracle's own
lower-order outputs, a textbook solver (scikit-learn's logistic regression),
torch's float64 autograd, invariants of the method (w = 0 is the identity,
translation covariance, det > 0 under eta L < 1, inverse round trip) and
hand-built label cases.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as wl


# --------------------------------------------------------------------------
# sigmoid and its derivatives (Sec. 3.1: sigmoid output layer)
def test_sigmoid_derivatives_match_sympy_and_maxima():
    sp = pytest.importorskip("sympy")
    s = sp.symbols("s")
    sig = 1 / (1 + sp.exp(-s))
    d1, d2 = sp.diff(sig, s), sp.diff(sig, s, 2)
    f0, f1, f2 = (sp.lambdify(s, e, "math") for e in (sig, d1, d2))
    for v in np.linspace(-30, 30, 121):
        got = oracle.sigmoid3(v)
        for g, ref in zip(got, (f0(v), f1(v), f2(v))):
            assert abs(g - ref) <= 1e-15 + 1e-12 * abs(ref)
    # maxima used by the Lipschitz bound: max sigma' = 1/4, max |sigma''| = 1/(6 sqrt 3)
    crit = sp.solve(sp.diff(d2, s), s)
    best = max(abs(float(d2.subs(s, c))) for c in crit if c.is_real)
    assert abs(best - 1 / (6 * math.sqrt(3))) < 1e-14
    grid = np.linspace(-20, 20, 40001)
    vals = np.array([oracle.sigmoid3(v) for v in grid[::40]])
    assert vals[:, 1].max() <= 0.25 + 1e-15
    assert np.abs(vals[:, 2]).max() <= 1 / (6 * math.sqrt(3)) + 1e-15


# --------------------------------------------------------------------------
# single-feature closed forms (Sec. 3.1) against sympy
def _sympy_cost(kind, d, centre, phase, gamma, w, bias):
    sp = pytest.importorskip("sympy")
    xs = sp.symbols(f"x0:{d}")
    if kind == wl.RBF:
        phi = sp.exp(-gamma * sum((xs[i] - centre[i]) ** 2 for i in range(d)))
    else:
        phi = sp.cos(sum(centre[i] * xs[i] for i in range(d)) + phase)
    c = 1 / (1 + sp.exp(-(w * phi + bias)))
    grad = [sp.diff(c, xi) for xi in xs]
    hess = [[sp.diff(g, xj) for xj in xs] for g in grad]
    return (sp.lambdify(xs, c, "math"), [sp.lambdify(xs, g, "math") for g in grad],
            [[sp.lambdify(xs, h, "math") for h in row] for row in hess])


@pytest.mark.parametrize("kind,d", [(wl.RBF, 2), (wl.RBF, 3), (wl.RFF, 3)])
def test_single_feature_gradient_and_hessian_match_sympy(kind, d):
    g = wl.rng(11, 1)
    centre = [float(v) for v in g.uniform(-1, 1, d)]
    phase = float(g.uniform(0, 6.28))
    gamma, w, bias = 1.7, 2.3, -0.4
    fld = wl.Field(kind, np.array([centre]), np.array([w]), gamma=gamma,
                   phase=np.array([phase]) if kind == wl.RFF else None, bias=bias)
    cf, gf, hf = _sympy_cost(kind, d, centre, phase, gamma, w, bias)
    X = g.uniform(-1.5, 1.5, (25, d))
    out = oracle.evaluate(fld, X, hess=True)
    for n, x in enumerate(X):
        assert abs(out["c"][n] - cf(*x)) < 1e-14
        for i in range(d):
            ref = gf[i](*x)
            assert abs(out["grad"][n, i] - ref) <= 1e-14 + 1e-11 * abs(ref)
            for j in range(d):
                ref = hf[i][j](*x)
                assert abs(out["hess"][n, i, j] - ref) <= 1e-13 + 1e-10 * abs(ref)
    # with one feature the absolute-sum scale equals |grad c| exactly
    np.testing.assert_allclose(out["scale"], np.linalg.norm(out["grad"], axis=1), rtol=1e-13, atol=1e-300)


# --------------------------------------------------------------------------
# many features: central finite differences of c and of grad c
@pytest.mark.parametrize("kind,d,M", [(wl.RBF, 2, 40), (wl.RBF, 3, 40), (wl.RFF, 7, 60)])
def test_gradient_and_hessian_match_central_differences(kind, d, M):
    fld = wl.random_field(5, kind, d, M, lo=0, hi=3, gamma=2.0, wscale=1.5 if kind == wl.RBF else 8.0, bias=0.3)
    X = wl.uniform_box(7, 3, 12, np.zeros(d), np.full(d, 3.0)).astype(np.float64)
    out = oracle.evaluate(fld, X, hess=True)
    h = 1e-5
    for i in range(d):
        e = np.zeros(d)
        e[i] = h
        cp = oracle.evaluate(fld, X + e)
        cm = oracle.evaluate(fld, X - e)
        fd_g = (cp["c"] - cm["c"]) / (2 * h)
        np.testing.assert_allclose(out["grad"][:, i], fd_g, rtol=1e-6, atol=1e-10)
        fd_h = (cp["grad"] - cm["grad"]) / (2 * h)
        np.testing.assert_allclose(out["hess"][:, :, i], fd_h, rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(out["hess"], np.swapaxes(out["hess"], 1, 2), atol=1e-14)
    # triangle inequality: the absolute-sum scale dominates |grad c|
    assert np.all(out["scale"] >= np.linalg.norm(out["grad"], axis=1) * (1 - 1e-12))


# --------------------------------------------------------------------------
# morph: Eq. (1) with Euler steps
def test_morph_zero_weights_is_identity():
    fld = wl.random_field(3, wl.RBF, 2, 50).with_weights(np.zeros(50), bias=0.7)
    x0 = wl.uniform_box(3, 3, 100, [0, 0], [10, 10])
    xT = oracle.morph(fld, x0, 25, 0.3)
    assert np.array_equal(xT, x0.astype(np.float64))


def test_morph_scalar_recurrence_matches_sympy_iteration():
    sp = pytest.importorskip("sympy")
    x = sp.symbols("x")
    mu, gamma, w, b = 0.3, 3.0, -1.8, 0.2
    c = 1 / (1 + sp.exp(-(w * sp.exp(-gamma * (x - mu) ** 2) + b)))
    dc = sp.lambdify(x, sp.diff(c, x), "math")
    fld = wl.Field(wl.RBF, np.array([[mu]]), np.array([w]), gamma=gamma, bias=b)
    eta, T = 0.05, 40
    starts = np.linspace(-1.0, 1.5, 11)
    got = oracle.morph(fld, starts[:, None], T, eta)[:, 0]
    for s0, g in zip(starts, got):
        v = float(s0)
        for _ in range(T):
            v = v - eta * dc(v)
        assert abs(g - v) < 1e-13


def test_morph_one_step_uses_finite_difference_gradient():
    fld = wl.random_field(8, wl.RBF, 3, 30, lo=0, hi=2, gamma=3.0, wscale=2.0)
    x0 = wl.uniform_box(8, 3, 20, np.zeros(3), np.full(3, 2.0)).astype(np.float64)
    eta, h = 0.02, 1e-5
    fd = np.zeros_like(x0)
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        fd[:, i] = (oracle.evaluate(fld, x0 + e)["c"] - oracle.evaluate(fld, x0 - e)["c"]) / (2 * h)
    np.testing.assert_allclose(oracle.morph(fld, x0, 1, eta), x0 - eta * fd, rtol=0, atol=1e-10)


def test_morph_translation_covariant():
    fld = wl.random_field(4, wl.RBF, 2, 64, gamma=4.0)
    x0 = wl.uniform_box(4, 3, 50, [0, 0], [10, 10]).astype(np.float64)
    v = np.array([3.25, -1.5])
    moved = wl.Field(wl.RBF, fld.centres.astype(np.float64) + v, fld.w, gamma=fld.gamma)
    a = oracle.morph(fld, x0, 10, 0.01)
    b = oracle.morph(moved, x0 + v, 10, 0.01)
    np.testing.assert_allclose(b - v, a, atol=1e-12)


def test_morph_trajectory_consistent_with_final():
    fld = wl.random_field(6, wl.RFF, 7, 32)
    x0 = wl.uniform_box(6, 3, 9, np.full(7, -np.pi), np.full(7, np.pi))
    tr = oracle.morph(fld, x0, 6, 0.01, traj=True)
    assert np.array_equal(tr[:, 0], x0.astype(np.float64))
    np.testing.assert_array_equal(tr[:, -1], oracle.morph(fld, x0, 6, 0.01))
    np.testing.assert_array_equal(tr[:, 3], oracle.morph(fld, x0, 3, 0.01))


# --------------------------------------------------------------------------
# Lipschitz bound, step size and the diffeomorphism invariant
def _config1_eta():
    w1 = wl.config1()
    L, G = oracle.lipschitz(w1.field, w1.lo, w1.hi, cells=64)
    return w1, L, G


def test_rbf_lipschitz_bound_dominates_sampled_hessian_norm():
    w1, L, G = _config1_eta()
    pts = wl.uniform_box(21, 3, 20000, w1.lo, w1.hi).astype(np.float64)
    out = oracle.evaluate(w1.field, pts, hess=True)
    hn = np.abs(np.linalg.eigvalsh(out["hess"])).max(axis=1)
    gn = np.linalg.norm(out["grad"], axis=1)
    assert hn.max() <= L
    assert gn.max() <= G
    assert L < 50 * hn.max()          # certified but not useless
    # a finer cell grid can only tighten (never loosen by more than rounding) the bound
    L2, _ = oracle.lipschitz(w1.field, w1.lo, w1.hi, cells=128)
    assert hn.max() <= L2 <= L * (1 + 1e-12)


def test_rbf_lipschitz_single_centre_envelopes():
    # one centre, w = 1, no bias: at r = 0 |Hess s| = 2 gamma, grad s = 0, sigma'(1) known
    gamma = 2.5
    fld = wl.Field(wl.RBF, np.array([[0.0, 0.0]]), np.array([1.0]), gamma=gamma)
    L, G = oracle.lipschitz(fld, [-0.01, -0.01], [0.01, 0.01], cells=1)
    # the bound on a cell around the centre is 1/4 * 2 gamma + (1/(6 sqrt3)) * h1(0.01*sqrt2)^2
    r = 0.01 * math.sqrt(2)
    h1 = 2 * gamma * r * math.exp(-gamma * r * r)
    assert abs(L - (0.25 * 2 * gamma + h1 ** 2 / (6 * math.sqrt(3)))) < 1e-12
    # far from the centre the h1 envelope peaks at r = 1/sqrt(2 gamma)
    L3, G3 = oracle.lipschitz(fld, [-3, -3], [3, 3], cells=1)
    assert abs(G3 - 0.25 * 2 * gamma / math.sqrt(2 * gamma) * math.exp(-0.5)) < 1e-12


def test_rff_lipschitz_bound_dominates_sampled_hessian_norm():
    fld = wl.random_field(9, wl.RFF, 7, 128)
    L, G = oracle.lipschitz(fld)
    pts = wl.uniform_box(9, 4, 3000, np.full(7, -np.pi), np.full(7, np.pi))
    out = oracle.evaluate(fld, pts, hess=True)
    assert np.abs(np.linalg.eigvalsh(out["hess"])).max() <= L
    assert np.linalg.norm(out["grad"], axis=1).max() <= G


def test_det_positive_at_every_step_when_eta_L_below_one():
    w1, L, _ = _config1_eta()
    eta = float(np.float32(0.5 / L))
    ld, xT, md = oracle.logdet(w1.field, w1.x0[:512], w1.T, eta)
    assert np.all(md > 0)
    # eigenvalues of I - eta H lie in (1 - eta L, 1 + eta L) => per-step det bounds
    d = 2
    assert np.all(ld >= w1.T * d * math.log(1 - eta * L) - 1e-12)
    assert np.all(ld <= w1.T * d * math.log(1 + eta * L) + 1e-12)
    np.testing.assert_array_equal(xT, oracle.morph(w1.field, w1.x0[:512], w1.T, eta))


# --------------------------------------------------------------------------
# inverse: Eq. (2)
def test_inverse_round_trip():
    w1, L, _ = _config1_eta()
    eta = 0.5 / L
    x0 = w1.x0[:64].astype(np.float64)
    z = oracle.morph(w1.field, x0, 10, eta)
    y, its = oracle.morph_inverse(w1.field, z, 10, eta, tol=1e-14, maxit=200)
    assert np.abs(y - x0).max() <= 1e-10
    assert its.max() < 200
    assert np.abs(z - x0).max() > 1e-3        # the map did move the samples


# --------------------------------------------------------------------------
# VJP, parameter gradient and log-det against the finite-difference Jacobian
def _fd_jacobian(fld, x0, T, eta, h=1e-6):
    N, d = x0.shape
    J = np.zeros((N, d, d))
    for j in range(d):
        e = np.zeros(d)
        e[j] = h
        J[:, :, j] = (oracle.morph(fld, x0 + e, T, eta) - oracle.morph(fld, x0 - e, T, eta)) / (2 * h)
    return J


@pytest.mark.parametrize("kind,d", [(wl.RBF, 2), (wl.RBF, 3), (wl.RFF, 7)])
def test_vjp_and_logdet_match_fd_jacobian(kind, d):
    if kind == wl.RBF:
        fld = wl.random_field(12, kind, d, 60, lo=0, hi=3, gamma=3.0, wscale=2.0, bias=-0.2)
        L, _ = oracle.lipschitz(fld, np.full(d, -1.0), np.full(d, 4.0), cells=24 if d == 2 else 10)
        x0 = wl.uniform_box(12, 3, 6, np.zeros(d), np.full(d, 3.0)).astype(np.float64)
    else:
        fld = wl.random_field(12, kind, d, 48, wscale=6.0)
        L, _ = oracle.lipschitz(fld)
        x0 = wl.uniform_box(12, 3, 6, np.full(d, -np.pi), np.full(d, np.pi)).astype(np.float64)
    eta, T = 0.5 / L, 8
    J = _fd_jacobian(fld, x0, T, eta)
    gT = wl.rng(12, 5).standard_normal(x0.shape)
    g0 = oracle.morph_vjp(fld, x0, T, eta, gT)
    np.testing.assert_allclose(g0, np.einsum("nij,ni->nj", J, gT), rtol=1e-6, atol=1e-8)
    ld, _, md = oracle.logdet(fld, x0, T, eta)
    np.testing.assert_allclose(ld, np.linalg.slogdet(J)[1], atol=1e-7)
    assert np.all(md > 0)
    assert np.all(np.linalg.slogdet(J)[0] > 0)


@pytest.mark.parametrize("kind,d", [(wl.RBF, 2), (wl.RFF, 5)])
def test_weight_and_bias_gradient_match_fd(kind, d):
    if kind == wl.RBF:
        fld = wl.random_field(13, kind, d, 20, lo=0, hi=2, gamma=2.0, wscale=2.0, bias=0.1)
        x0 = wl.uniform_box(13, 3, 5, np.zeros(d), np.full(d, 2.0)).astype(np.float64)
    else:
        fld = wl.random_field(13, kind, d, 20, wscale=4.0, bias=0.1)
        x0 = wl.uniform_box(13, 3, 5, np.full(d, -np.pi), np.full(d, np.pi)).astype(np.float64)
    T, eta = 6, 0.05
    gT = wl.rng(13, 5).standard_normal(x0.shape)
    _, gw, gb = oracle.morph_vjp(fld, x0, T, eta, gT, want_gw=True)
    w = fld.w.astype(np.float64)
    h = 1e-6

    def objective(wv, bv):
        f2 = wl.Field(fld.kind, fld.centres, wv, gamma=fld.gamma, phase=fld.phase, bias=bv)
        return float(np.sum(gT * oracle.morph(f2, x0, T, eta)))

    for m in (0, 3, 7, 19):
        e = np.zeros_like(w)
        e[m] = h
        fd = (objective(w + e, fld.bias) - objective(w - e, fld.bias)) / (2 * h)
        assert abs(gw[m] - fd) <= 1e-7 + 1e-6 * abs(fd)
    fd_b = (objective(w, fld.bias + h) - objective(w, fld.bias - h)) / (2 * h)
    assert abs(gb - fd_b) <= 1e-7 + 1e-6 * abs(fd_b)


# --------------------------------------------------------------------------
# the occupancy fit (Sec. 3.1): BCE by gradient descent
def _small_fit_problem(n=1500, side=8):
    g = np.linspace(0, 10, side)
    gx, gy = np.meshgrid(g, g, indexing="ij")
    centres = np.stack([gx.ravel(), gy.ravel()], 1).astype(np.float32)
    fld = wl.Field(wl.RBF, centres, np.zeros(centres.shape[0], np.float32), gamma=0.5)
    boxes = wl.random_boxes(31, 6, [0, 0], [10, 10], 1.0, 3.0)
    X = wl.uniform_box(31, wl.S_POINTS, n, [0, 0], [10, 10])
    y = wl.inside_boxes(boxes, X)
    return fld, X, y


def test_fit_objective_gradient_matches_fd():
    fld, X, y = _small_fit_problem(n=300, side=4)
    w = wl.rng(1, 1).standard_normal(fld.M)
    l2 = 1e-2
    loss, gw, gb = oracle.fit_objective(fld, X, y, l2, w, 0.3)
    h = 1e-6
    for m in range(fld.M):
        e = np.zeros(fld.M)
        e[m] = h
        fd = (oracle.fit_objective(fld, X, y, l2, w + e, 0.3)[0] - oracle.fit_objective(fld, X, y, l2, w - e, 0.3)[0]) / (2 * h)
        assert abs(gw[m] - fd) < 1e-8
    fdb = (oracle.fit_objective(fld, X, y, l2, w, 0.3 + h)[0] - oracle.fit_objective(fld, X, y, l2, w, 0.3 - h)[0]) / (2 * h)
    assert abs(gb - fdb) < 1e-8


def test_fit_converges_to_textbook_logistic_regression():
    skl = pytest.importorskip("sklearn.linear_model")
    fld, X, y = _small_fit_problem()
    l2 = 1e-3
    w, b, loss, alpha = oracle.fit(fld, X, y, l2, power_iters=50, iters=3000)
    Phi = np.exp(-fld.gamma * ((X.astype(np.float64)[:, None, :] - fld.centres.astype(np.float64)[None]) ** 2).sum(-1))
    ref = skl.LogisticRegression(C=1.0 / (len(y) * l2), tol=1e-12, max_iter=100000).fit(Phi, y)
    np.testing.assert_allclose(w, ref.coef_[0], rtol=0, atol=2e-4 * np.abs(ref.coef_).max())
    assert abs(b - ref.intercept_[0]) < 2e-4 * max(1.0, abs(ref.intercept_[0]))
    # KKT: the gradient vanishes at the optimum
    _, gw, gb = oracle.fit_objective(fld, X, y, l2, w, b)
    assert np.abs(gw).max() < 1e-6 and abs(gb) < 1e-6
    assert alpha > 0


def test_fit_power_iteration_step_is_the_curvature_bound():
    fld, X, y = _small_fit_problem(n=400, side=5)
    l2 = 1e-3
    _, _, _, alpha = oracle.fit(fld, X, y, l2, power_iters=200, iters=0)
    Phi = np.exp(-fld.gamma * ((X.astype(np.float64)[:, None, :] - fld.centres.astype(np.float64)[None]) ** 2).sum(-1))
    A = np.concatenate([Phi, np.ones((len(X), 1))], 1)
    lam = np.linalg.eigvalsh(A.T @ A / len(X)).max()
    assert abs(alpha - 1.0 / (0.25 * lam + l2)) < 1e-9 * alpha


# --------------------------------------------------------------------------
# ground-truth labels from closed boxes
def test_box_labels_closed_boundaries():
    boxes = np.array([[1.0, 1.0, 2.0, 3.0], [5.0, 5.0, 5.0, 5.0]], np.float32)  # lo.., hi..
    up = np.nextafter(np.float32(2.0), np.float32(3.0))
    dn = np.nextafter(np.float32(1.0), np.float32(0.0))
    pts = np.array([[1.0, 1.0], [2.0, 3.0], [1.5, 2.0], [up, 2.0], [dn, 2.0], [1.5, 3.0000002],
                    [5.0, 5.0], [5.0, np.nextafter(np.float32(5.0), np.float32(6.0))], [0, 0], [2.0, 1.0]], np.float32)
    want = np.array([1, 1, 1, 0, 0, 0, 1, 0, 0, 1], np.uint8)
    np.testing.assert_array_equal(oracle.box_labels(boxes, pts), want)
    assert oracle.box_labels(np.zeros((0, 4), np.float32), pts).sum() == 0


def test_box_labels_3d_corner_cases():
    boxes = np.array([[0, 0, 0, 1, 1, 1]], np.float32)
    pts = np.array([[0, 0, 0], [1, 1, 1], [1, 1, 1.0000001], [-0.0, 0.5, 1], [0.5, 0.5, -1e-30]], np.float32)
    np.testing.assert_array_equal(oracle.box_labels(boxes, pts), [1, 1, 0, 1, 0])


# --------------------------------------------------------------------------
# surrogate MLP against torch float64 autograd and finite differences
def test_mlp_loss_and_gradients_match_torch_autograd():
    torch = pytest.importorskip("torch")
    g = wl.rng(40, 1)
    widths = [3, 16, 16, 16, 3]
    Ws = [g.standard_normal((widths[i + 1], widths[i])) * 0.5 for i in range(4)]
    Bs = [g.standard_normal(widths[i + 1]) * 0.1 for i in range(4)]
    X = g.standard_normal((37, 3))
    Y = g.standard_normal((37, 3))
    loss, dW, dB = oracle.mlp_loss_backward(Ws, Bs, X, Y)
    tW = [torch.tensor(w, dtype=torch.float64, requires_grad=True) for w in Ws]
    tB = [torch.tensor(b, dtype=torch.float64, requires_grad=True) for b in Bs]
    a = torch.tensor(X)
    for i in range(4):
        a = a @ tW[i].T + tB[i]
        if i < 3:
            a = torch.nn.functional.silu(a)
    np.testing.assert_allclose(oracle.mlp_forward(Ws, Bs, X), a.detach().numpy(), rtol=1e-13, atol=1e-13)
    tl = ((a - torch.tensor(Y)) ** 2).mean()
    tl.backward()
    assert abs(loss - tl.item()) < 1e-13
    for i in range(4):
        np.testing.assert_allclose(dW[i], tW[i].grad.numpy(), rtol=1e-11, atol=1e-14)
        np.testing.assert_allclose(dB[i], tB[i].grad.numpy(), rtol=1e-11, atol=1e-14)


def test_mlp_gradient_matches_fd():
    g = wl.rng(41, 1)
    widths = [3, 8, 8, 3]
    Ws = [g.standard_normal((widths[i + 1], widths[i])) for i in range(3)]
    Bs = [g.standard_normal(widths[i + 1]) for i in range(3)]
    X, Y = g.standard_normal((9, 3)), g.standard_normal((9, 3))
    _, dW, _ = oracle.mlp_loss_backward(Ws, Bs, X, Y)
    h = 1e-6
    for layer, (i, j) in ((0, (2, 1)), (1, (5, 7)), (2, (0, 4))):
        Wp = [w.copy() for w in Ws]
        Wm = [w.copy() for w in Ws]
        Wp[layer][i, j] += h
        Wm[layer][i, j] -= h
        fd = (oracle.mlp_loss_backward(Wp, Bs, X, Y)[0] - oracle.mlp_loss_backward(Wm, Bs, X, Y)[0]) / (2 * h)
        assert abs(dW[layer][i, j] - fd) < 1e-8


def test_mlp_encoding_identities():
    u = wl.rng(42, 1).uniform(-1, 1, (50, 3))
    e = oracle.mlp_encode(u, 6)
    assert e.shape == (50, 39)
    np.testing.assert_array_equal(e[:, :3], u)
    for k in range(6):
        s_, c_ = e[:, 3 + 6 * k:6 + 6 * k], e[:, 6 + 6 * k:9 + 6 * k]
        np.testing.assert_allclose(s_ ** 2 + c_ ** 2, 1.0, atol=1e-14)
        if k:
            ps, pc = e[:, 3 + 6 * (k - 1):6 + 6 * (k - 1)], e[:, 6 + 6 * (k - 1):9 + 6 * (k - 1)]
            np.testing.assert_allclose(s_, 2 * ps * pc, atol=1e-13)      # octaves double the angle
            np.testing.assert_allclose(c_, pc ** 2 - ps ** 2, atol=1e-13)
    np.testing.assert_allclose(e[:, 3:6], np.sin(np.pi * u), atol=1e-15)   # first octave is pi u


# --------------------------------------------------------------------------
# The tanh occupancy network of Sec. 3.1 as the cost
def test_tanh_net_matches_sympy_on_a_tiny_network():
    sp = pytest.importorskip("sympy")
    net = wl.tanh_net(11, 2, 3, lo=0.0, hi=4.0, gain=1.5, out_scale=3.0, b3=0.3)
    x0, x1 = sp.symbols("x0 x1")
    X = sp.Matrix([x0, x1])
    W1, b1 = sp.Matrix(net.W1.astype(float)), sp.Matrix(net.b1.astype(float))
    W2, b2 = sp.Matrix(net.W2.astype(float)), sp.Matrix(net.b2.astype(float))
    w3 = sp.Matrix(net.w3.astype(float))
    h1 = (W1 * X + b1).applyfunc(sp.tanh)
    h2 = (W2 * h1 + b2).applyfunc(sp.tanh)
    s = (w3.T * h2)[0, 0] + net.b3
    c = 1 / (1 + sp.exp(-s))
    grad = [sp.diff(c, v) for v in (x0, x1)]
    hess = [[sp.diff(c, a, b) for b in (x0, x1)] for a in (x0, x1)]
    pts = wl.uniform_box(12, 3, 5, np.zeros(2), np.full(2, 4.0))
    r = oracle.tnet_evaluate(net, pts, hess=True)
    for i, p in enumerate(pts.astype(float)):
        sub = {x0: p[0], x1: p[1]}
        assert abs(r["c"][i] - float(c.subs(sub))) <= 1e-13
        assert abs(r["s"][i] - float(s.subs(sub))) <= 1e-13
        for a in range(2):
            assert abs(r["grad"][i, a] - float(grad[a].subs(sub))) <= 1e-12
            for b in range(2):
                assert abs(r["hess"][i, a, b] - float(hess[a][b].subs(sub))) <= 1e-11


@pytest.mark.parametrize("d,H", [(2, 64), (3, 32), (7, 16)])
def test_tanh_net_derivatives_match_central_differences(d, H):
    net = wl.tanh_net(13 + d, d, H, lo=-3.0, hi=3.0, gain=2.0, out_scale=2.0, b3=-0.5)
    x = wl.uniform_box(14, 3, 6, np.full(d, -3.0), np.full(d, 3.0)).astype(np.float64)
    r = oracle.tnet_evaluate(net, x, hess=True)
    h = 1e-5
    for i in range(x.shape[0]):
        for a in range(d):
            e = np.zeros(d)
            e[a] = h
            cp = oracle.tnet_evaluate(net, (x[i] + e)[None], hess=False)
            cm = oracle.tnet_evaluate(net, (x[i] - e)[None], hess=False)
            fd_g = (cp["c"][0] - cm["c"][0]) / (2 * h)
            assert abs(r["grad"][i, a] - fd_g) <= 1e-8
            fd_h = (cp["grad"][0] - cm["grad"][0]) / (2 * h)
            assert np.abs(r["hess"][i, a] - fd_h).max() <= 1e-7
        assert np.abs(r["hess"][i] - r["hess"][i].T).max() <= 1e-14


def test_tanh_net_lipschitz_bound_dominates_sampled_derivatives():
    for d, H, gain in ((2, 64, 1.0), (2, 64, 4.0), (3, 32, 2.0)):
        net = wl.tanh_net(17 + H, d, H, gain=gain)
        L, G = oracle.tnet_lipschitz(net)
        x = wl.uniform_box(18, 3, 3000, np.full(d, -5.0), np.full(d, 15.0))
        r = oracle.tnet_evaluate(net, x, hess=True)
        hn = np.linalg.norm(r["hess"], ord=2, axis=(1, 2))
        assert hn.max() <= L
        sig = np.array([oracle.sigmoid3(v)[1] for v in r["s"]])
        assert (np.linalg.norm(r["grad"], axis=1) / sig).max() <= G * (1 + 1e-12)
        # the gradient bound is the product of the spectral norms (numpy's SVD)
        W1, W2, w3 = (a.astype(np.float64) for a in (net.W1, net.W2, net.w3))
        ref = np.linalg.norm(W1, 2) * np.linalg.norm(W2, 2) * np.linalg.norm(w3)
        assert ref <= G <= ref * (1 + 1e-10)


def test_tanh_net_morph_identity_one_step_and_contraction():
    d, H = 2, 64
    net = wl.tanh_net(19, d, H)
    x0 = wl.uniform_box(20, 3, 50, np.zeros(2), np.full(2, 10.0))
    zero = wl.TanhNet(net.W1, net.b1, net.W2, net.b2, np.zeros(H), net.b3)
    assert np.array_equal(oracle.tnet_morph(zero, x0, 7, 0.1), x0.astype(np.float64))
    L, _ = oracle.tnet_lipschitz(net)
    eta = 0.5 / L
    one = oracle.tnet_morph(net, x0, 1, eta)
    h = 1e-6
    for i in range(5):
        g = np.zeros(d)
        for a in range(d):
            e = np.zeros(d)
            e[a] = h
            cp = oracle.tnet_evaluate(net, (x0[i] + e)[None])["c"][0]
            cm = oracle.tnet_evaluate(net, (x0[i] - e)[None])["c"][0]
            g[a] = (cp - cm) / (2 * h)
        assert np.abs(one[i] - (x0[i] - eta * g)).max() <= 1e-9
    # eta L < 1: two samples never swap order along the map (injective steps)
    xa = oracle.tnet_morph(net, x0, 20, eta)
    for i in range(10):
        for j in range(i + 1, 10):
            d0 = np.linalg.norm(x0[i] - x0[j])
            assert np.linalg.norm(xa[i] - xa[j]) >= d0 * (1 - eta * L) ** 20 - 1e-12


# --------------------------------------------------------------------------
# Configuration space: Eq. (3) on a planar serial chain
def _cspace_case(seed=23, n=4, p=3, M=300):
    f = wl.random_field(seed, wl.RBF, 2, M, lo=0, hi=10, gamma=2.0, wscale=1.0, bias=-0.5)
    ch = wl.planar_arm(n, 4.0, (5.0, 5.0), p)
    lo, hi = wl.joint_box(n)
    Q = wl.uniform_box(seed, 3, 8, lo, hi).astype(np.float64)
    return f, ch, Q


def test_cspace_forward_kinematics_hand_cases():
    ch = wl.Chain([1.0, 2.0], base=(1.0, -1.0), p=2)
    P = oracle.cspace_points(ch, np.array([[0.0, 0.0], [np.pi / 2, -np.pi / 2], [np.pi, np.pi]]))
    exp = np.array([
        [[1.5, -1], [2, -1], [3, -1], [4, -1]],                 # straight along +x
        [[1, -0.5], [1, 0], [2, 0], [3, 0]],                    # up, then right
        [[0.5, -1], [0, -1], [1, -1], [2, -1]],                 # back along -x, then folded forward
    ])
    assert np.abs(P - exp).max() <= 1e-14


def test_cspace_gradient_matches_central_differences():
    f, ch, Q = _cspace_case()
    fc, gq = oracle.cspace_evaluate(f, ch, Q)
    h = 1e-6
    for i in range(Q.shape[0]):
        for j in range(ch.n):
            e = np.zeros(ch.n)
            e[j] = h
            fp, _ = oracle.cspace_evaluate(f, ch, (Q[i] + e)[None])
            fm, _ = oracle.cspace_evaluate(f, ch, (Q[i] - e)[None])
            assert abs(gq[i, j] - (fp[0] - fm[0]) / (2 * h)) <= 1e-7 * (1 + abs(gq[i, j]))
    # f_c is the occupancy summed over the body points
    P = oracle.cspace_points(ch, Q)
    c = oracle.evaluate(f, P.reshape(-1, 2))["c"].reshape(Q.shape[0], -1).sum(axis=1)
    assert np.abs(fc - c).max() <= 1e-12


def test_cspace_lipschitz_bound_dominates_sampled_hessian():
    f, ch, _ = _cspace_case(seed=24, n=5, p=2)
    Lx, Gx = oracle.lipschitz(f, np.full(2, -1.0), np.full(2, 11.0), cells=32)
    Lq = oracle.cspace_lipschitz(ch, Lx, Gx)
    lo, hi = wl.joint_box(ch.n)
    Q = wl.uniform_box(25, 3, 60, lo, hi).astype(np.float64)
    h = 1e-5
    worst = 0.0
    for q in Q:
        Hs = np.zeros((ch.n, ch.n))
        for j in range(ch.n):
            e = np.zeros(ch.n)
            e[j] = h
            _, gp = oracle.cspace_evaluate(f, ch, (q + e)[None])
            _, gm = oracle.cspace_evaluate(f, ch, (q - e)[None])
            Hs[j] = (gp[0] - gm[0]) / (2 * h)
        worst = max(worst, np.linalg.norm(0.5 * (Hs + Hs.T), 2))
    assert worst <= Lq


def test_cspace_morph_identity_and_one_step():
    f, ch, Q = _cspace_case(seed=26)
    zero = wl.Field(f.kind, f.centres, np.zeros_like(f.w), gamma=f.gamma, bias=f.bias)
    assert np.array_equal(oracle.cspace_morph(zero, ch, Q, 5, 0.1), Q)
    eta = 0.01
    q1 = oracle.cspace_morph(f, ch, Q, 1, eta)
    _, g = oracle.cspace_evaluate(f, ch, Q)
    assert np.abs(q1 - (Q - eta * g)).max() <= 1e-15
    q3 = oracle.cspace_morph(f, ch, Q, 3, eta)
    q = Q.copy()
    for _ in range(3):
        q = q - eta * oracle.cspace_evaluate(f, ch, q)[1]
    assert np.abs(q3 - q).max() <= 1e-14


# --------------------------------------------------------------------------
# The counter-based generator of device-drawn base samples
def test_philox4x32_known_answers():
    """Known-answer vectors published with the Philox generator (Random123)."""
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, want in cases:
        assert [int(v) for v in oracle.philox4x32(ctr, key)] == list(want)


def test_uniform_batch_layout_and_range():
    lo, hi = np.array([-1.0, 2.0, 0.0], np.float32), np.array([1.0, 6.0, 10.0], np.float32)
    x = oracle.uniform_batch(1234, 7, 1000, lo, hi)
    assert x.shape == (1000, 3) and (x >= lo).all() and (x < hi).all()
    # element e = i d + j is word e mod 4 of block e / 4 with counter (block, 0, batch, 0)
    for e in (0, 1, 5, 2999):
        i, j = divmod(e, 3)
        w = oracle.philox4x32((e // 4, 0, 7, 0), (1234, 0))[e % 4]
        u = np.float32(int(w) >> 8) * np.float32(2.0 ** -24)
        assert x[i, j] == np.float32(np.float32(u) * (hi[j] - lo[j]) + lo[j]) or \
            abs(float(x[i, j]) - (float(u) * float(hi[j] - lo[j]) + float(lo[j]))) <= 1e-6
    # roughly uniform per coordinate
    m = (x - lo) / (hi - lo)
    assert np.abs(m.mean(axis=0) - 0.5).max() < 0.03
    # different batches and seeds differ
    assert not np.array_equal(x, oracle.uniform_batch(1234, 8, 1000, lo, hi))
    assert not np.array_equal(x, oracle.uniform_batch(1235, 7, 1000, lo, hi))
