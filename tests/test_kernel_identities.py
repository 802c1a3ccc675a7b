"""The rearrangements the fast kernels compute, evaluated in FP64 on the CPU
against the oracle's plain definitions (s, grad s and Hess s from its c,
grad c and Hess c through sigma', sigma''), so that an error in a kernel's
algebra fails here as well as in the GPU parity tests:

* RBF sorted tiles: the expanded exponent about a tile origin o (log2 of
  |w| phi = a + b . u - g'|u|^2), the Hessian-vector product from the
  moments S, G, H alone (sum e'(c . v) = v . G, sum e'(c . v) c = H v), and
  the log-det's full Hessian from the same moments;
* RFF tensor-core VJP: (Hess s) v = 2 pi sum_m cos(theta_m) (omega_m . v / 2 pi)(-w_m omega_m);
* the sorted tiles' weight-gradient pass: cA phi_m + cB grad phi_m . g =
  phi_m (alpha + beta . c_m) with alpha = cA - 2 gamma cB (u . g) and
  beta = 2 gamma cB g;
* the tensor-core RBF form: its TF32 K slots sum to the expanded exponent
  a + b . u, and its weighted records' moments give s and grad s."""
import numpy as np
import pytest

import oracle
import workloads as wl

LOG2E = 1.0 / np.log(2.0)


def _plain_s(f, x):
    """s, grad s, Hess s at one point from the oracle's c, grad c, Hess c."""
    ev = oracle.evaluate(f, x[None], hess=True)
    s = float(ev["s"][0])
    _, d1, d2 = oracle.sigmoid3(s)
    gs = ev["grad"][0] / d1
    hs = (ev["hess"][0] - d2 * np.outer(gs, gs)) / d1
    return s, gs, hs


@pytest.mark.parametrize("d", [2, 3])
def test_rbf_expanded_moments_give_s_grad_and_hessian_vector(d):
    f = wl.random_field(11 + d, wl.RBF, d, 300, lo=0.0, hi=3.0, gamma=4.0, wscale=1.5, bias=0.25)
    rng = np.random.default_rng(d)
    mu, w, gamma = f.centres.astype(np.float64), f.w.astype(np.float64), float(f.gamma)
    gl2e = gamma * LOG2E
    for _ in range(5):
        o = rng.uniform(0.5, 2.5, d)                       # the tile's origin
        x = o + rng.uniform(-0.3, 0.3, d)                  # a sample of the tile
        v = rng.standard_normal(d)
        u, c = x - o, mu - o
        a = np.log2(np.abs(w)) - gl2e * (c * c).sum(1)
        e = np.sign(w) * np.exp2(a + 2.0 * gl2e * (c @ u))  # e'_m = sg 2^(a + b . u)
        f_u = np.exp2(-gl2e * (u @ u))
        S, G, H = e.sum(), e @ c, (e[:, None, None] * c[:, :, None] * c[:, None, :]).sum(0)
        usg = u * S - G
        s_k = f_u * S + f.bias
        grad_k = -2.0 * gamma * f_u * usg
        hv_k = 4 * gamma ** 2 * f_u * ((u @ v) * usg - (u * (v @ G) - H @ v)) - 2.0 * gamma * f_u * S * v
        s, gs, hs = _plain_s(f, x)
        assert abs(s_k - s) <= 1e-12 * max(1.0, abs(s))
        np.testing.assert_allclose(grad_k, gs, rtol=0, atol=1e-11 * max(1.0, np.abs(gs).max()))
        np.testing.assert_allclose(hv_k, hs @ v, rtol=0, atol=1e-10 * max(1.0, np.abs(hs @ v).max()))
        # the log-det's Hessian from the same moments
        hs_k = 4 * gamma ** 2 * f_u * (S * np.outer(u, u) - np.outer(G, u) - np.outer(u, G) + H) \
            - 2.0 * gamma * f_u * S * np.eye(d)
        np.testing.assert_allclose(hs_k, hs, rtol=0, atol=1e-10 * max(1.0, np.abs(hs).max()))


@pytest.mark.parametrize("d", [2, 3])
def test_rbf_direct_form_sums(d):
    """Tiles too wide for the expanded form sum, about the origin 0,
    S = sum w phi, G = sum w phi (x - mu), P = sum w phi ((x - mu) . v)(x - mu):
    grad s = -2 gamma G and (Hess s) v = 4 gamma^2 P - 2 gamma S v."""
    f = wl.random_field(31 + d, wl.RBF, d, 300, lo=0.0, hi=3.0, gamma=4.0, wscale=1.5, bias=-0.2)
    rng = np.random.default_rng(50 + d)
    mu, w, gamma = f.centres.astype(np.float64), f.w.astype(np.float64), float(f.gamma)
    for _ in range(5):
        x, v = rng.uniform(0.0, 3.0, d), rng.standard_normal(d)
        dx = x - mu
        we = w * np.exp2(-gamma * LOG2E * (dx * dx).sum(1))
        S, G, P = we.sum(), we @ dx, (we * (dx @ v)) @ dx
        s, gs, hs = _plain_s(f, x)
        assert abs(S + f.bias - s) <= 1e-12 * max(1.0, abs(s))
        np.testing.assert_allclose(-2.0 * gamma * G, gs, rtol=0, atol=1e-11 * max(1.0, np.abs(gs).max()))
        np.testing.assert_allclose(4 * gamma ** 2 * P - 2.0 * gamma * S * v, hs @ v, rtol=0,
                                   atol=1e-10 * max(1.0, np.abs(hs @ v).max()))


@pytest.mark.parametrize("d", [3, 7])
def test_rff_hessian_vector_contraction(d):
    f = wl.random_field(21 + d, wl.RFF, d, 256, wscale=6.0, bias=0.1)
    rng = np.random.default_rng(30 + d)
    om, ph, w = f.centres.astype(np.float64), f.phase.astype(np.float64), f.w.astype(np.float64)
    for _ in range(5):
        x, v = rng.uniform(-np.pi, np.pi, d), rng.standard_normal(d)
        theta = om @ x + ph
        o = om @ v / (2.0 * np.pi)                          # the omega . g MMA, in turns
        P = (np.cos(theta) * o) @ (-w[:, None] * om)        # the P MMA against the gradient table
        grad_k = (-np.sin(theta) * w) @ om                  # the gradient MMA
        s, gs, hs = _plain_s(f, x)
        np.testing.assert_allclose(grad_k, gs, rtol=0, atol=1e-11 * max(1.0, np.abs(gs).max()))
        np.testing.assert_allclose(2.0 * np.pi * P, hs @ v, rtol=0, atol=1e-10 * max(1.0, np.abs(hs @ v).max()))


@pytest.mark.parametrize("d", [2, 3])
def test_rbf_weight_gradient_terms(d):
    rng = np.random.default_rng(40 + d)
    gamma = 4.0
    mu = rng.uniform(0, 3, (50, d))
    o = np.full(d, 1.5)
    for _ in range(5):
        x, g = rng.uniform(1.0, 2.0, d), rng.standard_normal(d)
        cA, cB = rng.standard_normal(2)
        phi = np.exp(-gamma * ((x - mu) ** 2).sum(1))
        grad_phi = -2.0 * gamma * phi[:, None] * (x - mu)
        plain = cA * phi + cB * (grad_phi @ g)
        u, c = x - o, mu - o
        alpha = cA - 2.0 * gamma * cB * (u @ g)
        beta = 2.0 * gamma * cB * g
        np.testing.assert_allclose(phi * (alpha + c @ beta), plain, rtol=1e-12, atol=1e-14)


def _tf32(v):
    """round to TF32 (10 explicit mantissa bits), nearest with ties away, as
    cvt.rna.tf32.f32 does on a float32 input"""
    b = np.asarray(v, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x1000) & 0xFFFFE000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _tc05_rows(a, b, u):
    """The tensor-core form's K slots: A row (sample) [1, 1, u_jh, u_jh, u_jl ..]
    and B row (centre) [a_h, a_l, b_jh, b_jl, b_jh ..], each a TF32 piece of
    the FP32 value."""
    A, B = [1.0, 1.0], [_tf32(a), _tf32(np.float32(a) - np.float32(_tf32(a)))]
    for uj, bj in zip(u, b):
        uh, bh = _tf32(uj), _tf32(bj)
        A += [uh, uh, _tf32(np.float32(uj) - np.float32(uh))]
        B += [bh, _tf32(np.float32(bj) - np.float32(bh)), bh]
    return np.array(A, np.float64), np.array(B, np.float64)


@pytest.mark.parametrize("d", [2, 3])
def test_tc05_slots_give_the_expanded_exponent_and_the_weighted_records_the_moments(d):
    """morph_rbf_tc05.cu: the K-slot products sum to a + b . u (a = -g'|c|^2,
    b = 2 g' c) to about 2^-21 of |a| + |b . u| (only the lo x lo products are
    left out), while dropping any one slot breaks that; and the moments it sums
    with the weights in the records, S = sum w e, G = sum w e c, give s and
    grad s exactly as the plain definitions."""
    f = wl.random_field(21 + d, wl.RBF, d, 200, lo=0.0, hi=3.0, gamma=4.0, wscale=1.5, bias=0.1)
    rng = np.random.default_rng(5 + d)
    mu, w, gamma = f.centres.astype(np.float64), f.w.astype(np.float64), float(f.gamma)
    gl2e = gamma * LOG2E
    for _ in range(4):
        o = rng.uniform(0.8, 2.2, d)
        x = o + rng.uniform(-0.25, 0.25, d)
        u, c = x - o, mu - o
        a = -gl2e * (c * c).sum(1)
        b = 2.0 * gl2e * c
        for m in range(0, mu.shape[0], 17):
            A, B = _tc05_rows(np.float32(a[m]), b[m].astype(np.float32), u.astype(np.float32))
            exact = float(np.float32(a[m])) + float(b[m].astype(np.float32).astype(np.float64) @ u.astype(np.float32))
            scale = abs(a[m]) + abs(b[m] @ u)
            assert abs(A @ B - exact) <= 2.0 ** -20 * scale
            for k in range(2, A.size):                  # every u, b slot carries its share
                drop = A.copy()
                drop[k] = 0.0
                if abs(A[k] * B[k]) > 2.0 ** -16 * scale:
                    assert abs(drop @ B - exact) > 2.0 ** -20 * scale
        e = np.exp2(a + b @ u)                            # e_m = 2^(a_m + b_m . u)
        f_u = np.exp2(-gl2e * (u @ u))
        S, G = (w * e).sum(), (w * e) @ c                 # the weighted records' sums
        s_k = f_u * S + f.bias
        grad_k = -2.0 * gamma * f_u * (u * S - G)
        s, gs, _ = _plain_s(f, x)
        assert abs(s_k - s) <= 1e-12 * max(1.0, abs(s))
        np.testing.assert_allclose(grad_k, gs, rtol=0, atol=1e-11 * max(1.0, np.abs(gs).max()))
