"""FP64 CPU oracle for the PDMP sample-morphing path (arXiv 2108.11775).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA library in ``paper_2108_11775_gb300``; neither
imports the other.  Inputs come from ``workloads`` (seeded generators with
none of the method's arithmetic).

The arithmetic lives in ``pdmp_oracle.c`` (plain C, double precision, libm),
compiled here with gcc into ``oracle/_build/liboracle.so``.  Each wrapper
below names the passage of the paper it follows:

* ``evaluate``       -- Sec. 3.1: occupancy c = sigmoid(s), s = w.phi(x) + b,
                        and its input gradient / Hessian.
* ``morph``          -- Eq. (1) with Euler's method (Sec. 3.2).
* ``morph_inverse``  -- Eq. (2), each Euler step undone by a fixed point.
* ``morph_vjp``      -- chain rule through the Euler steps of Eq. (1).
* ``logdet``         -- log|det| of the Jacobian of the map (Sec. 3.2,
                        "Drawing Samples": the quantity sampling avoids).
* ``lipschitz``      -- Sec. 3.2: Lipschitz gradient => Euler step eta < 1/L.
* ``fit`` / ``fit_objective`` -- Sec. 3.1: BCE minimised by gradient descent.
* ``box_labels``     -- ground-truth occupancy labels of the dataset D.
* ``mlp_*``          -- the surrogate network (no counterpart in the paper).
* ``philox4x32`` / ``uniform_batch`` -- the counter-based generator of the
                        base samples a device-side sampler draws.
* ``cspace_*``       -- Sec. 3.2, Eq. (3): the occupancy cost on a planar
                        chain's body points pulled back to joint space.
* ``tnet_*``         -- Sec. 3.1's own occupancy model: a fully connected
                        network with tanh hidden layers and a sigmoid output,
                        used as the cost of the morph of Eq. (1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdmp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_ip = ctypes.POINTER(ctypes.c_int)
_L = ctypes.c_long
_I = ctypes.c_int
_D = ctypes.c_double


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (IEEE double, no FMA contraction, so the
    x86 and Arm builds round identically)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _field_args():
    return [_I, _I, _L, _dp, _dp, _D, _dp, _D]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.orc_set_threads.argtypes = [_I]
            L.orc_get_threads.restype = _I
            L.orc_sigmoid3.argtypes = [_D, _dp]
            L.orc_eval.argtypes = _field_args() + [_dp, _L, _dp, _dp, _dp, _dp, _dp]
            L.orc_morph.argtypes = _field_args() + [_dp, _L, _I, _D, _dp, _dp]
            L.orc_morph_inverse.argtypes = _field_args() + [_dp, _L, _I, _D, _D, _I, _dp, _ip]
            L.orc_morph_vjp.argtypes = _field_args() + [_dp, _L, _I, _D, _dp, _dp, _dp, _dp]
            L.orc_logdet.argtypes = _field_args() + [_dp, _L, _I, _D, _dp, _dp, _dp]
            L.orc_lipschitz_rbf.argtypes = [_I, _L, _dp, _D, _dp, _dp, _dp, _I, _dp, _dp]
            L.orc_lipschitz_rff.argtypes = [_I, _L, _dp, _dp, _dp, _dp]
            L.orc_fit.argtypes = [_I, _I, _L, _dp, _dp, _D, _dp, _u8p, _L, _D, _I, _I, _dp, _dp, _dp, _dp]
            L.orc_fit_objective.argtypes = [_I, _I, _L, _dp, _dp, _D, _dp, _u8p, _L, _D, _dp, _D, _dp, _dp, _dp]
            L.orc_box_labels.argtypes = [_I, _fp, _L, _fp, _L, _u8p]
            L.orc_mlp_forward.argtypes = [_I, _ip, _dp, _dp, _dp, _L, _dp, _dp]
            L.orc_mlp_loss_backward.argtypes = [_I, _ip, _dp, _dp, _dp, _dp, _L, _dp, _dp, _dp]
            L.orc_mlp_encode.argtypes = [_dp, _L, _I, _dp]
            tnet = [_I, _I, _dp, _dp, _dp, _dp, _dp, _D]
            L.orc_tnet_eval.argtypes = tnet + [_dp, _L, _dp, _dp, _dp, _dp]
            L.orc_tnet_morph.argtypes = tnet + [_dp, _L, _I, _D, _dp]
            L.orc_tnet_lipschitz.argtypes = [_I, _I, _dp, _dp, _dp, _dp, _dp]
            cs = _field_args() + [_I, _I, _dp, _dp]
            L.orc_cspace_eval.argtypes = cs + [_dp, _L, _dp, _dp]
            L.orc_cspace_points.argtypes = [_I, _I, _dp, _dp, _dp, _L, _dp]
            L.orc_cspace_morph.argtypes = cs + [_dp, _L, _I, _D, _dp]
            L.orc_cspace_lipschitz.argtypes = [_I, _I, _dp, _D, _D, _dp]
            u32p = ctypes.POINTER(ctypes.c_uint32)
            L.orc_philox4x32.argtypes = [u32p, u32p, u32p]
            L.orc_uniform_batch.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _L, _I, _fp, _fp, _fp]
            for name in ("orc_philox4x32", "orc_uniform_batch", "orc_cspace_eval", "orc_cspace_points", "orc_cspace_morph", "orc_cspace_lipschitz",
                         "orc_tnet_eval", "orc_tnet_morph", "orc_tnet_lipschitz","orc_eval", "orc_morph", "orc_morph_inverse", "orc_morph_vjp", "orc_logdet",
                         "orc_lipschitz_rbf", "orc_lipschitz_rff", "orc_fit", "orc_fit_objective",
                         "orc_box_labels", "orc_mlp_forward", "orc_mlp_loss_backward", "orc_mlp_encode"):
                getattr(L, name).restype = _I
            L.orc_set_threads(os.cpu_count() or 1)
            _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


# ---------------------------------------------------------------------------
def _d(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    if a.dtype == np.float64:
        return a.ctypes.data_as(_dp)
    if a.dtype == np.float32:
        return a.ctypes.data_as(_fp)
    if a.dtype == np.uint8:
        return a.ctypes.data_as(_u8p)
    if a.dtype == np.int32:
        return a.ctypes.data_as(_ip)
    raise TypeError(a.dtype)


class _F:
    """The field's arrays promoted (exactly) to float64 and kept alive."""

    def __init__(self, field):
        self.kind = int(field.kind)
        self.centres = _d(field.centres)
        self.M, self.d = self.centres.shape
        self.phase = _d(field.phase) if field.phase is not None else None
        self.gamma = float(field.gamma)
        self.w = _d(field.w)
        self.bias = float(field.bias)
        assert self.w.shape == (self.M,)

    def args(self):
        return [self.kind, self.d, self.M, _ptr(self.centres), _ptr(self.phase), self.gamma,
                _ptr(self.w), self.bias]


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (code {rc})")


def sigmoid3(s: float):
    out = np.zeros(3)
    lib().orc_sigmoid3(float(s), _ptr(out))
    return out


def evaluate(field, x, hess: bool = False) -> dict:
    """c, s, grad c, (Hess c) and sigma'(s) * sum_m |w_m| |grad phi_m| at points x (n x d)."""
    f = _F(field)
    x = _d(x).reshape(-1, f.d)
    n = x.shape[0]
    c, s, g, sc = np.zeros(n), np.zeros(n), np.zeros((n, f.d)), np.zeros(n)
    h = np.zeros((n, f.d, f.d)) if hess else None
    _check(lib().orc_eval(*f.args(), _ptr(x), n, _ptr(c), _ptr(s), _ptr(g), _ptr(h), _ptr(sc)), "eval")
    out = {"c": c, "s": s, "grad": g, "scale": sc}
    if hess:
        out["hess"] = h
    return out


def morph(field, x0, T: int, eta: float, traj: bool = False):
    """x_T (N x d); with traj=True the whole trajectory (N x (T+1) x d)."""
    f = _F(field)
    x0 = _d(x0).reshape(-1, f.d)
    N = x0.shape[0]
    xT = np.zeros((N, f.d))
    tr = np.zeros((N, T + 1, f.d)) if traj else None
    _check(lib().orc_morph(*f.args(), _ptr(x0), N, int(T), float(eta), _ptr(xT), _ptr(tr)), "morph")
    return tr if traj else xT


def morph_inverse(field, z, T: int, eta: float, tol: float = 1e-13, maxit: int = 200):
    f = _F(field)
    z = _d(z).reshape(-1, f.d)
    N = z.shape[0]
    y = np.zeros((N, f.d))
    its = np.zeros(N, dtype=np.int32)
    _check(lib().orc_morph_inverse(*f.args(), _ptr(z), N, int(T), float(eta), float(tol), int(maxit),
                                   _ptr(y), _ptr(its)), "inverse")
    return y, its


def morph_vjp(field, x0, T: int, eta: float, gT, want_gw: bool = False):
    """g0 = (dx_T/dx_0)^T g_T per sample; with want_gw also d/dw and d/dbias of
    sum_n <g_T[n], x_T[n]>."""
    f = _F(field)
    x0 = _d(x0).reshape(-1, f.d)
    gT = _d(gT).reshape(-1, f.d)
    N = x0.shape[0]
    g0 = np.zeros((N, f.d))
    gw = np.zeros(f.M) if want_gw else None
    gb = np.zeros(1) if want_gw else None
    _check(lib().orc_morph_vjp(*f.args(), _ptr(x0), N, int(T), float(eta), _ptr(gT), _ptr(g0),
                               _ptr(gw), _ptr(gb)), "vjp")
    if want_gw:
        return g0, gw, float(gb[0])
    return g0


def logdet(field, x0, T: int, eta: float):
    """(logdet (N), x_T (N x d), min over steps of det(I - eta Hess c) (N))."""
    f = _F(field)
    x0 = _d(x0).reshape(-1, f.d)
    N = x0.shape[0]
    ld, xT, md = np.zeros(N), np.zeros((N, f.d)), np.zeros(N)
    _check(lib().orc_logdet(*f.args(), _ptr(x0), N, int(T), float(eta), _ptr(ld), _ptr(xT), _ptr(md)),
           "logdet")
    return ld, xT, md


def lipschitz(field, lo=None, hi=None, cells: int = 64):
    """(L, G): certified bounds on sup |Hess c|_2 and sup |grad c|_2 (RBF: over
    the box [lo, hi] by cells^d cells; RFF: everywhere)."""
    f = _F(field)
    L, G = np.zeros(1), np.zeros(1)
    if f.kind == 0:
        lo, hi = _d(lo), _d(hi)
        _check(lib().orc_lipschitz_rbf(f.d, f.M, _ptr(f.centres), f.gamma, _ptr(f.w), _ptr(lo), _ptr(hi),
                                       int(cells), _ptr(L), _ptr(G)), "lipschitz")
    else:
        _check(lib().orc_lipschitz_rff(f.d, f.M, _ptr(f.centres), _ptr(f.w), _ptr(L), _ptr(G)), "lipschitz")
    return float(L[0]), float(G[0])


def fit(field, X, y, l2: float, power_iters: int, iters: int):
    """(w (M), bias, final loss, step size alpha) of the BCE fit; the field's
    w and bias are ignored (the fit starts from zero)."""
    f = _F(field)
    X = _d(X).reshape(-1, f.d)
    y = np.ascontiguousarray(np.asarray(y, dtype=np.uint8))
    n = X.shape[0]
    w, b, loss, alpha = np.zeros(f.M), np.zeros(1), np.zeros(1), np.zeros(1)
    _check(lib().orc_fit(f.kind, f.d, f.M, _ptr(f.centres), _ptr(f.phase), f.gamma, _ptr(X), _ptr(y), n,
                         float(l2), int(power_iters), int(iters), _ptr(w), _ptr(b), _ptr(loss), _ptr(alpha)),
           "fit")
    return w, float(b[0]), float(loss[0]), float(alpha[0])


def fit_objective(field, X, y, l2: float, w, b: float):
    """(loss, grad_w, grad_b) of mean BCE + (l2/2)|w|^2 at (w, b)."""
    f = _F(field)
    X = _d(X).reshape(-1, f.d)
    y = np.ascontiguousarray(np.asarray(y, dtype=np.uint8))
    w = _d(w)
    n = X.shape[0]
    loss, gw, gb = np.zeros(1), np.zeros(f.M), np.zeros(1)
    _check(lib().orc_fit_objective(f.kind, f.d, f.M, _ptr(f.centres), _ptr(f.phase), f.gamma, _ptr(X), _ptr(y),
                                   n, float(l2), _ptr(w), float(b), _ptr(loss), _ptr(gw), _ptr(gb)), "fit_objective")
    return float(loss[0]), gw, float(gb[0])


def box_labels(boxes, x):
    """1 where the float32 point lies in some closed box (boxes: nb x 2d float32)."""
    boxes = np.ascontiguousarray(np.asarray(boxes, dtype=np.float32))
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    d = x.shape[1]
    out = np.zeros(x.shape[0], dtype=np.uint8)
    _check(lib().orc_box_labels(d, _ptr(boxes), boxes.shape[0], _ptr(x), x.shape[0], _ptr(out)), "labels")
    return out


# ---------------------------------------------------------------------------
# surrogate MLP: widths[0] -> widths[1] -> ... -> widths[-1], SiLU between the
# linear layers, none after the last.  Weights W_l are (out x in) row-major,
# passed as one flat float64 buffer in layer order, biases likewise.
def _mlp_pack(weights, biases):
    widths = [weights[0].shape[1]] + [w.shape[0] for w in weights]
    wflat = np.concatenate([_d(w).ravel() for w in weights])
    bflat = np.concatenate([_d(b).ravel() for b in biases])
    return np.asarray(widths, dtype=np.int32), wflat, bflat


def mlp_encode(u, n_freq: int = 6):
    """Fourier encoding of normalised inputs u (n x 3) -> n x (3 + 6 n_freq)."""
    u = _d(u).reshape(-1, 3)
    out = np.zeros((u.shape[0], 3 + 6 * n_freq))
    _check(lib().orc_mlp_encode(_ptr(u), u.shape[0], int(n_freq), _ptr(out)), "mlp_encode")
    return out


def mlp_forward(weights, biases, X):
    widths, wf, bf = _mlp_pack(weights, biases)
    X = _d(X)
    n = X.shape[0]
    out = np.zeros((n, int(widths[-1])))
    _check(lib().orc_mlp_forward(len(weights), _ptr(widths), _ptr(wf), _ptr(bf), _ptr(X), n, _ptr(out), None),
           "mlp_forward")
    return out


def mlp_loss_backward(weights, biases, X, Y):
    """(loss, [dW_l], [db_l]) of loss = mean over samples and outputs of (f(x) - y)^2."""
    widths, wf, bf = _mlp_pack(weights, biases)
    X, Y = _d(X), _d(Y)
    n = X.shape[0]
    gw, gb, loss = np.zeros_like(wf), np.zeros_like(bf), np.zeros(1)
    _check(lib().orc_mlp_loss_backward(len(weights), _ptr(widths), _ptr(wf), _ptr(bf), _ptr(X), _ptr(Y), n,
                                       _ptr(loss), _ptr(gw), _ptr(gb)), "mlp_backward")
    dws, dbs, ow, ob = [], [], 0, 0
    for w, b in zip(weights, biases):
        dws.append(gw[ow:ow + w.size].reshape(w.shape))
        dbs.append(gb[ob:ob + b.size].reshape(b.shape))
        ow += w.size
        ob += b.size
    return float(loss[0]), dws, dbs


# ---------------------------------------------------------------------------
class _Net:
    """A tanh network's arrays promoted (exactly) to float64 and kept alive."""

    def __init__(self, net):
        self.W1, self.b1 = _d(net.W1), _d(net.b1)
        self.W2, self.b2 = _d(net.W2), _d(net.b2)
        self.w3, self.b3 = _d(net.w3), float(net.b3)
        self.H, self.d = self.W1.shape
        assert self.W2.shape == (self.H, self.H) and self.w3.shape == (self.H,)

    def args(self):
        return [self.d, self.H, _ptr(self.W1), _ptr(self.b1), _ptr(self.W2), _ptr(self.b2), _ptr(self.w3), self.b3]


def tnet_evaluate(net, x, hess: bool = False) -> dict:
    """Sec. 3.1: c = sigmoid(w3 . tanh(W2 tanh(W1 x + b1) + b2) + b3) and its input derivatives."""
    n = _Net(net)
    x = _d(x).reshape(-1, n.d)
    N = x.shape[0]
    c, s, gc = np.zeros(N), np.zeros(N), np.zeros((N, n.d))
    hc = np.zeros((N, n.d, n.d)) if hess else None
    _check(lib().orc_tnet_eval(*n.args(), _ptr(x), N, _ptr(c), _ptr(s), _ptr(gc), _ptr(hc)), "tnet_eval")
    out = {"c": c, "s": s, "grad": gc}
    if hess:
        out["hess"] = hc
    return out


def tnet_morph(net, x0, T: int, eta: float):
    """Eq. (1) by Euler's method with the tanh network's occupancy as the cost."""
    n = _Net(net)
    x0 = _d(x0).reshape(-1, n.d)
    xT = np.zeros_like(x0)
    _check(lib().orc_tnet_morph(*n.args(), _ptr(x0), x0.shape[0], int(T), float(eta), _ptr(xT)), "tnet_morph")
    return xT


def tnet_lipschitz(net):
    """(L, G): certified bounds on sup |Hess c|_2 and sup |grad s|_2 over all inputs."""
    n = _Net(net)
    L, G = ctypes.c_double(0), ctypes.c_double(0)
    _check(lib().orc_tnet_lipschitz(n.d, n.H, _ptr(n.W1), _ptr(n.W2), _ptr(n.w3), ctypes.byref(L),
                                    ctypes.byref(G)), "tnet_lipschitz")
    return float(L.value), float(G.value)


# ---------------------------------------------------------------------------
def _chain(chain):
    return (int(chain.n), int(chain.p), _d(chain.base), _d(chain.lengths))


def cspace_points(chain, Q):
    """Body points psi_i(q) (N x n p x 2) of the planar chain."""
    n, p, base, ln = _chain(chain)
    Q = _d(Q).reshape(-1, n)
    P = np.zeros((Q.shape[0], n * p, 2))
    _check(lib().orc_cspace_points(n, p, _ptr(base), _ptr(ln), _ptr(Q), Q.shape[0], _ptr(P)), "cspace_points")
    return P


def cspace_evaluate(field, chain, Q):
    """(f_c, grad_q f_c): the occupancy summed over the body points and its
    joint-space gradient by Eq. (3)."""
    f = _F(field)
    n, p, base, ln = _chain(chain)
    Q = _d(Q).reshape(-1, n)
    fc, gq = np.zeros(Q.shape[0]), np.zeros_like(Q)
    _check(lib().orc_cspace_eval(*f.args(), n, p, _ptr(base), _ptr(ln), _ptr(Q), Q.shape[0], _ptr(fc), _ptr(gq)),
           "cspace_eval")
    return fc, gq


def cspace_morph(field, chain, Q0, T: int, eta: float):
    """Eq. (1) in joint space with the gradient of Eq. (3)."""
    f = _F(field)
    n, p, base, ln = _chain(chain)
    Q0 = _d(Q0).reshape(-1, n)
    QT = np.zeros_like(Q0)
    _check(lib().orc_cspace_morph(*f.args(), n, p, _ptr(base), _ptr(ln), _ptr(Q0), Q0.shape[0], int(T), float(eta),
                                  _ptr(QT)), "cspace_morph")
    return QT


def cspace_lipschitz(chain, Lx: float, Gx: float) -> float:
    """Certified bound on sup |Hess_q f_c| from task-space bounds Lx (Hessian) and Gx (gradient)."""
    n, p, _, ln = _chain(chain)
    out = ctypes.c_double(0)
    _check(lib().orc_cspace_lipschitz(n, p, _ptr(ln), float(Lx), float(Gx), ctypes.byref(out)), "cspace_lipschitz")
    return float(out.value)


# ---------------------------------------------------------------------------
def philox4x32(counter, key):
    """Philox4x32-10 of one 4-word counter under a 2-word key (uint32 words)."""
    c = np.ascontiguousarray(np.asarray(counter, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib().orc_philox4x32(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p), out.ctypes.data_as(u32p))
    return out


def uniform_batch(seed: int, batch: int, n: int, lo, hi):
    """Batch `batch` of n base samples uniform on [lo, hi] (float32) from the counter-based generator."""
    lo = np.ascontiguousarray(np.asarray(lo, dtype=np.float32))
    hi = np.ascontiguousarray(np.asarray(hi, dtype=np.float32))
    d = lo.shape[0]
    x = np.zeros((n, d), dtype=np.float32)
    _check(lib().orc_uniform_batch(int(seed), int(batch), int(n), d, _ptr(lo), _ptr(hi), _ptr(x)), "uniform_batch")
    return x
