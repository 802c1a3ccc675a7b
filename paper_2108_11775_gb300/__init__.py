"""Python binding of libpdmp, the GB300 (sm_103a) library for the sample-
morphing hot path of PDMP (arXiv 2108.11775).

Argument marshalling only: every computation runs in the library's CUDA
kernels (``csrc/``), reached through the C ABI declared in
``include/pdmp.h``.  Tensors are torch CUDA tensors (PyTorch provides device
memory and streams); each call runs on torch's current stream.  There is no
CPU path: if the library cannot be loaded, every call raises.

Names follow the C ABI: ``morph``, ``morph_vjp``, ``logdet``,
``occupancy_query``, ``box_labels``, ``lipschitz_bound``, ``fit_occupancy``,
``stream_status``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

__all__ = [
    "PdmpError", "DeviceField", "lib", "morph", "morph_trace", "morph_workspace", "morph_vjp", "morph_vjp_workspace", "logdet",
    "occupancy_query", "box_labels", "lipschitz_bound", "fit_occupancy", "fit_workspace", "stream_status",
    "RBF", "RFF",
]

RBF = 0
RFF = 1

OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "STEP_TOO_LARGE", 3: "WORKSPACE_TOO_SMALL", 4: "CUDA_ERROR",
                5: "NOT_CONVERGED", 6: "TIMEOUT", 7: "DEVICE_FLAG", 8: "UNSUPPORTED"}


class PdmpError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = int(status)
        msg = lib().pdmp_status_string(int(status)).decode() if _lib is not None else STATUS_NAMES.get(status, "?")
        super().__init__(f"{what}: {STATUS_NAMES.get(self.status, self.status)} ({msg})")


class _Field(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("d", ctypes.c_int32), ("M", ctypes.c_int64),
                ("centres", ctypes.c_void_p), ("phase", ctypes.c_void_p), ("gamma", ctypes.c_float),
                ("w", ctypes.c_void_p), ("bias", ctypes.c_float), ("lipschitz", ctypes.c_double)]


_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p
_i32, _i64, _f32, _f64, _sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double, ctypes.c_size_t
_FP = ctypes.POINTER(_Field)


def lib():
    """Loads libpdmp.so (building it with nvcc if it is not built yet)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                path = _build.build()
            L = ctypes.CDLL(path)
            L.pdmp_status_string.restype = ctypes.c_char_p
            L.pdmp_status_string.argtypes = [_i32]
            L.pdmp_version.restype = _i32
            sigs = {
                "pdmp_stream_status": [_P, ctypes.POINTER(_i32)],
                "pdmp_morph": [_FP, _P, _i64, _i32, _f32, _P, _P, _i32, _P, _sz, _P],
                "pdmp_morph_trace": [_FP, _P, _i64, _i32, _f32, _P, _P, _P, _sz, _P],
                "pdmp_morph_vjp": [_FP, _P, _i64, _i32, _f32, _i32, _P, _P, _P, _P, _P, _P, _sz, _P],
                "pdmp_logdet": [_FP, _P, _i64, _i32, _f32, _P, _P, _P],
                "pdmp_occupancy_query": [_FP, _P, _i64, _P, _P, _P, _P],
                "pdmp_box_labels": [_i32, _P, _i64, _P, _i64, _P, _P],
                "pdmp_lipschitz_bound": [_FP, ctypes.POINTER(_f64), ctypes.POINTER(_f64), _i32,
                                         ctypes.POINTER(_f64), ctypes.POINTER(_f64), _P],
                "pdmp_fit_occupancy": [_FP, _P, _P, _i64, _f32, _i32, _i32, _P, ctypes.POINTER(_f32),
                                       ctypes.POINTER(_f32), ctypes.POINTER(_f32), _P, _sz, _P],
            }
            for name, argt in sigs.items():
                fn = getattr(L, name)
                fn.argtypes = argt
                fn.restype = _i32
            L.pdmp_morph_workspace.argtypes = [_FP, _i64]
            L.pdmp_morph_workspace.restype = _sz
            L.pdmp_morph_vjp_workspace.argtypes = [_FP, _i64, _i32, _i32, _i32]
            L.pdmp_morph_vjp_workspace.restype = _sz
            L.pdmp_fit_workspace.argtypes = [_i64, _i64]
            L.pdmp_fit_workspace.restype = _sz
            _lib = L
    return _lib


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(status: int, what: str):
    if status != OK:
        raise PdmpError(status, what)


def _ptr(t: torch.Tensor | None, dtype=torch.float32, shape=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


class DeviceField:
    """An occupancy field resident on the GPU (float32, contiguous).

    kind RBF: centres = mu (M x d), gamma > 0.   kind RFF: centres = omega
    (M x d), phase = b (M).  ``lipschitz`` (optional) is a bound on |Hess c|
    that calls taking a step size check eta against.
    """

    def __init__(self, kind, centres, w, gamma=0.0, phase=None, bias=0.0, lipschitz=0.0, device="cuda"):
        def dev(a):
            if a is None:
                return None
            t = a if isinstance(a, torch.Tensor) else torch.as_tensor(a)
            return t.to(device=device, dtype=torch.float32).contiguous()

        self.kind = int(kind)
        self.centres = dev(centres)
        self.w = dev(w)
        self.phase = dev(phase) if self.kind == RFF else None
        self.gamma = float(gamma)
        self.bias = float(bias)
        self.lipschitz = float(lipschitz)
        if self.centres.dim() != 2:
            raise ValueError("centres must be M x d")

    @classmethod
    def from_host(cls, f, lipschitz: float = 0.0, device="cuda"):
        """From any object with kind, centres, w, gamma, phase, bias (e.g. workloads.Field)."""
        return cls(f.kind, f.centres, f.w, f.gamma, f.phase, f.bias, lipschitz, device)

    @property
    def d(self) -> int:
        return int(self.centres.shape[1])

    @property
    def M(self) -> int:
        return int(self.centres.shape[0])

    def with_weights(self, w, bias=None) -> "DeviceField":
        return DeviceField(self.kind, self.centres, w, self.gamma, self.phase,
                           self.bias if bias is None else bias, self.lipschitz, self.centres.device)

    def struct(self) -> _Field:
        f = _Field()
        f.kind, f.d, f.M = self.kind, self.d, self.M
        f.centres = self.centres.data_ptr()
        f.phase = self.phase.data_ptr() if self.phase is not None else None
        f.gamma = self.gamma
        f.w = self.w.data_ptr()
        f.bias = self.bias
        f.lipschitz = self.lipschitz
        return f


def stream_status():
    """Synchronises torch's current stream; returns (status, detail)."""
    detail = _i32(0)
    st = lib().pdmp_stream_status(_stream(), ctypes.byref(detail))
    return int(st), int(detail.value)


def morph_workspace(field: DeviceField, N: int) -> int:
    f = field.struct()
    return int(lib().pdmp_morph_workspace(ctypes.byref(f), int(N)))


def _workspace(field, N, fast, ws):
    """(pointer, bytes) of the morph workspace: the caller's, a fresh one, or none."""
    if not fast:
        return None, 0, None
    nbytes = morph_workspace(field, N)
    if nbytes == 0:
        return None, 0, None
    if ws is None or ws.numel() < nbytes:
        ws = torch.empty(nbytes, dtype=torch.uint8, device=field.centres.device)
    return ctypes.c_void_p(ws.data_ptr()), nbytes, ws


def morph(field: DeviceField, x0: torch.Tensor, T: int, eta: float, out: torch.Tensor | None = None,
          ckpt: torch.Tensor | None = None, k: int = 0, fast: bool = True,
          ws: torch.Tensor | None = None) -> torch.Tensor:
    """x_T of T Euler steps of Eq. (1) for every row of x0 (N x d).  ``out``
    may be x0 itself.  ``ckpt`` ((T/k) x N x d) receives x_k, x_2k, ..., x_T.
    ``fast`` gives the library a workspace (``ws``, a uint8 CUDA tensor, or a
    fresh one) so that 2-D / 3-D RBF fields take the fast path."""
    N = x0.shape[0]
    d = field.d
    if out is None:
        out = torch.empty_like(x0)
    wp, wb, _keep = _workspace(field, N, fast, ws)
    f = field.struct()
    st = lib().pdmp_morph(ctypes.byref(f), _ptr(x0, shape=(N, d), name="x0"), N, int(T), float(eta),
                          _ptr(out, shape=(N, d), name="out"),
                          _ptr(ckpt, shape=(T // k if k else 0, N, d), name="ckpt") if ckpt is not None else None,
                          int(k), wp, wb, _stream())
    _check(st, "pdmp_morph")
    return out


def morph_trace(field: DeviceField, x0: torch.Tensor, T: int, eta: float, fast: bool = True):
    """(traj ((T+1) x N x d), steps (T x N x d)): every state and every FP32
    increment as the morph kernel computes it (diagnostic)."""
    N, d = x0.shape[0], field.d
    traj = torch.empty(T + 1, N, d, device=x0.device, dtype=torch.float32)
    steps = torch.empty(max(T, 1), N, d, device=x0.device, dtype=torch.float32)
    wp, wb, _keep = _workspace(field, N, fast, None)
    f = field.struct()
    st = lib().pdmp_morph_trace(ctypes.byref(f), _ptr(x0, shape=(N, d), name="x0"), N, int(T), float(eta),
                                _ptr(traj), _ptr(steps), wp, wb, _stream())
    _check(st, "pdmp_morph_trace")
    return traj, steps[:T]


def morph_noalloc(field: DeviceField, x0: torch.Tensor, T: int, eta: float,
                  out: torch.Tensor | None = None) -> torch.Tensor:
    """pdmp_morph_noalloc: the fast RBF morph on the library's built-in
    scratch, for callers that cannot allocate device memory (RBF, d = 2 or 3,
    N <= 2^20, M <= 16384; calls must not overlap on the GPU)."""
    L = lib()
    fn = L.pdmp_morph_noalloc
    fn.argtypes = [_FP, _P, _i64, _i32, _f32, _P, _P]
    fn.restype = _i32
    N, d = x0.shape[0], field.d
    if out is None:
        out = torch.empty_like(x0)
    f = field.struct()
    st = fn(ctypes.byref(f), _ptr(x0, shape=(N, d), name="x0"), N, int(T), float(eta),
            _ptr(out, shape=(N, d), name="out"), _stream())
    _check(st, "pdmp_morph_noalloc")
    return out


def morph_vjp_workspace(field: DeviceField, N: int, T: int, k: int, want_param_grad: bool) -> int:
    f = field.struct()
    return int(lib().pdmp_morph_vjp_workspace(ctypes.byref(f), int(N), int(T), int(k), int(bool(want_param_grad))))


def morph_vjp(field: DeviceField, x0: torch.Tensor, T: int, eta: float, k: int, gT: torch.Tensor,
              ckpt: torch.Tensor | None = None, want_param_grad: bool = False, g0: torch.Tensor | None = None):
    """g0 = (dx_T/dx_0)^T gT per sample; with want_param_grad also (gw, gbias)
    = d/d(w, bias) of sum_n <gT[n], x_T[n]>."""
    N, d = x0.shape[0], field.d
    if g0 is None:
        g0 = torch.empty_like(x0)
    gw = gb = ws = None
    nbytes = 0
    if want_param_grad:
        gw = torch.empty(field.M, device=x0.device, dtype=torch.float32)
        gb = torch.empty(1, device=x0.device, dtype=torch.float32)
        nbytes = morph_vjp_workspace(field, N, T, k, True)
        ws = torch.empty(max(nbytes, 16), device=x0.device, dtype=torch.uint8)
    f = field.struct()
    st = lib().pdmp_morph_vjp(ctypes.byref(f), _ptr(x0, shape=(N, d), name="x0"), N, int(T), float(eta), int(k),
                              _ptr(ckpt, shape=(T // k, N, d), name="ckpt") if ckpt is not None else None,
                              _ptr(gT, shape=(N, d), name="gT"), _ptr(g0, shape=(N, d), name="g0"),
                              _ptr(gw, name="gw"), _ptr(gb, name="gbias"),
                              _ptr(ws, dtype=torch.uint8, name="ws") if ws is not None else None, nbytes, _stream())
    _check(st, "pdmp_morph_vjp")
    if want_param_grad:
        return g0, gw, gb
    return g0


def logdet(field: DeviceField, x0: torch.Tensor, T: int, eta: float, want_xT: bool = False):
    N, d = x0.shape[0], field.d
    ld = torch.empty(N, device=x0.device, dtype=torch.float32)
    xT = torch.empty_like(x0) if want_xT else None
    f = field.struct()
    st = lib().pdmp_logdet(ctypes.byref(f), _ptr(x0, shape=(N, d), name="x0"), N, int(T), float(eta),
                           _ptr(ld, name="logdet"), _ptr(xT, name="xT"), _stream())
    _check(st, "pdmp_logdet")
    return (ld, xT) if want_xT else ld


def occupancy_query(field: DeviceField, x: torch.Tensor, want=("c", "s", "grad")):
    N, d = x.shape[0], field.d
    c = torch.empty(N, device=x.device, dtype=torch.float32) if "c" in want else None
    s = torch.empty(N, device=x.device, dtype=torch.float32) if "s" in want else None
    g = torch.empty(N, d, device=x.device, dtype=torch.float32) if "grad" in want else None
    f = field.struct()
    st = lib().pdmp_occupancy_query(ctypes.byref(f), _ptr(x, shape=(N, d), name="x"), N, _ptr(c), _ptr(s), _ptr(g),
                                    _stream())
    _check(st, "pdmp_occupancy_query")
    return {"c": c, "s": s, "grad": g}


def box_labels(boxes: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    N, d = x.shape
    nb = boxes.shape[0]
    lab = torch.empty(N, device=x.device, dtype=torch.uint8)
    st = lib().pdmp_box_labels(int(d), _ptr(boxes, shape=(nb, 2 * d), name="boxes") if nb else None, nb,
                               _ptr(x, name="x"), N, _ptr(lab, dtype=torch.uint8, name="label"), _stream())
    _check(st, "pdmp_box_labels")
    return lab


def lipschitz_bound(field: DeviceField, lo=None, hi=None, cells: int = 64):
    """(L, G): certified bounds on |Hess c|_2 and |grad c|_2 (FP64 on the GPU;
    synchronises the current stream)."""
    d = field.d
    lo_a = (_f64 * d)(*([float(v) for v in lo] if lo is not None else [0.0] * d))
    hi_a = (_f64 * d)(*([float(v) for v in hi] if hi is not None else [1.0] * d))
    L, G = _f64(0.0), _f64(0.0)
    f = field.struct()
    st = lib().pdmp_lipschitz_bound(ctypes.byref(f), lo_a, hi_a, int(cells), ctypes.byref(L), ctypes.byref(G),
                                    _stream())
    _check(st, "pdmp_lipschitz_bound")
    return float(L.value), float(G.value)


def fit_workspace(M: int, n: int) -> int:
    return int(lib().pdmp_fit_workspace(int(M), int(n)))


def fit_occupancy(field: DeviceField, X: torch.Tensor, y: torch.Tensor, l2: float, power_iters: int, iters: int):
    """(w (M, device), bias, final loss, step alpha) of the BCE fit."""
    n, d = X.shape
    w = torch.empty(field.M, device=X.device, dtype=torch.float32)
    nbytes = fit_workspace(field.M, n)
    ws = torch.empty(nbytes, device=X.device, dtype=torch.uint8)
    b, loss, alpha = _f32(0), _f32(0), _f32(0)
    f = field.struct()
    st = lib().pdmp_fit_occupancy(ctypes.byref(f), _ptr(X, shape=(n, field.d), name="X"),
                                  _ptr(y, dtype=torch.uint8, shape=(n,), name="y"), n, float(l2), int(power_iters),
                                  int(iters), _ptr(w, name="w"), ctypes.byref(b), ctypes.byref(loss),
                                  ctypes.byref(alpha), _ptr(ws, dtype=torch.uint8, name="ws"), nbytes, _stream())
    _check(st, "pdmp_fit_occupancy")
    return w, float(b.value), float(loss.value), float(alpha.value)
