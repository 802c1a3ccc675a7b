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
    "PdmpError", "DeviceField", "lib", "stream_wait", "morph", "morph_trace", "morph_workspace", "morph_inverse", "log_density", "morph_culled", "morph_culled_workspace", "cull_radius", "DeviceTanhNet", "tanh_net_morph", "cspace_morph", "cspace_workspace",
    "cspace_lipschitz", "chain_struct", "Queue", "Sampler",
    "tanh_net_query", "tanh_net_lipschitz", "morph_vjp", "morph_vjp_workspace", "logdet",
    "occupancy_query", "box_labels", "lipschitz_bound", "fit_occupancy", "fit_workspace", "stream_status", "Batch",
    "Surrogate", "displacement_rms", "morph_autograd",
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


class _SamplerConfig(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("lo", ctypes.c_float * 8), ("hi", ctypes.c_float * 8),
                ("batch", ctypes.c_int32), ("capacity", ctypes.c_int64), ("T", ctypes.c_int32),
                ("eta", ctypes.c_float), ("seed", ctypes.c_uint64)]


class _SamplerStats(ctypes.Structure):
    _fields_ = [("produced", ctypes.c_int64), ("batches", ctypes.c_int64), ("drawn_morphed", ctypes.c_int64),
                ("drawn_prior", ctypes.c_int64), ("queued", ctypes.c_int64), ("error", ctypes.c_int32)]


class _Chain(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("p", ctypes.c_int32), ("base", ctypes.c_float * 2),
                ("lengths", ctypes.c_float * 16)]


class _TanhNet(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("H", ctypes.c_int32), ("W1", ctypes.c_void_p), ("b1", ctypes.c_void_p),
                ("W2", ctypes.c_void_p), ("b2", ctypes.c_void_p), ("w3", ctypes.c_void_p), ("b3", ctypes.c_float),
                ("lipschitz", ctypes.c_double)]
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
                "pdmp_stream_wait": [_P, _i32, ctypes.POINTER(_i32)],
                "pdmp_selftest_stage_wait": [_P, _P, _i64, _i32, _P],
                "pdmp_morph": [_FP, _P, _i64, _i32, _f32, _P, _P, _i32, _P, _sz, _P],
                "pdmp_morph_trace": [_FP, _P, _i64, _i32, _f32, _P, _P, _P, _sz, _P],
                "pdmp_morph_vjp": [_FP, _P, _i64, _i32, _f32, _i32, _P, _P, _P, _P, _P, _P, _sz, _P],
                "pdmp_logdet": [_FP, _P, _i64, _i32, _f32, _P, _P, _P, _sz, _P],
                "pdmp_queue_create": [_i32, _i64, ctypes.POINTER(_P)],
                "pdmp_queue_push": [_P, _P, _i64, _i32, ctypes.POINTER(_i64)],
                "pdmp_queue_pop": [_P, _P, _i64, ctypes.POINTER(_i64)],
                "pdmp_queue_size": [_P, ctypes.POINTER(_i64)],
                "pdmp_queue_close": [_P],
                "pdmp_queue_destroy": [_P],
                "pdmp_sampler_create": [_FP, ctypes.POINTER(_SamplerConfig), ctypes.POINTER(_P)],
                "pdmp_sampler_draw": [_P, _P, _i64, ctypes.POINTER(_i64)],
                "pdmp_sampler_stats": [_P, ctypes.POINTER(_SamplerStats)],
                "pdmp_sampler_destroy": [_P],
                "pdmp_cspace_morph": [_FP, ctypes.POINTER(_Chain), _P, _i64, _i32, _f32, _P, _P, _sz, _P],
                "pdmp_cspace_lipschitz": [ctypes.POINTER(_Chain), _f64, _f64, ctypes.POINTER(_f64)],
                "pdmp_tanh_net_morph": [ctypes.POINTER(_TanhNet), _P, _i64, _i32, _f32, _P, _P, _i32, _P],
                "pdmp_tanh_net_query": [ctypes.POINTER(_TanhNet), _P, _i64, _P, _P, _P, _P],
                "pdmp_tanh_net_lipschitz": [ctypes.POINTER(_TanhNet), ctypes.POINTER(_f64), ctypes.POINTER(_f64), _P],
                "pdmp_morph_culled": [_FP, _P, _i64, _i32, _f32, _f32, _P, _P, _i32, _P, _sz, _P, _P],
                "pdmp_cull_radius": [_FP, _f32, ctypes.POINTER(_f32), ctypes.POINTER(_f64), _P],
                "pdmp_morph_inverse": [_FP, _P, _i64, _i32, _f32, _f32, _i32, _P, _P, _P, _sz, _P, _P],
                "pdmp_log_density": [_FP, _P, _i64, _i32, _f32, _P, _P, _f32, _i32, _P, _P, _P, _sz, _P],
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
            L.pdmp_cspace_workspace.argtypes = [_FP, ctypes.POINTER(_Chain), _i64]
            L.pdmp_cspace_workspace.restype = _sz
            L.pdmp_morph_culled_workspace.argtypes = [_FP, _i64]
            L.pdmp_morph_culled_workspace.restype = _sz
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



def stream_wait(timeout_ms: int):
    """(status, detail): waits at most timeout_ms for the current stream's
    queued work (host-side watchdog); status PDMP_ERR_TIMEOUT (6) if it is
    still running, else as stream_status."""
    d = ctypes.c_int32(0)
    st = lib().pdmp_stream_wait(_stream(), int(timeout_ms), ctypes.byref(d))
    return int(st), int(d.value)

def selftest_stage_wait(limit_clocks: int, src: torch.Tensor | None = None, dst: torch.Tensor | None = None):
    """Runs the kernels' bounded stage-copy wait once: with src and dst (16
    float32 each on the device) the copy completes and dst receives src;
    without them the wait runs out after limit_clocks SM clocks and raises
    PDMP_FLAG_STAGE_TIMEOUT.  Returns stream_status()."""
    with_copy = src is not None
    _check(lib().pdmp_selftest_stage_wait(_ptr(src, shape=(16,), name="src") if with_copy else None,
                                          _ptr(dst, shape=(16,), name="dst") if with_copy else None,
                                          int(limit_clocks), int(with_copy), _stream()), "pdmp_selftest_stage_wait")
    return stream_status()


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


class Queue:
    """The bounded concurrent FIFO bucket of host samples (pdmp_queue_*); host only."""

    def __init__(self, d: int, capacity: int):
        h = ctypes.c_void_p()
        _check(lib().pdmp_queue_create(int(d), int(capacity), ctypes.byref(h)), "pdmp_queue_create")
        self._h, self.d = h, int(d)

    def push(self, x, timeout_ms: int = 0) -> int:
        import numpy as np
        a = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, self.d)
        n = ctypes.c_int64(0)
        _check(lib().pdmp_queue_push(self._h, a.ctypes.data_as(ctypes.c_void_p), a.shape[0], int(timeout_ms),
                                     ctypes.byref(n)), "pdmp_queue_push")
        return int(n.value)

    def pop(self, n: int):
        import numpy as np
        out = np.empty((int(n), self.d), dtype=np.float32)
        got = ctypes.c_int64(0)
        _check(lib().pdmp_queue_pop(self._h, out.ctypes.data_as(ctypes.c_void_p), int(n), ctypes.byref(got)),
               "pdmp_queue_pop")
        return out[:got.value]

    def size(self) -> int:
        n = ctypes.c_int64(0)
        _check(lib().pdmp_queue_size(self._h, ctypes.byref(n)), "pdmp_queue_size")
        return int(n.value)

    def close(self):
        _check(lib().pdmp_queue_close(self._h), "pdmp_queue_close")

    def __del__(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().pdmp_queue_destroy(self._h)
            self._h = None


class Sampler:
    """The diffeomorphic sampler of Sec. 3.3: a background thread fills a bucket
    with morphed samples; draw() never waits for the GPU and falls back to the
    prior (uniform on [lo, hi]) when the bucket is empty."""

    def __init__(self, field: DeviceField, lo, hi, T: int, eta: float, batch: int = 65536,
                 capacity: int = 1 << 20, seed: int = 0):
        c = _SamplerConfig()
        c.d = field.d
        for j in range(field.d):
            c.lo[j], c.hi[j] = float(lo[j]), float(hi[j])
        c.batch, c.capacity, c.T, c.eta, c.seed = int(batch), int(capacity), int(T), float(eta), int(seed)
        self._field = field                      # keeps the device arrays alive
        self._fs = field.struct()
        h = ctypes.c_void_p()
        _check(lib().pdmp_sampler_create(ctypes.byref(self._fs), ctypes.byref(c), ctypes.byref(h)),
               "pdmp_sampler_create")
        self._h, self.d = h, field.d

    def draw(self, n: int):
        """(samples n x d float32 on the host, how many of them, first, are morphed)."""
        import numpy as np
        out = np.empty((int(n), self.d), dtype=np.float32)
        m = ctypes.c_int64(0)
        _check(lib().pdmp_sampler_draw(self._h, out.ctypes.data_as(ctypes.c_void_p), int(n), ctypes.byref(m)),
               "pdmp_sampler_draw")
        return out, int(m.value)

    def stats(self) -> dict:
        st = _SamplerStats()
        _check(lib().pdmp_sampler_stats(self._h, ctypes.byref(st)), "pdmp_sampler_stats")
        return {k: int(getattr(st, k)) for k, _ in _SamplerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(lib().pdmp_sampler_destroy(self._h), "pdmp_sampler_destroy")
            self._h = None

    def __del__(self):
        self.close()


def chain_struct(chain) -> _Chain:
    """A planar serial chain (any object with lengths, base, p) as the C struct."""
    c = _Chain()
    ln = [float(v) for v in chain.lengths]
    if not 1 <= len(ln) <= 16:
        raise ValueError("a chain has 1 to 16 links")
    c.n, c.p = len(ln), int(chain.p)
    c.base[0], c.base[1] = (float(v) for v in chain.base)
    for i, v in enumerate(ln):
        c.lengths[i] = v
    return c


def cspace_workspace(field: DeviceField, chain, N: int) -> int:
    f, c = field.struct(), chain_struct(chain)
    return int(lib().pdmp_cspace_workspace(ctypes.byref(f), ctypes.byref(c), int(N)))


def cspace_morph(field: DeviceField, chain, q0: torch.Tensor, T: int, eta: float, out: torch.Tensor | None = None,
                 ws: torch.Tensor | None = None):
    """Eq. (1) in joint space with the pulled-back gradient of Eq. (3)."""
    f, c = field.struct(), chain_struct(chain)
    N = q0.shape[0]
    qT = torch.empty_like(q0) if out is None else out
    if ws is None:
        ws = torch.empty(max(cspace_workspace(field, chain, N), 16), dtype=torch.uint8, device=q0.device)
    _check(lib().pdmp_cspace_morph(ctypes.byref(f), ctypes.byref(c), _ptr(q0, shape=(N, c.n), name="q0"), N, int(T),
                                   float(eta), _ptr(qT), _ptr(ws, dtype=torch.uint8), ws.numel(), _stream()),
           "pdmp_cspace_morph")
    return qT


def cspace_lipschitz(chain, Lx: float, Gx: float) -> float:
    """Certified bound on the joint-space Hessian of the summed body-point occupancy."""
    c = chain_struct(chain)
    out = ctypes.c_double(0)
    _check(lib().pdmp_cspace_lipschitz(ctypes.byref(c), float(Lx), float(Gx), ctypes.byref(out)),
           "pdmp_cspace_lipschitz")
    return float(out.value)


class DeviceTanhNet:
    """The tanh occupancy network of Sec. 3.1 (d -> H -> H -> 1) resident on the GPU (float32)."""

    def __init__(self, W1, b1, W2, b2, w3, b3: float, lipschitz: float = 0.0, device="cuda"):
        t = lambda a: torch.as_tensor(a, dtype=torch.float32).to(device).contiguous()
        self.W1, self.b1, self.W2, self.b2, self.w3 = t(W1), t(b1), t(W2), t(b2), t(w3)
        self.b3 = float(b3)
        self.lipschitz = float(lipschitz)
        self.H, self.d = self.W1.shape

    @classmethod
    def from_host(cls, net, lipschitz: float = 0.0, device="cuda"):
        """From any object with W1, b1, W2, b2, w3, b3 (e.g. workloads.TanhNet)."""
        return cls(net.W1, net.b1, net.W2, net.b2, net.w3, net.b3, lipschitz, device)

    def struct(self) -> _TanhNet:
        s = _TanhNet()
        s.d, s.H = self.d, self.H
        s.W1, s.b1, s.W2, s.b2, s.w3 = (t.data_ptr() for t in (self.W1, self.b1, self.W2, self.b2, self.w3))
        s.b3, s.lipschitz = self.b3, self.lipschitz
        return s


def tanh_net_morph(net: DeviceTanhNet, x0: torch.Tensor, T: int, eta: float, out: torch.Tensor | None = None,
                   ckpt: torch.Tensor | None = None, k: int = 0):
    """Eq. (1) by Euler's method with the tanh network's occupancy as the cost."""
    N, d = x0.shape[0], net.d
    xT = torch.empty_like(x0) if out is None else out
    s = net.struct()
    _check(lib().pdmp_tanh_net_morph(ctypes.byref(s), _ptr(x0, shape=(N, d), name="x0"), N, int(T), float(eta),
                                     _ptr(xT), _ptr(ckpt, name="ckpt"), int(k), _stream()), "pdmp_tanh_net_morph")
    return xT


def tanh_net_query(net: DeviceTanhNet, x: torch.Tensor):
    """(c, s, grad c) of the tanh network at points x (N x d)."""
    N, d = x.shape[0], net.d
    c = torch.empty(N, device=x.device)
    s_out = torch.empty(N, device=x.device)
    g = torch.empty(N, d, device=x.device)
    s = net.struct()
    _check(lib().pdmp_tanh_net_query(ctypes.byref(s), _ptr(x, shape=(N, d), name="x"), N, _ptr(c), _ptr(s_out),
                                     _ptr(g), _stream()), "pdmp_tanh_net_query")
    return c, s_out, g


def tanh_net_lipschitz(net: DeviceTanhNet):
    """(L, G): certified bounds on sup |Hess c|_2 and sup |grad s| (FP64, host)."""
    L, G = ctypes.c_double(0), ctypes.c_double(0)
    s = net.struct()
    _check(lib().pdmp_tanh_net_lipschitz(ctypes.byref(s), ctypes.byref(L), ctypes.byref(G), _stream()),
           "pdmp_tanh_net_lipschitz")
    return float(L.value), float(G.value)


def cull_radius(field: DeviceField, eps: float):
    """(r_cut, W): the cut-off radius whose dropped features change s and |grad s| by at most eps."""
    r = ctypes.c_float(0)
    W = ctypes.c_double(0)
    f = field.struct()
    _check(lib().pdmp_cull_radius(ctypes.byref(f), float(eps), ctypes.byref(r), ctypes.byref(W), _stream()),
           "pdmp_cull_radius")
    return float(r.value), float(W.value)


def surrogate_workspace(field: DeviceField, N: int) -> int:
    """Bytes of device workspace pdmp_surrogate_infer(_culled) needs for N samples."""
    L = _mlp_sigs()
    f = field.struct()
    return int(L.pdmp_surrogate_workspace(ctypes.byref(f), int(N)))


def morph_culled_workspace(field: DeviceField, N: int) -> int:
    """Bytes of device workspace pdmp_morph_culled needs for N samples."""
    f = field.struct()
    return int(lib().pdmp_morph_culled_workspace(ctypes.byref(f), int(N)))


def morph_culled(field: DeviceField, x0: torch.Tensor, T: int, eta: float, r_cut: float, out: torch.Tensor | None = None,
                 ckpt: torch.Tensor | None = None, k: int = 0, ws: torch.Tensor | None = None,
                 work: torch.Tensor | None = None):
    """The morph of Eq. (1) with features farther than r_cut from a sample tile dropped (RBF, d = 2, 3)."""
    L = lib()
    N, d = x0.shape[0], field.d
    xT = torch.empty_like(x0) if out is None else out
    f = field.struct()
    if ws is None:
        ws = torch.empty(max(morph_culled_workspace(field, N), 16), device=x0.device, dtype=torch.uint8)
    _check(L.pdmp_morph_culled(ctypes.byref(f), _ptr(x0, shape=(N, d), name="x0"), N, int(T), float(eta),
                               float(r_cut), _ptr(xT), _ptr(ckpt, name="ckpt"), int(k), _ptr(ws, dtype=torch.uint8),
                               ws.numel(), _ptr(work, dtype=torch.int64, name="work"), _stream()),
           "pdmp_morph_culled")
    return xT


def morph_inverse(field: DeviceField, z: torch.Tensor, T: int, eta: float, tol: float = 1e-6, maxit: int = 60,
                  want_iters: bool = False, out: torch.Tensor | None = None, fast: bool = True,
                  ws: torch.Tensor | None = None, work: torch.Tensor | None = None):
    """Eq. (2): the inverse of the T-step map by per-step fixed points.
    ``fast`` gives the library the morph's workspace so that 2-D / 3-D RBF
    fields run on sorted tiles; ``work`` (int64 CUDA tensor of one element)
    is incremented by the feature evaluations performed."""
    fn = lib().pdmp_morph_inverse
    N, d = z.shape[0], field.d
    y = torch.empty_like(z) if out is None else out
    its = torch.empty(N, device=z.device, dtype=torch.int32) if want_iters else None
    wp, wb, _keep = _workspace(field, N, fast, ws)
    f = field.struct()
    _check(fn(ctypes.byref(f), _ptr(z, shape=(N, d), name="z"), N, int(T), float(eta), float(tol), int(maxit),
              _ptr(y, shape=(N, d), name="out"), _ptr(its, dtype=torch.int32, name="iters"), wp, wb,
              _ptr(work, dtype=torch.int64, name="work"), _stream()), "pdmp_morph_inverse")
    return (y, its) if want_iters else y


def log_density(field: DeviceField, z: torch.Tensor, T: int, eta: float, lo, hi, tol: float = 1e-6,
                maxit: int = 60, fast: bool = True, ws: torch.Tensor | None = None):
    """log p_z of morphed samples for a base density uniform on [lo, hi]; returns (log_p, y = phi^{-1}(z))."""
    fn = lib().pdmp_log_density
    N, d = z.shape[0], field.d
    lo_h = (ctypes.c_double * d)(*[float(v) for v in lo])
    hi_h = (ctypes.c_double * d)(*[float(v) for v in hi])
    y = torch.empty_like(z)
    lp = torch.empty(N, device=z.device, dtype=torch.float32)
    wp, wb, _keep = _workspace(field, N, fast, ws)
    f = field.struct()
    _check(fn(ctypes.byref(f), _ptr(z, shape=(N, d), name="z"), N, int(T), float(eta), ctypes.addressof(lo_h),
              ctypes.addressof(hi_h), float(tol), int(maxit), _ptr(y), _ptr(lp), wp, wb, _stream()),
           "pdmp_log_density")
    return lp, y


def morph_vjp_workspace(field: DeviceField, N: int, T: int, k: int, want_param_grad: bool | int) -> int:
    """Bytes of workspace for pdmp_morph_vjp; want_param_grad 1 (True) sizes it
    for the fastest kernel, 2 for the parameter gradient's rows alone."""
    f = field.struct()
    return int(lib().pdmp_morph_vjp_workspace(ctypes.byref(f), int(N), int(T), int(k), int(want_param_grad)))


def morph_vjp(field: DeviceField, x0: torch.Tensor, T: int, eta: float, k: int, gT: torch.Tensor,
              ckpt: torch.Tensor | None = None, want_param_grad: bool = False, g0: torch.Tensor | None = None,
              fast: bool = True, ws: torch.Tensor | None = None):
    """g0 = (dx_T/dx_0)^T gT per sample; with want_param_grad also (gw, gbias)
    = d/d(w, bias) of sum_n <gT[n], x_T[n]>.  Without the parameter gradient,
    ``fast`` gives the library a workspace (``ws`` or a fresh one) so that RFF
    fields with d <= 7 and k <= 16 run on the tensor cores; with it, the
    parameter gradient does too (``fast=False``: the direct kernel)."""
    N, d = x0.shape[0], field.d
    if g0 is None:
        g0 = torch.empty_like(x0)
    gw = gb = None
    nbytes = 0
    if want_param_grad:
        gw = torch.empty(field.M, device=x0.device, dtype=torch.float32)
        gb = torch.empty(1, device=x0.device, dtype=torch.float32)
        nbytes = morph_vjp_workspace(field, N, T, k, 1 if fast else 2)
        if ws is None or ws.numel() < nbytes:
            ws = torch.empty(max(nbytes, 16), device=x0.device, dtype=torch.uint8)
    elif fast:
        nbytes = morph_vjp_workspace(field, N, T, k, False)
        if nbytes == 0:
            ws = None
        elif ws is None or ws.numel() < nbytes:
            ws = torch.empty(nbytes, device=x0.device, dtype=torch.uint8)
    else:
        ws = None
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


def logdet(field: DeviceField, x0: torch.Tensor, T: int, eta: float, want_xT: bool = False, fast: bool = True,
           ws: torch.Tensor | None = None):
    """sum_t log det(I - eta Hess c(x_t)) per sample (and x_T); ``fast`` gives
    the library the morph's workspace, with which RFF fields with d <= 7 run
    on the tensor cores."""
    N, d = x0.shape[0], field.d
    ld = torch.empty(N, device=x0.device, dtype=torch.float32)
    xT = torch.empty_like(x0) if want_xT else None
    wp, wb, _keep = _workspace(field, N, fast, ws)
    f = field.struct()
    st = lib().pdmp_logdet(ctypes.byref(f), _ptr(x0, shape=(N, d), name="x0"), N, int(T), float(eta),
                           _ptr(ld, name="logdet"), _ptr(xT, name="xT"), wp, wb, _stream())
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


# ---------------------------------------------------------------------------
# many environments in one persistent launch
class _Env(ctypes.Structure):
    _fields_ = [("field", _Field), ("x0", ctypes.c_void_p), ("xT", ctypes.c_void_p), ("N", ctypes.c_int64),
                ("eta", ctypes.c_float), ("T", ctypes.c_int32)]


class BatchPlan(ctypes.Structure):
    _fields_ = [("n_envs", ctypes.c_int32), ("variant", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("block", ctypes.c_int32), ("smem_bytes", ctypes.c_size_t), ("n_units", ctypes.c_int64),
                ("total_N", ctypes.c_int64), ("total_M", ctypes.c_int64), ("total_cells", ctypes.c_int64),
                ("nchunks", ctypes.c_int64), ("ws_bytes", ctypes.c_size_t), ("work", ctypes.c_double),
                ("off", ctypes.c_size_t * 12)]


def _batch_sigs():
    L = lib()
    if getattr(L, "_batch_ready", False):
        return L
    EP = ctypes.POINTER(_Env)
    PP = ctypes.POINTER(BatchPlan)
    L.pdmp_batch_variants.restype = _i32
    L.pdmp_batch_workspace.argtypes = [EP, _i32, _i32]
    L.pdmp_batch_workspace.restype = _sz
    for name, argt in {
        "pdmp_batch_prepare": [EP, _i32, _i32, _P, _sz, PP, _P],
        "pdmp_morph_batched": [PP, _P, _P],
        "pdmp_batch_autotune": [EP, _i32, _i32, _P, _sz, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_float), PP,
                                _P],
        "pdmp_batch_graph_create": [PP, _P, _P, ctypes.POINTER(ctypes.c_void_p)],
        "pdmp_graph_launch": [_P, _P],
        "pdmp_graph_destroy": [_P],
    }.items():
        fn = getattr(L, name)
        fn.argtypes = argt
        fn.restype = _i32
    L._batch_ready = True
    return L


class Batch:
    """Several environments (RBF fields in 2-D or 3-D, each with its own
    samples, step size and step count) morphed by one persistent launch.

    envs: list of (DeviceField, x0 (N x d CUDA tensor), eta, T).  Outputs are
    written to ``self.outputs`` (one tensor per environment).  ``prepare`` picks
    a tile shape (``autotune`` times all of them; results are cached in a JSON
    file keyed by the environments' shapes), ``run`` launches, ``capture``
    builds a CUDA graph of ``run`` on a side stream and ``replay`` launches it.
    """

    def __init__(self, envs, cache_path: str | None = None):
        self.fields = [e[0] for e in envs]
        self.inputs = [e[1] for e in envs]
        self.outputs = [torch.empty_like(e[1]) for e in envs]
        self.etas = [float(e[2]) for e in envs]
        self.Ts = [int(e[3]) for e in envs]
        n = len(envs)
        self._structs = [f.struct() for f in self.fields]
        self._envs = (_Env * n)()
        for i in range(n):
            self._envs[i].field = self._structs[i]
            self._envs[i].x0 = self.inputs[i].data_ptr() if self.inputs[i].numel() else None
            self._envs[i].xT = self.outputs[i].data_ptr() if self.outputs[i].numel() else None
            self._envs[i].N = int(self.inputs[i].shape[0])
            self._envs[i].eta = self.etas[i]
            self._envs[i].T = self.Ts[i]
        self.n = n
        self.plan = BatchPlan()
        self.ws = None
        self.graph = None
        self.cache_path = cache_path or os.environ.get(
            "PDMP_AUTOTUNE_CACHE", os.path.join(os.path.dirname(_build.LIB), "autotune.json"))
        L = _batch_sigs()
        self.n_variants = int(L.pdmp_batch_variants())
        need = max(int(L.pdmp_batch_workspace(self._envs, n, v)) for v in range(self.n_variants))
        if need == 0:
            raise PdmpError(1, "pdmp_batch_workspace")
        self.ws = torch.empty(need, dtype=torch.uint8, device=self.inputs[0].device)

    def signature(self) -> str:
        import hashlib
        h = hashlib.sha256()
        for f, x, T in zip(self.fields, self.inputs, self.Ts):
            h.update(f"{f.d},{f.M},{x.shape[0]},{T};".encode())
        return f"{torch.cuda.get_device_name()}|{self.n}|{h.hexdigest()[:20]}"

    def prepare(self, variant: int = 0):
        L = _batch_sigs()
        st = L.pdmp_batch_prepare(self._envs, self.n, int(variant), ctypes.c_void_p(self.ws.data_ptr()),
                                  self.ws.numel(), ctypes.byref(self.plan), _stream())
        _check(st, "pdmp_batch_prepare")
        return self.plan

    def autotune(self, reps: int = 2, use_cache: bool = True):
        """(best variant, times in ms per variant or None when read from the cache)."""
        import json
        key = self.signature()
        cache = {}
        if use_cache and os.path.exists(self.cache_path):
            try:
                with open(self.cache_path) as f:
                    cache = json.load(f)
            except (OSError, ValueError):
                cache = {}
        if use_cache and key in cache:
            best = int(cache[key]["variant"])
            self.prepare(best)
            return best, None
        L = _batch_sigs()
        best = _i32(-1)
        times = (ctypes.c_float * self.n_variants)()
        st = L.pdmp_batch_autotune(self._envs, self.n, int(reps), ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                                   ctypes.byref(best), times, ctypes.byref(self.plan), _stream())
        _check(st, "pdmp_batch_autotune")
        tl = [float(t) for t in times]
        cache[key] = {"variant": int(best.value), "times_ms": tl}
        try:
            os.makedirs(os.path.dirname(self.cache_path), exist_ok=True)
            tmp = self.cache_path + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1)
            os.replace(tmp, self.cache_path)
        except OSError:
            pass
        return int(best.value), tl

    def run(self):
        L = _batch_sigs()
        _check(L.pdmp_morph_batched(ctypes.byref(self.plan), ctypes.c_void_p(self.ws.data_ptr()), _stream()),
               "pdmp_morph_batched")
        return self.outputs

    def capture(self, stream: torch.cuda.Stream | None = None):
        """Captures run() into a CUDA graph on a side stream."""
        L = _batch_sigs()
        self.graph_stream = stream or torch.cuda.Stream()
        self.graph_stream.wait_stream(torch.cuda.current_stream())
        ex = ctypes.c_void_p()
        st = L.pdmp_batch_graph_create(ctypes.byref(self.plan), ctypes.c_void_p(self.ws.data_ptr()),
                                       ctypes.c_void_p(self.graph_stream.cuda_stream), ctypes.byref(ex))
        _check(st, "pdmp_batch_graph_create")
        self.graph = ex
        return ex

    def replay(self):
        L = _batch_sigs()
        _check(L.pdmp_graph_launch(self.graph, _stream()), "pdmp_graph_launch")
        return self.outputs

    def work(self) -> float:
        return float(self.plan.work)

    def __del__(self):
        try:
            if self.graph is not None and _lib is not None:
                _lib.pdmp_graph_destroy(self.graph)
        except Exception:
            pass


# ---------------------------------------------------------------------------
# learned surrogate (MLP over a 39-wide Fourier encoding -> 128 -> 128 -> 128 -> 3)
MLP_NW, MLP_NB, MLP_H, MLP_ENC = 38144, 387, 128, 39


class _Mlp(ctypes.Structure):
    _fields_ = [("W", ctypes.c_void_p), ("b", ctypes.c_void_p), ("W_bf16", ctypes.c_void_p),
                ("Wt_bf16", ctypes.c_void_p), ("adam", ctypes.c_void_p), ("lo", ctypes.c_float * 3),
                ("in_scale", ctypes.c_float * 3), ("out_scale", ctypes.c_float * 3)]


def _mlp_sigs():
    L = lib()
    if getattr(L, "_mlp_ready", False):
        return L
    MP = ctypes.POINTER(_Mlp)
    for name, argt in {
        "pdmp_mlp_refresh": [MP, _P],
        "pdmp_mlp_forward": [MP, _P, _i64, _P, _P],
        "pdmp_mlp_forward_fp32act": [MP, _P, _i64, _P, _P],
        "pdmp_mlp_gradient": [MP, _P, _P, _i32, _i32, _P, _P, _P, _P, _sz, _P],
        "pdmp_mlp_train_step": [MP, _P, _P, _i32, _f32, _f32, _f32, _f32, _i32, _P, _P, _sz, _P],
        "pdmp_surrogate_infer": [MP, _FP, _P, _i64, _i32, _f32, _f32, _P, ctypes.POINTER(_i64), _P, _sz, _P],
        "pdmp_surrogate_infer_culled": [MP, _FP, _P, _i64, _i32, _f32, _f32, _f32, _P, ctypes.POINTER(_i64), _P, _sz,
                                        _P],
        "pdmp_displacement_rms": [_P, _P, _i64, _i32, _P, _P],
        "pdmp_residual_threshold": [_FP, _P, _i64, _i32, _f32, _f32, ctypes.POINTER(_f32), _P, _P, _sz, _P],
    }.items():
        fn = getattr(L, name)
        fn.argtypes = argt
        fn.restype = _i32
    L.pdmp_mlp_train_workspace.argtypes = [_i32]
    L.pdmp_mlp_train_workspace.restype = _sz
    L.pdmp_surrogate_workspace.argtypes = [_FP, _i64]
    L.pdmp_surrogate_workspace.restype = _sz
    L.pdmp_residual_threshold_workspace.argtypes = [_FP, _i64]
    L.pdmp_residual_threshold_workspace.restype = _sz
    L._mlp_ready = True
    return L


def residual_threshold(field: DeviceField, x0: torch.Tensor, T: int, eta: float, q: float = 0.99,
                       out: torch.Tensor | None = None):
    """(tau_r, x_T): the q-quantile (nearest rank) of the plain morph's
    last-step length over the samples x0, and their x_T."""
    L = _mlp_sigs()
    N = x0.shape[0]
    if out is None:
        out = torch.empty_like(x0)
    f = field.struct()
    need = int(L.pdmp_residual_threshold_workspace(ctypes.byref(f), N))
    ws = torch.empty(max(need, 16), dtype=torch.uint8, device=x0.device)
    tau = _f32(0.0)
    _check(L.pdmp_residual_threshold(ctypes.byref(f), _ptr(x0, name="x0"), N, int(T), float(eta), float(q),
                                     ctypes.byref(tau), _ptr(out, shape=x0.shape, name="out"),
                                     ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream()), "pdmp_residual_threshold")
    return float(tau.value), out


def displacement_rms(x0: torch.Tensor, xT: torch.Tensor) -> torch.Tensor:
    L = _mlp_sigs()
    out = torch.empty(x0.shape[1], device=x0.device, dtype=torch.float32)
    _check(L.pdmp_displacement_rms(_ptr(x0), _ptr(xT, shape=x0.shape), x0.shape[0], x0.shape[1], _ptr(out), _stream()),
           "pdmp_displacement_rms")
    return out


class Surrogate:
    """The surrogate network: FP32 master weights, BF16 copies and Adam state
    on the GPU; normalisation from the workspace box [lo, hi] and the output
    scale (root mean square displacement of the training pairs)."""

    def __init__(self, lo, hi, out_scale, seed: int = 0, device="cuda"):
        import numpy as np
        g = np.random.Generator(np.random.Philox(key=np.array([seed, 0x5eed], dtype=np.uint64)))
        H = MLP_H
        shapes = [(H, MLP_ENC), (H, H), (H, H), (3, H)]
        Ws = [g.uniform(-1.0, 1.0, s) * np.sqrt(3.0 / s[1]) for s in shapes]   # unit-variance outputs
        Ws[-1] *= 0.1
        self.W = torch.tensor(np.concatenate([w.ravel() for w in Ws]), dtype=torch.float32, device=device)
        self.b = torch.zeros(MLP_NB, dtype=torch.float32, device=device)
        self.W_bf16 = torch.empty(MLP_NW, dtype=torch.int16, device=device)
        self.Wt_bf16 = torch.empty(2 * H * H, dtype=torch.int16, device=device)
        self.adam = torch.zeros(2 * MLP_NW + 2 * MLP_NB, dtype=torch.float32, device=device)
        lo = [float(v) for v in lo]
        hi = [float(v) for v in hi]
        self.lo = lo
        self.in_scale = [2.0 / (h - l) for l, h in zip(lo, hi)]
        self.out_scale = [float(v) for v in out_scale]
        self.step = 0
        self._ws = None
        self.refresh()

    def struct(self) -> _Mlp:
        m = _Mlp()
        m.W, m.b = self.W.data_ptr(), self.b.data_ptr()
        m.W_bf16, m.Wt_bf16, m.adam = self.W_bf16.data_ptr(), self.Wt_bf16.data_ptr(), self.adam.data_ptr()
        for i in range(3):
            m.lo[i], m.in_scale[i], m.out_scale[i] = self.lo[i], self.in_scale[i], self.out_scale[i]
        return m

    def refresh(self):
        m = self.struct()
        _check(_mlp_sigs().pdmp_mlp_refresh(ctypes.byref(m), _stream()), "pdmp_mlp_refresh")

    def weights(self):
        """FP32 master weights and biases as numpy arrays, per layer."""
        H = MLP_H
        W = self.W.cpu().numpy()
        b = self.b.cpu().numpy()
        sizes = [(H, MLP_ENC), (H, H), (H, H), (3, H)]
        out_w, out_b, o = [], [], 0
        for s in sizes:
            out_w.append(W[o:o + s[0] * s[1]].reshape(s))
            o += s[0] * s[1]
        out_b = [b[0:H], b[H:2 * H], b[2 * H:3 * H], b[3 * H:3 * H + 3]]
        return out_w, out_b

    def save(self, path: str) -> None:
        """Writes the network: a one-line JSON header (format, sizes, the
        normalisation, the Adam step), then the FP32 master weights, biases and
        Adam moments as raw little-endian float32."""
        import json
        import numpy as np
        head = {"format": "pdmp-surrogate-1", "nw": MLP_NW, "nb": MLP_NB, "enc": MLP_ENC, "hidden": MLP_H,
                "lo": self.lo, "in_scale": self.in_scale, "out_scale": self.out_scale, "step": self.step}
        with open(path, "wb") as f:
            f.write((json.dumps(head) + "\n").encode())
            for t in (self.W, self.b, self.adam):
                f.write(t.detach().cpu().numpy().astype("<f4").tobytes())

    @classmethod
    def load(cls, path: str, device="cuda") -> "Surrogate":
        """Reads what save() wrote and rebuilds the BF16 copies."""
        import json
        import numpy as np
        with open(path, "rb") as f:
            head = json.loads(f.readline().decode())
            raw = np.frombuffer(f.read(), dtype="<f4")
        if head.get("format") != "pdmp-surrogate-1" or head["nw"] != MLP_NW or head["nb"] != MLP_NB:
            raise ValueError(f"{path}: not a surrogate file of this library version ({head.get('format')})")
        nw, nb = MLP_NW, MLP_NB
        if raw.size != nw + nb + 2 * nw + 2 * nb:
            raise ValueError(f"{path}: {raw.size} floats, expected {3 * (nw + nb)}")
        net = cls.__new__(cls)
        t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=device)
        net.W, net.b, net.adam = t(raw[:nw]), t(raw[nw:nw + nb]), t(raw[nw + nb:])
        net.W_bf16 = torch.empty(MLP_NW, dtype=torch.int16, device=device)
        net.Wt_bf16 = torch.empty(2 * MLP_H * MLP_H, dtype=torch.int16, device=device)
        net.lo, net.in_scale, net.out_scale = head["lo"], head["in_scale"], head["out_scale"]
        net.step = int(head["step"])
        net._ws = None
        net.refresh()
        return net

    def bf16_weights(self):
        """The BF16 weights the kernels use, upcast to float64 numpy arrays."""
        import numpy as np
        H = MLP_H
        bits = self.W_bf16.cpu().numpy().astype(np.uint16).astype(np.uint32) << 16
        W = bits.view(np.float32).astype(np.float64)
        sizes = [(H, MLP_ENC), (H, H), (H, H), (3, H)]
        out, o = [], 0
        for s in sizes:
            out.append(W[o:o + s[0] * s[1]].reshape(s))
            o += s[0] * s[1]
        return out

    def forward(self, x0: torch.Tensor, out: torch.Tensor | None = None, fp32_act: bool = False) -> torch.Tensor:
        """The predicted x_T; fp32_act selects the FP32-activation mode (diagnostic)."""
        if out is None:
            out = torch.empty_like(x0)
        m = self.struct()
        name = "pdmp_mlp_forward_fp32act" if fp32_act else "pdmp_mlp_forward"
        _check(getattr(_mlp_sigs(), name)(ctypes.byref(m), _ptr(x0, name="x0"), x0.shape[0],
                                          _ptr(out, shape=x0.shape, name="out"), _stream()), name)
        return out

    def gradient(self, x0: torch.Tensor, xT: torch.Tensor, fp32_act: bool = False):
        """(loss, gW, gb) of one batch without an update (diagnostic): the
        gradient with respect to the BF16 weights, in the layouts of W and b."""
        L = _mlp_sigs()
        B = x0.shape[0]
        need = int(L.pdmp_mlp_train_workspace(B))
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=x0.device)
        loss = torch.zeros(1, device=x0.device)
        gW = torch.empty(MLP_NW, device=x0.device)
        gb = torch.empty(MLP_NB, device=x0.device)
        m = self.struct()
        _check(L.pdmp_mlp_gradient(ctypes.byref(m), _ptr(x0, name="x0"), _ptr(xT, shape=x0.shape, name="xT"), B,
                                   int(bool(fp32_act)), _ptr(loss), _ptr(gW), _ptr(gb),
                                   ctypes.c_void_p(self._ws.data_ptr()), self._ws.numel(), _stream()),
               "pdmp_mlp_gradient")
        return loss, gW, gb

    def train_step(self, x0: torch.Tensor, xT: torch.Tensor, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                   loss: torch.Tensor | None = None):
        L = _mlp_sigs()
        B = x0.shape[0]
        need = int(L.pdmp_mlp_train_workspace(B))
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=x0.device)
        self.step += 1
        m = self.struct()
        _check(L.pdmp_mlp_train_step(ctypes.byref(m), _ptr(x0, name="x0"), _ptr(xT, shape=x0.shape, name="xT"), B,
                                     float(lr), float(beta1), float(beta2), float(eps), self.step,
                                     _ptr(loss, name="loss"), ctypes.c_void_p(self._ws.data_ptr()), self._ws.numel(),
                                     _stream()), "pdmp_mlp_train_step")
        return loss

    def infer(self, field: DeviceField, x0: torch.Tensor, T: int, eta: float, tau_r: float,
              out: torch.Tensor | None = None, ws: torch.Tensor | None = None, r_cut: float | None = None):
        """(x_T, number of samples that fell back to the plain morph).  r_cut:
        run the residual check on the culled kernel with that cut-off radius
        (pdmp_surrogate_infer_culled; from cull_radius(field, eps))."""
        L = _mlp_sigs()
        N = x0.shape[0]
        if out is None:
            out = torch.empty_like(x0)
        f = field.struct()
        need = int(L.pdmp_surrogate_workspace(ctypes.byref(f), N))
        if ws is None or ws.numel() < need:
            ws = torch.empty(max(need, 16), dtype=torch.uint8, device=x0.device)
        nf = _i64(0)
        m = self.struct()
        if r_cut is None:
            _check(L.pdmp_surrogate_infer(ctypes.byref(m), ctypes.byref(f), _ptr(x0, name="x0"), N, int(T),
                                          float(eta), float(tau_r), _ptr(out, shape=x0.shape, name="out"),
                                          ctypes.byref(nf), ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream()),
                   "pdmp_surrogate_infer")
        else:
            _check(L.pdmp_surrogate_infer_culled(ctypes.byref(m), ctypes.byref(f), _ptr(x0, name="x0"), N, int(T),
                                                 float(eta), float(tau_r), float(r_cut),
                                                 _ptr(out, shape=x0.shape, name="out"), ctypes.byref(nf),
                                                 ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream()),
                   "pdmp_surrogate_infer_culled")
        return out, int(nf.value)


# ---------------------------------------------------------------------------
# autograd through the Euler chain
class _MorphFn(torch.autograd.Function):
    """x_T = morph(x_0; w, bias): forward by pdmp_morph with checkpoints every
    k steps, backward by pdmp_morph_vjp from them (and d/dw, d/dbias when the
    weights require gradients).  No PyTorch arithmetic on the path."""

    @staticmethod
    def forward(ctx, x0, w, bias, field, T, eta, k):
        fld = field.with_weights(w.detach(), bias=float(bias.detach()) if bias is not None else field.bias)
        ck = torch.empty(T // k, x0.shape[0], field.d, device=x0.device, dtype=torch.float32) if T else None
        xT = morph(fld, x0.detach().contiguous(), T, eta, ckpt=ck, k=k if T else 0)
        ctx.fld, ctx.T, ctx.eta, ctx.k = fld, T, eta, k
        ctx.save_for_backward(x0.detach(), ck if ck is not None else torch.empty(0, device=x0.device))
        return xT

    @staticmethod
    def backward(ctx, gT):
        x0, ck = ctx.saved_tensors
        want_w = ctx.needs_input_grad[1] or ctx.needs_input_grad[2]
        if ctx.T == 0:
            gw = torch.zeros(ctx.fld.M, device=x0.device) if ctx.needs_input_grad[1] else None
            gb = torch.zeros((), device=x0.device) if ctx.needs_input_grad[2] else None
            return gT, gw, gb, None, None, None, None
        res = morph_vjp(ctx.fld, x0, ctx.T, ctx.eta, ctx.k, gT.contiguous(), ckpt=ck, want_param_grad=want_w)
        if want_w:
            g0, gw, gb = res
            return (g0, gw if ctx.needs_input_grad[1] else None, gb.reshape(()) if ctx.needs_input_grad[2] else None,
                    None, None, None, None)
        return res, None, None, None, None, None, None


def morph_autograd(field: DeviceField, x0: torch.Tensor, T: int, eta: float, k: int = 1,
                   w: torch.Tensor | None = None, bias: torch.Tensor | None = None) -> torch.Tensor:
    """Differentiable morph: gradients flow to x0 and, when given as tensors
    that require grad, to the weights w (M) and the bias (a 0-d tensor)."""
    if T % max(k, 1) != 0:
        raise ValueError("k must divide T")
    w = field.w if w is None else w
    if bias is None:
        bias = torch.tensor(field.bias, device=x0.device, dtype=torch.float32)
    return _MorphFn.apply(x0, w, bias, field, int(T), float(eta), int(k))
