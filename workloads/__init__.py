"""Seeded synthetic inputs shaped like the PDMP workloads.

This module only draws numbers and lays them out; it holds none of the
method's arithmetic (no features, costs, gradients, steps or fits).  Both the
FP64 oracle (``oracle``) and the CUDA library (``paper_2108_11775_gb300``)
consume what it produces, and it imports neither.

Every draw comes from NumPy's Philox4x32-10 counter-based generator keyed by
(seed, stream id), one stream per tensor, so each tensor is reproducible on
its own and identical on x86 and Arm hosts.

The paper's own workloads (7-DOF arm scenes, occupancy from depth sensors,
Sec. 4) are not available; these stand in for them:

* ``config1``  plain morph, 2-D [0,10]^2: 32 x 32 RBF centres on an
  edge-inclusive grid, gamma = 4, w ~ N(0,1), N = 4096, T = 10.
* ``config2``  plain morph at scale, 2-D: 16,384 centres U[0,10]^2, gamma = 8,
  64 random axis-aligned boxes, 200k labelled points for the fit,
  N = 2^20 samples, T = 50.
* ``config3``  differentiation, 7-D [-pi,pi]^7: 4096 random Fourier features
  Omega ~ N(0, 2I), b ~ U[0, 2 pi), w ~ N(0, 1/M); N = 2^20, T = 20, k = 5.
* ``config4``  256 environments, d in {2,3}, M ~ U[256, 8192],
  N ~ U[1024, 65536], gamma = 4, w ~ N(0,1), T = 30.
* ``config5``  3-D [0,5]^3: 8192 centres, gamma = 8, 48 boxes, T = 40,
  2^20 training pairs, inference on N = 2^24.
"""
from __future__ import annotations

import os
from dataclasses import dataclass, field as dc_field

import numpy as np

RBF = 0
RFF = 1

# stream ids: one per tensor kind
S_CENTRES, S_WEIGHTS, S_SAMPLES, S_PHASE, S_BOXES, S_POINTS, S_COTANGENT, S_ENV, S_EXTRA = range(1, 10)


def rng(seed: int, stream: int) -> np.random.Generator:
    """Philox4x32-10 keyed by (seed, stream)."""
    key = np.array([int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key))


@dataclass
class Field:
    """An occupancy field: kind, centres (RBF mu / RFF omega, M x d float32),
    weights w (M float32), RBF width gamma, RFF phases (M float32), bias."""
    kind: int
    centres: np.ndarray
    w: np.ndarray
    gamma: float = 0.0
    phase: np.ndarray | None = None
    bias: float = 0.0

    @property
    def d(self) -> int:
        return int(self.centres.shape[1])

    @property
    def M(self) -> int:
        return int(self.centres.shape[0])

    def with_weights(self, w, bias: float = 0.0) -> "Field":
        return Field(self.kind, self.centres, np.ascontiguousarray(np.asarray(w, dtype=np.float32)),
                     self.gamma, self.phase, float(np.float32(bias)))


@dataclass
class Workload:
    name: str
    field: Field
    x0: np.ndarray                 # N x d float32 base samples
    T: int
    lo: np.ndarray                 # workspace box
    hi: np.ndarray
    boxes: np.ndarray | None = None      # nb x 2d float32 obstacles
    fit_X: np.ndarray | None = None      # n x d float32 labelled points
    fit_y: np.ndarray | None = None      # n uint8 labels
    extra: dict = dc_field(default_factory=dict)


def f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def uniform_box(seed: int, stream: int, n: int, lo, hi) -> np.ndarray:
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    u = rng(seed, stream).random((n, lo.size))
    return f32(lo + (hi - lo) * u)


def random_boxes(seed: int, nb: int, lo, hi, side_lo: float, side_hi: float) -> np.ndarray:
    """nb axis-aligned boxes: centre U(box), side U[side_lo, side_hi] per axis.
    Row layout: lo_0..lo_{d-1}, hi_0..hi_{d-1} (float32)."""
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    g = rng(seed, S_BOXES)
    d = lo.size
    c = lo + (hi - lo) * g.random((nb, d))
    side = side_lo + (side_hi - side_lo) * g.random((nb, d))
    return f32(np.concatenate([c - side / 2, c + side / 2], axis=1))


def inside_boxes(boxes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Dataset labels y in {0,1}: 1 where a float32 point lies in a closed box.
    (Labelling the synthetic dataset D is input generation; the library's and
    the oracle's label kernels are separate implementations.)"""
    x = f32(x)
    d = x.shape[1]
    y = np.zeros(x.shape[0], dtype=bool)
    for b in boxes:
        y |= np.all((b[:d] <= x) & (x <= b[d:]), axis=1)
    return y.astype(np.uint8)


def config1(seed: int = 1, N: int = 4096) -> Workload:
    g = np.linspace(0.0, 10.0, 32)
    gx, gy = np.meshgrid(g, g, indexing="ij")
    centres = f32(np.stack([gx.ravel(), gy.ravel()], axis=1))
    w = f32(rng(seed, S_WEIGHTS).standard_normal(centres.shape[0]))
    fld = Field(RBF, centres, w, gamma=4.0)
    x0 = uniform_box(seed, S_SAMPLES, N, [0, 0], [10, 10])
    return Workload("rbf2d-grid-M1024-N4096-T10", fld, x0, 10, np.zeros(2), np.full(2, 10.0))


def config2(seed: int = 2, N: int = 1 << 20, M: int = 16384, n_fit: int = 200_000, nb: int = 64) -> Workload:
    lo, hi = np.zeros(2), np.full(2, 10.0)
    centres = uniform_box(seed, S_CENTRES, M, lo, hi)
    boxes = random_boxes(seed, nb, lo, hi, 0.3, 1.5)
    X = uniform_box(seed, S_POINTS, n_fit, lo, hi)
    y = inside_boxes(boxes, X)
    # placeholder weights until the occupancy fit replaces them
    fld = Field(RBF, centres, np.zeros(M, np.float32), gamma=8.0)
    x0 = uniform_box(seed, S_SAMPLES, N, lo, hi)
    return Workload(f"rbf2d-fitted-M{M}-N{N}-T50", fld, x0, 50, lo, hi, boxes, X, y)


GOLDEN_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")
FITTED_RBF2D = "fit_rbf2d_fitted.txt"


def read_fixture(path: str):
    """(params, arrays) of a text fixture: '#' header lines, '@ name value'
    numbers and '= name shape...' arrays followed by rows of numbers."""
    params, arrays, cur = {}, {}, None
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            if line.startswith("@ "):
                _, k, v = line.rstrip("\n").split(" ", 2)
                params[k] = int(v) if v.lstrip("-").isdigit() else float(v)
            elif line.startswith("= "):
                parts = line.split()
                cur = [parts[1], tuple(int(x) for x in parts[2:]), []]
                arrays[cur[0]] = cur
            else:
                cur[2].extend(float(v) for v in line.split())
    return params, {k: np.array(v[2], dtype=np.float64).reshape(v[1]) for k, v in arrays.items()}


def config2_fitted(seed: int = 2, N: int = 1 << 20):
    """config2 with the occupancy weights and bias stored in
    tests/golden/fit_rbf2d_fitted.txt (the oracle's fit of this workload,
    rounded to float32), and that file's parameters (its certified bound L
    among them).  Raises if the fixture is missing."""
    if seed != 2:
        raise ValueError("the stored fit is of the seed-2 workload")
    params, arrays = read_fixture(os.path.join(GOLDEN_DIR, FITTED_RBF2D))
    wk = config2(seed=seed, N=N)
    if int(params["M"]) != wk.field.M:
        raise ValueError("the stored fit has another number of centres")
    wk.field = wk.field.with_weights(f32(arrays["w"].ravel()), bias=params["bias"])
    return wk, params


def proxy_fitted_weights(seed: int, centres: np.ndarray, boxes: np.ndarray, scale: float = 0.5) -> np.ndarray:
    """Weights shaped like a fitted occupancy map (positive on centres inside
    an obstacle, negative outside, with spread) for parity runs that must not
    take their weights from the GPU fit."""
    occ = inside_boxes(boxes, centres).astype(np.float64)
    noise = rng(seed, S_EXTRA).standard_normal(centres.shape[0])
    return f32(scale * (2.0 * occ - 1.0) * (0.5 + 0.5 * np.abs(noise)))


def config3(seed: int = 3, N: int = 1 << 20, M: int = 4096, d: int = 7) -> Workload:
    omega = f32(np.sqrt(2.0) * rng(seed, S_CENTRES).standard_normal((M, d)))
    phase = f32(2.0 * np.pi * rng(seed, S_PHASE).random(M))
    w = f32(rng(seed, S_WEIGHTS).standard_normal(M) / np.sqrt(M))
    fld = Field(RFF, omega, w, phase=phase)
    lo, hi = np.full(d, -np.pi), np.full(d, np.pi)
    x0 = uniform_box(seed, S_SAMPLES, N, lo, hi)
    gT = f32(rng(seed, S_COTANGENT).standard_normal((N, d)))
    return Workload(f"rff7d-M{M}-N{N}-T20", fld, x0, 20, lo, hi, extra={"gT": gT, "k": 5})


def config4(seed: int = 4, n_envs: int = 256, T: int = 30, M_range=(256, 8192), N_range=(1024, 65536)) -> list:
    ge = rng(seed, S_ENV)
    envs = []
    for e in range(n_envs):
        d = int(ge.integers(2, 4))
        M = int(ge.integers(M_range[0], M_range[1] + 1))
        N = int(ge.integers(N_range[0], N_range[1] + 1))
        s = seed * 100_003 + e
        lo, hi = np.zeros(d), np.full(d, 10.0)
        centres = uniform_box(s, S_CENTRES, M, lo, hi)
        w = f32(rng(s, S_WEIGHTS).standard_normal(M))
        x0 = uniform_box(s, S_SAMPLES, N, lo, hi)
        envs.append(Workload(f"env{e}", Field(RBF, centres, w, gamma=4.0), x0, T, lo, hi))
    return envs


def config5(seed: int = 5, N: int = 1 << 24, M: int = 8192, n_fit: int = 200_000, nb: int = 48,
            n_train: int = 1 << 20) -> Workload:
    lo, hi = np.zeros(3), np.full(3, 5.0)
    centres = uniform_box(seed, S_CENTRES, M, lo, hi)
    boxes = random_boxes(seed, nb, lo, hi, 0.15, 0.75)
    X = uniform_box(seed, S_POINTS, n_fit, lo, hi)
    y = inside_boxes(boxes, X)
    fld = Field(RBF, centres, np.zeros(M, np.float32), gamma=8.0)
    x0 = uniform_box(seed, S_SAMPLES, N, lo, hi)
    xtrain = uniform_box(seed, S_EXTRA, n_train, lo, hi)
    return Workload(f"rbf3d-surrogate-M{M}-N{N}-T40", fld, x0, 40, lo, hi, boxes, X, y,
                    extra={"x_train": xtrain})


def random_field(seed: int, kind: int, d: int, M: int, lo=0.0, hi=10.0, gamma: float = 4.0,
                 wscale: float = 1.0, bias: float = 0.0) -> Field:
    """Small fields for tests."""
    if kind == RBF:
        centres = uniform_box(seed, S_CENTRES, M, np.full(d, lo), np.full(d, hi))
        w = f32(wscale * rng(seed, S_WEIGHTS).standard_normal(M))
        return Field(RBF, centres, w, gamma=float(np.float32(gamma)), bias=float(np.float32(bias)))
    omega = f32(np.sqrt(2.0) * rng(seed, S_CENTRES).standard_normal((M, d)))
    phase = f32(2.0 * np.pi * rng(seed, S_PHASE).random(M))
    w = f32(wscale * rng(seed, S_WEIGHTS).standard_normal(M) / np.sqrt(M))
    return Field(RFF, omega, w, phase=phase, bias=float(np.float32(bias)))


class TanhNet:
    """Weights of a tanh occupancy network (d -> H -> H -> 1), float32."""

    def __init__(self, W1, b1, W2, b2, w3, b3):
        self.W1, self.b1, self.W2, self.b2, self.w3 = (f32(a) for a in (W1, b1, W2, b2, w3))
        self.b3 = float(np.float32(b3))
        self.H, self.d = self.W1.shape


def tanh_net(seed: int, d: int, H: int, lo=0.0, hi=10.0, gain: float = 1.0, out_scale: float = 2.0,
             b3: float = -1.0) -> TanhNet:
    """Random-initialised network whose first layer maps the box [lo, hi]^d to
    about [-gain, gain] per unit (so the field varies across the box):
    W1 ~ N(0, (2 gain / (hi - lo))^2 / d), b1 centres the box, W2 ~ N(0, 1/H),
    w3 ~ N(0, out_scale^2 / H)."""
    g = rng(seed, S_WEIGHTS)
    span = float(hi) - float(lo)
    W1 = g.standard_normal((H, d)) * (2.0 * gain / span) / np.sqrt(d)
    b1 = -W1 @ np.full(d, 0.5 * (float(lo) + float(hi))) + 0.1 * g.standard_normal(H)
    W2 = g.standard_normal((H, H)) / np.sqrt(H)
    b2 = 0.1 * g.standard_normal(H)
    w3 = g.standard_normal(H) * out_scale / np.sqrt(H)
    return TanhNet(W1, b1, W2, b2, w3, b3)


class Chain:
    """A planar serial chain: n revolute joints at base, link lengths, p body points per link."""

    def __init__(self, lengths, base=(0.0, 0.0), p: int = 4):
        self.lengths = f32(np.asarray(lengths))
        self.base = f32(np.asarray(base))
        self.n = int(self.lengths.shape[0])
        self.p = int(p)


def planar_arm(n: int = 7, reach: float = 4.5, base=(5.0, 5.0), p: int = 4) -> Chain:
    """An n-link planar arm of total reach `reach` (equal links) based at `base`
    (the centre of the 2-D workspace [0, 10]^2), p body points per link."""
    return Chain(np.full(n, reach / n), base, p)


def joint_box(n: int):
    """The joint limits [-pi, pi]^n."""
    return np.full(n, -np.pi), np.full(n, np.pi)
