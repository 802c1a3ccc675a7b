"""Writes the golden fixtures of this directory from the FP64 oracle.

The paper prints no worked example, so the stored values are the oracle's:
seeded inputs from ``workloads`` and the oracle's outputs for them, written
with 17 significant digits.  Each fixture's header names the passage of the
paper the computation follows.  Run from the repository root:

    python tests/golden/make_golden.py
    python tests/golden/make_golden.py --fit-rbf2d   # the fitted 2-D field (about 1.5 h on 8 cores)
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as wl  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def write(name, header, params, arrays, fmt="%.17g"):
    with open(os.path.join(HERE, name), "w") as f:
        for line in header:
            f.write(f"# {line}\n")
        for k, v in params.items():
            f.write(f"@ {k} {v!r}\n")
        for k, a in arrays.items():
            a = np.asarray(a, dtype=np.float64)
            f.write(f"= {k} {' '.join(str(s) for s in a.shape)}\n")
            for row in a.reshape(a.shape[0], -1):
                f.write(" ".join(fmt % v for v in row) + "\n")


def fit_rbf2d(threads=None):
    """The occupancy of the 2-D fitted workload (16,384 RBF centres U[0,10]^2,
    gamma = 8, 200k points labelled by 64 boxes; workloads.config2, seed 2)
    fitted by the oracle alone with the same settings the GPU fit uses
    (lambda = 1e-4, 20 power iterations, 200 Nesterov iterations).  Its w
    (rounded to float32, the precision both sides consume) and bias are the
    field whose morph is benchmarked and parity-tested."""
    if threads:
        oracle.set_threads(threads)
    wk = wl.config2(N=16)
    l2, power_iters, iters = 1e-4, 20, 200
    w, b, loss, alpha = oracle.fit(wk.field, wk.fit_X, wk.fit_y, l2, power_iters, iters)
    w32, b32 = wl.f32(w), float(np.float32(b))
    f32 = wk.field.with_weights(w32, bias=b32)
    loss32, g, gb = oracle.fit_objective(f32, wk.fit_X, wk.fit_y, l2, w32, b32)
    L, G = oracle.lipschitz(f32, wk.lo - 0.5, wk.hi + 0.5, cells=128)
    write("fit_rbf2d_fitted.txt",
          ["Sec. 3.1: the occupancy fitted to labelled points by binary cross entropy and gradient descent,",
           "read as mean BCE + (l2/2)|w|^2 minimised from zero by Nesterov iterations with the step",
           "1 / (lambda_hat / 4 + l2), lambda_hat from power iterations (the same algorithm as pdmp_fit_occupancy).",
           "Field: workloads.config2 (seed 2): 16,384 RBF centres U[0,10]^2, gamma = 8, 200,000 points U[0,10]^2",
           "labelled by 64 boxes.  w is the oracle's FP64 solution rounded to float32 (what both sides consume);",
           "loss_f64 is the oracle's objective at the FP64 solution, loss_f32w at the rounded (w, bias);",
           "L is the oracle's certified Lipschitz bound of grad c over [-0.5, 10.5]^2 (128 cells) for the rounded field.",
           "Written by tests/golden/make_golden.py --fit-rbf2d from the FP64 oracle alone."],
          {"l2": l2, "power_iters": power_iters, "iters": iters, "n_fit": int(wk.fit_X.shape[0]),
           "M": int(wk.field.M), "bias": b32, "loss_f64": loss, "loss_f32w": loss32, "alpha": alpha,
           "kkt_norm": float(np.sqrt(np.sum(np.asarray(g, np.float64) ** 2) + gb * gb)), "L": L, "G": G},
          {"w": w32.reshape(-1, 8)}, fmt="%.9g")


def main():
    # Eq. (1) by Euler's method (Sec. 3.2), RBF occupancy on the 32 x 32 grid field
    w1 = wl.config1()
    L, _ = oracle.lipschitz(w1.field, w1.lo, w1.hi, cells=64)
    eta = float(np.float32(0.5 / L))
    x0 = w1.x0[:16]
    write("morph_rbf2d_grid.txt",
          ["Eq. (1), Euler's method (Sec. 3.2): x_{t+1} = x_t - eta grad c(x_t), c = sigmoid(w . phi(x)),",
           "RBF features on a 32 x 32 grid of [0,10]^2 (workloads.config1, seed 1), gamma = 4.",
           "Written by tests/golden/make_golden.py from the FP64 oracle; eta = 0.5 / L, L the oracle's certified bound."],
          {"T": 10, "eta": eta}, {"x0": x0, "xT": oracle.morph(w1.field, x0, 10, eta)})
    # the same with random Fourier features in 7-D, plus the VJP and the log-det (Sec. 3.2)
    w3 = wl.config3(N=8, M=256)
    f = w3.field
    eta3 = float(np.float32(0.5 / (2.0 * 50.0)))
    T3 = 6
    g = np.asarray(w3.extra["gT"], dtype=np.float64)
    ld, xT3, _ = oracle.logdet(f, w3.x0, T3, eta3)
    write("morph_rff7d.txt",
          ["Eq. (1) by Euler's method with random Fourier features phi_m = cos(omega_m . x + b_m) in 7-D",
           "(workloads.config3 with N = 8, M = 256, seed 3); g0 = (dx_T/dx_0)^T g_T (chain rule through Eq. (1));",
           "logdet = sum_t log det(I - eta Hess c(x_t)) (Sec. 3.2, 'Drawing Samples').",
           "Written by tests/golden/make_golden.py from the FP64 oracle."],
          {"T": T3, "eta": eta3},
          {"x0": w3.x0, "xT": xT3, "gT": g, "g0": oracle.morph_vjp(f, w3.x0, T3, eta3, g), "logdet": ld[:, None]})
    # Eq. (2): the inverse recovers the inputs
    z = oracle.morph(w1.field, x0, 10, eta)
    y, _ = oracle.morph_inverse(w1.field, z, 10, eta)
    write("inverse_rbf2d_grid.txt",
          ["Eq. (2): each Euler step undone, last first, by the fixed point y = z + eta grad c(y);",
           "the 32 x 32 grid field of morph_rbf2d_grid.txt.  Written by tests/golden/make_golden.py from the FP64 oracle."],
          {"T": 10, "eta": eta}, {"z": z, "y": y})
    print("written")


if __name__ == "__main__":
    if "--fit-rbf2d" in sys.argv:
        fit_rbf2d(threads=int(sys.argv[sys.argv.index("--threads") + 1]) if "--threads" in sys.argv else None)
        print("written")
    else:
        main()
