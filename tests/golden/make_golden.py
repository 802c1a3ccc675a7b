"""Writes the golden fixtures of this directory from the FP64 oracle.

The paper prints no worked example, so the stored values are the oracle's:
seeded inputs from ``workloads`` and the oracle's outputs for them, written
with 17 significant digits.  Each fixture's header names the passage of the
paper the computation follows.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as wl  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def write(name, header, params, arrays):
    with open(os.path.join(HERE, name), "w") as f:
        for line in header:
            f.write(f"# {line}\n")
        for k, v in params.items():
            f.write(f"@ {k} {v!r}\n")
        for k, a in arrays.items():
            a = np.asarray(a, dtype=np.float64)
            f.write(f"= {k} {' '.join(str(s) for s in a.shape)}\n")
            for row in a.reshape(a.shape[0], -1):
                f.write(" ".join(f"{v:.17g}" for v in row) + "\n")


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
    main()
