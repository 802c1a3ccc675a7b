"""Shared helpers for the GPU parity tests (inputs and step sizes from the
oracle and the seeded generators only -- never from the CUDA path)."""
import os

import numpy as np

import oracle
import workloads as wl


def setup_oracle_threads():
    oracle.set_threads(os.cpu_count() or 1)


def rbf_eta(field, lo, hi, cells=64, factor=0.5):
    """eta = factor / L with L the oracle's certified bound over [lo, hi]."""
    L, _ = oracle.lipschitz(field, lo, hi, cells=cells)
    return float(np.float32(factor / L)), L


def rff_eta_certified(field, factor=0.5):
    L, _ = oracle.lipschitz(field)
    return float(np.float32(factor / L)), L


def rff_eta_sampled(field, lo, hi, n=2000, safety=2.0, factor=0.5, seed=99):
    """eta from a sampled estimate of sup |Hess c| (safety factor 2); used for
    small parity cases where the certified RFF bound would make the chain
    nearly the identity.  Every such case also checks det > 0 at every step."""
    pts = wl.uniform_box(seed, 7, n, lo, hi)
    h = oracle.evaluate(field, pts, hess=True)["hess"]
    est = safety * np.abs(np.linalg.eigvalsh(h)).max()
    return float(np.float32(factor / est)), est


def max_abs(a, b):
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).max()) if np.size(a) else 0.0


def per_step_check(field, traj, steps, eta):
    """Every step's FP32 increment against the oracle's at the same state:
    |step_gpu - step_ref|_inf <= 1e-5 eta sigma'(s) sum_m |w_m| |grad phi_m|
    + 1e-5 |step_ref|_inf per sample, the oracle evaluated at the GPU's own
    state x_t promoted to FP64.  Returns the worst error over its tolerance."""
    T, N, d = steps.shape
    worst = 0.0
    for t in range(T):
        xt = traj[t].astype(np.float64)
        ev = oracle.evaluate(field, xt)
        ref = -eta * ev["grad"]
        tol = 1e-5 * eta * ev["scale"] + 1e-5 * np.abs(ref).max(axis=1)
        err = np.abs(steps[t].astype(np.float64) - ref).max(axis=1)
        assert np.all(err <= tol), f"step {t}: worst excess {np.max(err - tol):.3e}"
        worst = max(worst, float(np.max(err / np.maximum(tol, 1e-300))))
    return worst
