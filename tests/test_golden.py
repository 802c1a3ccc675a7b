"""Golden fixtures (tests/golden/, written by make_golden.py from the FP64
oracle; the paper prints no worked example): the oracle still reproduces
them, and the CUDA path matches them."""
import os

import numpy as np
import pytest
import torch

import oracle
import workloads as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    params, arrays, cur, rows, shape = {}, {}, None, [], None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.rstrip("\n")
            if line.startswith("#") or not line:
                continue
            if line.startswith("@ "):
                _, k, v = line.split(" ", 2)
                params[k] = eval(v, {"__builtins__": {}})          # a repr of a number
            elif line.startswith("= "):
                if cur is not None:
                    arrays[cur] = np.array(rows, dtype=np.float64).reshape(shape)
                parts = line.split()
                cur, shape, rows = parts[1], tuple(int(s) for s in parts[2:]), []
            else:
                rows.append([float(v) for v in line.split()])
    if cur is not None:
        arrays[cur] = np.array(rows, dtype=np.float64).reshape(shape)
    return params, arrays


def test_oracle_reproduces_the_fixtures():
    p, a = load("morph_rbf2d_grid.txt")
    w1 = wl.config1()
    assert np.array_equal(a["x0"], w1.x0[:16].astype(np.float64))
    assert np.abs(oracle.morph(w1.field, a["x0"], p["T"], p["eta"]) - a["xT"]).max() <= 1e-12
    p3, a3 = load("morph_rff7d.txt")
    w3 = wl.config3(N=8, M=256)
    ld, xT, mindet = oracle.logdet(w3.field, a3["x0"], p3["T"], p3["eta"])
    assert np.all(mindet > 0)
    assert np.abs(xT - a3["xT"]).max() <= 1e-12
    assert np.abs(ld - a3["logdet"][:, 0]).max() <= 1e-12
    g0 = oracle.morph_vjp(w3.field, a3["x0"], p3["T"], p3["eta"], a3["gT"])
    assert np.abs(g0 - a3["g0"]).max() <= 1e-12 * np.abs(a3["g0"]).max()
    pi, ai = load("inverse_rbf2d_grid.txt")
    assert np.abs(ai["y"] - a["x0"]).max() <= 1e-10                 # Eq. (2) recovers the inputs
    y, _ = oracle.morph_inverse(w1.field, ai["z"], pi["T"], pi["eta"])
    assert np.abs(y - ai["y"]).max() <= 1e-12


@pytest.mark.gpu
def test_cuda_path_matches_the_fixtures():
    import paper_2108_11775_gb300 as pdmp
    assert torch.cuda.is_available()
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    p, a = load("morph_rbf2d_grid.txt")
    fld = pdmp.DeviceField.from_host(wl.config1().field)
    for fast in (True, False):
        xT = pdmp.morph(fld, dev(a["x0"]), p["T"], p["eta"], fast=fast).cpu().numpy()
        assert np.abs(xT - a["xT"]).max() <= 1e-4
    pi, ai = load("inverse_rbf2d_grid.txt")
    y = pdmp.morph_inverse(fld, dev(ai["z"]), pi["T"], pi["eta"]).cpu().numpy()
    assert np.abs(y - ai["y"]).max() <= 1e-4
    p3, a3 = load("morph_rff7d.txt")
    f3 = pdmp.DeviceField.from_host(wl.config3(N=8, M=256).field)
    T, eta = p3["T"], p3["eta"]
    assert np.abs(pdmp.morph(f3, dev(a3["x0"]), T, eta).cpu().numpy() - a3["xT"]).max() <= 1e-4
    ld = pdmp.logdet(f3, dev(a3["x0"]), T, eta).cpu().numpy()
    assert np.abs(ld - a3["logdet"][:, 0]).max() <= 1e-4 * T
    g0 = pdmp.morph_vjp(f3, dev(a3["x0"]), T, eta, T, dev(a3["gT"])).cpu().numpy()
    assert np.abs(g0 - a3["g0"]).max() <= 1e-4 * np.abs(a3["g0"]).max()
    assert pdmp.stream_status()[0] == 0
