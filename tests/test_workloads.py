"""The seeded synthetic inputs match the recipes stated for them (shapes,
ranges, widths, step counts, distribution moments) and are reproducible:
the same seed gives the same bytes."""
import numpy as np

import workloads as wl


def test_grid_workload():
    w = wl.config1(N=4096)
    c = w.field.centres
    assert c.shape == (1024, 2) and w.field.gamma == 4.0 and w.T == 10
    assert np.array_equal(np.unique(c[:, 0]), np.linspace(0, 10, 32).astype(np.float32))   # edge-inclusive grid
    assert w.x0.shape == (4096, 2) and w.x0.min() >= 0.0 and w.x0.max() <= 10.0
    assert abs(w.field.w.mean()) < 0.1 and abs(w.field.w.std() - 1.0) < 0.1


def test_fitted_2d_workload_small():
    w = wl.config2(N=4096, M=2048, n_fit=20_000)
    assert w.field.centres.shape == (2048, 2) and w.field.gamma == 8.0 and w.T == 50
    assert w.boxes.shape == (64, 4)
    sides = w.boxes[:, 2:] - w.boxes[:, :2]
    assert sides.min() >= 0.3 - 1e-6 and sides.max() <= 1.5 + 1e-6
    assert np.array_equal(w.fit_y, wl.inside_boxes(w.boxes, w.fit_X))
    assert 0.0 < w.fit_y.mean() < 0.5                      # obstacles cover part of the square
    assert w.x0.min() >= 0.0 and w.x0.max() <= 10.0


def test_rff_7d_workload_small():
    w = wl.config3(N=2048, M=4096)
    om, ph, wt = w.field.centres, w.field.phase, w.field.w
    assert om.shape == (4096, 7) and w.T == 20 and w.extra["k"] == 5
    assert abs(om.var() - 2.0) < 0.05                      # Omega ~ N(0, 2 I)
    assert ph.min() >= 0.0 and ph.max() < 2 * np.pi + 1e-6
    assert abs(wt.var() * 4096 - 1.0) < 0.1                # w ~ N(0, 1 / M)
    assert np.abs(w.x0).max() <= np.pi + 1e-6 and w.extra["gT"].shape == (2048, 7)


def test_batched_environments():
    envs = wl.config4(n_envs=32)
    assert len(envs) == 32
    for e in envs:
        d, M, N = e.field.d, e.field.M, e.x0.shape[0]
        assert d in (2, 3) and 256 <= M <= 8192 and 1024 <= N <= 65536 and e.T == 30
        assert e.field.gamma == 4.0 and e.x0.min() >= 0.0 and e.x0.max() <= 10.0
    assert {e.field.d for e in envs} == {2, 3}


def test_surrogate_workload_small():
    w = wl.config5(N=4096, M=1024, n_fit=20_000, n_train=4096)
    assert w.field.centres.shape == (1024, 3) and w.field.gamma == 8.0 and w.T == 40
    assert w.boxes.shape == (48, 6)
    sides = w.boxes[:, 3:] - w.boxes[:, :3]
    assert sides.min() >= 0.15 - 1e-6 and sides.max() <= 0.75 + 1e-6
    assert w.x0.max() <= 5.0 and w.extra["x_train"].shape == (4096, 3)


def test_inputs_are_reproducible():
    a, b = wl.config3(N=256, M=64), wl.config3(N=256, M=64)
    assert np.array_equal(a.x0, b.x0) and np.array_equal(a.field.centres, b.field.centres)
    assert not np.array_equal(wl.config3(seed=4, N=256, M=64).x0, a.x0)
