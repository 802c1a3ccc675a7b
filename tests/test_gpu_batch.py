"""Batched environments in one persistent launch: every environment's result
against the single-field morph and, on samples, against the FP64 oracle;
CUDA-graph replay; the autotuner."""
import numpy as np
import pytest
import torch

import oracle
import paper_2108_11775_gb300 as pdmp
import workloads as wl
from gpu_util import rbf_eta, setup_oracle_threads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available()
    setup_oracle_threads()
    yield
    assert pdmp.stream_status()[0] == 0


def small_envs(seed=7, n=12):
    g = wl.rng(seed, wl.S_ENV)
    envs, host = [], []
    for e in range(n):
        d = int(g.integers(2, 4))
        M = int(g.integers(1, 700)) if e else 1
        N = [0, 1, 255, 256, 257][e] if e < 5 else int(g.integers(100, 3000))
        T = int(g.integers(2, 6))
        f = wl.random_field(seed * 1000 + e, wl.RBF, d, M, lo=0, hi=4, gamma=3.0, wscale=1.5, bias=0.1)
        eta, _ = rbf_eta(f, np.full(d, -0.5), np.full(d, 4.5), cells=24 if d == 2 else 10)
        x0 = wl.uniform_box(seed * 1000 + e, 3, N, np.zeros(d), np.full(d, 4.0))
        host.append((f, x0, eta, T))
        envs.append((pdmp.DeviceField.from_host(f), torch.from_numpy(x0).cuda().reshape(N, d), eta, T))
    return envs, host


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_batched_matches_single_field_and_oracle(variant):
    envs, host = small_envs()
    b = pdmp.Batch(envs)
    b.prepare(variant)
    outs = [o.cpu().numpy() for o in b.run()]
    assert pdmp.stream_status()[0] == 0
    for (fld, x0, eta, T), (f, xh, _, _), out in zip(envs, host, outs):
        if x0.shape[0] == 0:
            continue
        single = pdmp.morph(fld, x0, T, eta).cpu().numpy()
        # tiles too wide for the expanded form take the direct form about the
        # tile centre here and about 0 in the single-field launch: rounding only
        assert np.abs(out - single).max() <= (1e-5 if variant == 0 else 1e-4)
        idx = np.arange(0, x0.shape[0], max(1, x0.shape[0] // 8))
        ref = oracle.morph(f, xh[idx], T, eta)
        assert np.abs(out[idx] - ref).max() <= 1e-4


@pytest.mark.parametrize("variant,sizes", [(2, [(2, 20000 + 17), (3, 60000 + 5), (2, 321)]),
                                           (0, [(2, (1 << 18) + 17), (3, (1 << 18) + 5)])])
def test_batched_variant_is_the_single_field_launch_on_compact_tiles(variant, sizes):
    """Variant 0 has the single-field launch's tile shape for launches that fill
    the GPU (320 samples), variant 2 its shape for smaller ones (128 samples):
    where every tile is compact enough for the expanded form (dense samples,
    small steps) the two agree bit for bit, in d = 2 and 3, with ragged last
    tiles."""
    envs, host = [], []
    for e, (d, N) in enumerate(sizes):
        f = wl.random_field(500 + e, wl.RBF, d, 300 + 100 * e, lo=0, hi=4, gamma=3.0, wscale=1.5, bias=0.1)
        eta, _ = rbf_eta(f, np.full(d, -0.5), np.full(d, 4.5), cells=24 if d == 2 else 10)
        x0 = wl.uniform_box(500 + e, 3, N, np.zeros(d), np.full(d, 4.0))
        if N == 321:
            x0 = np.ascontiguousarray(0.5 + 0.05 * x0)     # 321 samples in a box of side 0.2
        envs.append((pdmp.DeviceField.from_host(f), torch.from_numpy(x0).cuda(), eta, 3))
        host.append((f, x0))
    b = pdmp.Batch(envs)
    b.prepare(variant)
    outs = b.run()
    for (fld, x0, eta, T), out in zip(envs, outs):
        assert torch.equal(out, pdmp.morph(fld, x0, T, eta))
    assert pdmp.stream_status()[0] == 0


def test_batched_graph_replay_and_autotune(tmp_path):
    envs, _ = small_envs(seed=9, n=20)
    b = pdmp.Batch(envs, cache_path=str(tmp_path / "tune.json"))
    best, times = b.autotune(reps=1)
    assert 0 <= best < b.n_variants and len(times) == b.n_variants and all(t > 0 for t in times)
    assert b.plan.variant == best
    direct = [o.clone() for o in b.run()]
    for o in b.outputs:
        o.fill_(float("nan"))
    b.capture()
    torch.cuda.current_stream().wait_stream(b.graph_stream)
    b.replay()
    b.replay()
    torch.cuda.synchronize()
    for o, r in zip(b.outputs, direct):
        assert torch.equal(o, r)
    again = pdmp.Batch(envs, cache_path=str(tmp_path / "tune.json"))
    best2, times2 = again.autotune()
    assert best2 == best and times2 is None               # from the cache


def test_batched_config4_shape_sampled():
    """The 256-environment shape, scaled down in N, checked per environment on samples."""
    hosts = wl.config4(n_envs=256, N_range=(64, 512))
    envs = []
    for w in hosts:
        eta, _ = rbf_eta(w.field, w.lo - 0.5, w.hi + 0.5, cells=16 if w.field.d == 2 else 6)
        envs.append((pdmp.DeviceField.from_host(w.field), torch.from_numpy(w.x0).cuda(), eta, w.T))
    b = pdmp.Batch(envs)
    b.prepare(0)
    outs = b.run()
    torch.cuda.synchronize()
    assert pdmp.stream_status()[0] == 0
    for i in range(0, 256, 37):
        w, (fld, x0, eta, T) = hosts[i], envs[i]
        idx = np.arange(0, w.x0.shape[0], 97)
        ref = oracle.morph(w.field, w.x0[idx], T, eta)
        assert np.abs(outs[i].cpu().numpy()[idx] - ref).max() <= 1e-4


def test_host_watchdog_times_out_then_completes():
    """pdmp_stream_wait on a morph that runs for about a second: a 1 ms limit
    reports a timeout while the kernel keeps running, a long one then sees it
    finish (nothing faults or hangs: the kernel ends by itself)."""
    wk = wl.config2(N=1 << 20, M=16384, n_fit=1000)
    fld = pdmp.DeviceField.from_host(wl.Field(wl.RBF, wk.field.centres, np.full(16384, 0.01, np.float32), gamma=8.0))
    x0 = torch.from_numpy(wk.x0).cuda()
    out = pdmp.morph(fld, x0, 300, 1e-4)
    st, _ = pdmp.stream_wait(1)
    assert st == 6
    st, detail = pdmp.stream_wait(120_000)
    assert st == 0 and detail == 0
    assert torch.isfinite(out).all()


def test_stage_copy_wait_is_bounded():
    """The bounded wait the random Fourier kernels use for their bulk stage
    copies: with a copy it completes (the 16 floats arrive through shared
    memory); with nothing to complete the barrier it gives up after the
    limit, raises PDMP_FLAG_STAGE_TIMEOUT and the kernel ends (the context
    stays usable: a morph afterwards is correct and leaves the flag clear)."""
    src = torch.arange(16, dtype=torch.float32, device="cuda") * 0.5 - 3.0
    dst = torch.zeros(16, dtype=torch.float32, device="cuda")
    assert pdmp.selftest_stage_wait(1 << 20, src, dst) == (0, 0)
    assert torch.equal(dst, src)
    st, detail = pdmp.selftest_stage_wait(2_000_000)        # about a millisecond of spinning
    assert st == 7 and detail == 8                          # PDMP_ERR_DEVICE_FLAG, PDMP_FLAG_STAGE_TIMEOUT
    assert pdmp.stream_status() == (0, 0)                   # read and cleared
    f = wl.random_field(71, wl.RFF, 7, 300, wscale=6.0, bias=0.1)
    L, _ = oracle.lipschitz(f)
    eta = float(np.float32(0.5 / L))
    x0 = wl.uniform_box(71, 3, 256, np.full(7, -np.pi), np.full(7, np.pi))
    out = pdmp.morph(pdmp.DeviceField.from_host(f, lipschitz=L), torch.from_numpy(x0).cuda(), 4, eta).cpu().numpy()
    assert np.abs(out - oracle.morph(f, x0, 4, eta)).max() <= 1e-4
    assert pdmp.stream_status() == (0, 0)


def test_bound_calls_from_several_host_threads():
    """pdmp_lipschitz_bound and pdmp_cull_radius reduce into fixed device slots;
    called from four host threads at once they still return each field's own
    bound (the library serialises them)."""
    import threading
    fields = [wl.random_field(70 + i, wl.RBF, 2, 512 * (i + 1), lo=0, hi=10, gamma=4.0, wscale=0.5 + i) for i in range(4)]
    devs = [pdmp.DeviceField.from_host(f) for f in fields]
    lo, hi = np.full(2, -0.5), np.full(2, 10.5)
    serial = [pdmp.lipschitz_bound(d, lo, hi, cells=32) for d in devs]
    radii = [pdmp.cull_radius(d, 1e-6) for d in devs]
    out = [None] * 4

    def work(i):
        torch.cuda.set_device(0)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            res = []
            for _ in range(20):
                res.append((pdmp.lipschitz_bound(devs[i], lo, hi, cells=32), pdmp.cull_radius(devs[i], 1e-6)))
            out[i] = res

    threads = [threading.Thread(target=work, args=(i,)) for i in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=120)
    for i in range(4):
        assert out[i] is not None
        for lb, rr in out[i]:
            assert lb == serial[i] and rr == radii[i]
