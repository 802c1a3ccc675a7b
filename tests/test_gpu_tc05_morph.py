"""GPU parity of the tensor-core RBF morph (the fast path's tcgen05 kernel:
the exponent's affine part as a TF32 hi/lo MMA, ex2 and the weighted sums on
the CUDA cores) against the FP64 oracle, and against the FP32 tile kernel.

The fast path takes that kernel only when PDMP_RBF_TC05=1 is set (it is
slower than the FP32 tile kernel on the benchmarked workload); these tests
set it at sizes the oracle checks in seconds, and unset it (=0) for the
comparison with the FP32 kernel.  Inputs are seeded and synthetic.
Tolerances are those of the other morph parity tests: the per-step bound of
gpu_util.per_step_check and 1e-4 on x_T.

256-sample groups whose bounding box is too wide for the expanded form
(g' R^2 > 2) take a direct FP32 loop; compact inputs (many samples in a small box)
exercise the tensor-core form, spread inputs the direct one, and a mixture
both within one launch."""
import numpy as np
import pytest
import torch

import oracle
import paper_2108_11775_gb300 as pdmp
import workloads as wl
from gpu_util import max_abs, per_step_check, rbf_eta, setup_oracle_threads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    setup_oracle_threads()
    pdmp.lib()
    yield
    st, detail = pdmp.stream_status()
    assert st == 0, (st, detail)


@pytest.fixture
def tc05(monkeypatch):
    def use(on: bool):
        monkeypatch.setenv("PDMP_RBF_TC05", "1" if on else "0")
    use(True)
    return use


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _field(d, M, seed=5):
    return wl.random_field(seed + d + M, wl.RBF, d, M, lo=0, hi=3, gamma=3.0, wscale=2.0, bias=0.25)


def _check(f, x0, T, eta, idx=None, exact=True):
    """Trace per step and x_T against the oracle (on the samples idx).
    exact: the morph and its trace twin agree bit for bit; not for clustered
    inputs, whose crowded sort cells keep the samples' arrival order, so that
    group membership (and the rounding) can differ from run to run."""
    fld = pdmp.DeviceField.from_host(f)
    traj, steps = pdmp.morph_trace(fld, dev(x0), T, eta)
    traj, steps = traj.cpu().numpy(), steps.cpu().numpy()
    xT = pdmp.morph(fld, dev(x0), T, eta).cpu().numpy()
    if exact:
        assert np.array_equal(xT, traj[-1]), "morph and its trace twin disagree"
    else:
        assert max_abs(xT, traj[-1]) <= 1e-6
    if idx is None:
        idx = np.arange(x0.shape[0])
    per_step_check(f, traj[:, idx], steps[:, idx], eta)
    assert max_abs(xT[idx], oracle.morph(f, x0[idx], T, eta)) <= 1e-4
    return fld, xT


@pytest.mark.parametrize("d,M,N,T", [
    (2, 300, 4000, 6), (2, 64, 1537, 5), (2, 65, 513, 4), (2, 1, 100, 3), (2, 1000, 2048, 4),
    (3, 513, 4000, 5), (3, 63, 777, 4), (3, 128, 1, 3),
])
def test_compact_samples_tensor_core_form(tc05, d, M, N, T):
    """Samples in a box of side 0.5 in the middle of the centres: even a group
    spanning the whole box has g' R^2 <= 0.82 < 2, so every step runs on the
    tensor cores; ragged N (partial groups and row tiles) and M (partial
    chunks)."""
    f = _field(d, M)
    eta, _ = rbf_eta(f, np.full(d, 0.5), np.full(d, 2.5), cells=32 if d < 3 else 12)
    x0 = wl.uniform_box(70 + N, 3, N, np.full(d, 1.25), np.full(d, 1.75))
    _check(f, x0, T, eta)


@pytest.mark.parametrize("d", [2, 3])
def test_spread_and_mixed_samples_direct_form(tc05, d):
    """Spread samples (wide groups: the direct FP32 loop) and a mixture of a
    dense cluster and spread samples (both forms in one launch)."""
    f = _field(d, 200)
    eta, _ = rbf_eta(f, np.full(d, -1.5), np.full(d, 4.5), cells=32 if d < 3 else 12)
    spread = wl.uniform_box(90 + d, 3, 600, np.full(d, -1.0), np.full(d, 4.0))
    _check(f, spread, 4, eta)
    cluster = wl.uniform_box(91 + d, 3, 3000, np.full(d, 1.2), np.full(d, 1.8))
    mixed = np.concatenate([cluster, spread]).astype(np.float32)
    _check(f, mixed, 4, eta, exact=False)


@pytest.mark.parametrize("d", [2, 3])
def test_tensor_core_kernel_against_fp32_kernel(tc05, d):
    """The same compact input through both tile kernels: x_T within 1e-5 of
    each other after T steps; each is deterministic run to run; checkpoints
    equal the trace."""
    # weights small enough that sigma' stays large: the samples move by up
    # to 1e-2 (d = 2) and 6e-3 (d = 3) over the T steps
    f = wl.random_field(11 + d + 700, wl.RBF, d, 700, lo=0, hi=3, gamma=3.0, wscale=0.5, bias=0.0)
    eta, _ = rbf_eta(f, np.full(d, 0.5), np.full(d, 2.5), cells=32 if d < 3 else 12)
    N, T, k = 6000, 20, 4
    x0 = dev(wl.uniform_box(120 + d, 3, N, np.full(d, 1.25), np.full(d, 1.75)))
    fld = pdmp.DeviceField.from_host(f)
    ckpt = torch.empty(T // k, N, d, device="cuda")
    a = pdmp.morph(fld, x0, T, eta, ckpt=ckpt, k=k).cpu().numpy()
    a2 = pdmp.morph(fld, x0, T, eta).cpu().numpy()
    assert np.array_equal(a, a2), "the tensor-core kernel is not deterministic"
    traj, _ = pdmp.morph_trace(fld, x0, T, eta)
    assert np.array_equal(ckpt.cpu().numpy(), traj.cpu().numpy()[k::k])
    tc05(False)
    b = pdmp.morph(fld, x0, T, eta).cpu().numpy()
    assert max_abs(a, b) <= 1e-5
    assert np.abs(b - x0.cpu().numpy()).max() > 1e-3   # the samples moved (100x the tolerance)


def test_in_place_and_single_step(tc05):
    f = _field(2, 257)
    eta, _ = rbf_eta(f, np.full(2, 0.5), np.full(2, 2.5), cells=32)
    x0 = wl.uniform_box(140, 3, 2500, np.full(2, 1.25), np.full(2, 1.75))
    fld = pdmp.DeviceField.from_host(f)
    ref = pdmp.morph(fld, dev(x0), 1, eta).cpu().numpy()
    x = dev(x0)
    pdmp.morph(fld, x, 1, eta, out=x)
    assert np.array_equal(x.cpu().numpy(), ref)
    assert max_abs(ref, oracle.morph(f, x0, 1, eta)) <= 1e-5
