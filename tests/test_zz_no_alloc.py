"""pdmp_morph_noalloc: the fast morph on the library's built-in scratch.

Some callers cannot allocate device memory (for example a planning loop that
must never touch the allocator); this entry point lets them morph samples
with only the input and output buffers they own.  It is checked here against
pdmp_morph with a caller-provided workspace, through the C ABI, on two calls
in a row (the scratch keeps the previous call's contents, so the second call
shows that whatever must start at zero is cleared).
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2108_11775_gb300 as pdmp
import workloads as wl

pytestmark = pytest.mark.gpu


def _call(f, x, T, eta, out):
    L = pdmp.lib()
    fn = L.pdmp_morph_noalloc
    fn.argtypes = [ctypes.POINTER(pdmp._Field), ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float,
                   ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int32
    s = f.struct()
    return fn(ctypes.byref(s), x.data_ptr(), x.shape[0], T, eta, out.data_ptr(),
              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("d", [2, 3])
def test_noalloc_matches_workspace_morph_on_two_calls(d):
    assert torch.cuda.is_available()
    oracle.set_threads(1)
    if d == 2:
        f = wl.config1().field
        lo, hi, N, T = np.zeros(2), np.full(2, 10.0), 1 << 16, 10
        L, _ = oracle.lipschitz(f, lo, hi, cells=64)
    else:
        f = wl.random_field(91, wl.RBF, 3, 4096, lo=0, hi=5, gamma=8.0, wscale=2.0)
        lo, hi, N, T = np.zeros(3), np.full(3, 5.0), 1 << 17, 6
        L, _ = oracle.lipschitz(f, lo - 0.5, hi + 0.5, cells=12)
    eta = float(np.float32(0.5 / L))
    fld = pdmp.DeviceField.from_host(f)
    xs = [torch.from_numpy(wl.uniform_box(200 + i, 3, N, lo, hi)).cuda() for i in range(2)]
    for i, x in enumerate(xs):                      # two calls in a row, different inputs
        out = torch.full_like(x, float("nan"))
        torch.cuda.synchronize()
        free0, allocs0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        assert _call(fld, x, T, eta, out) == 0
        torch.cuda.synchronize()
        if i:                                       # the first call may load the module; the second allocates nothing
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == allocs0
        ref = pdmp.morph(fld, x, T, eta, fast=True)
        torch.cuda.synchronize()
        assert pdmp.stream_status()[0] == 0
        assert torch.isfinite(out).all()
        assert float((out - ref).abs().max()) <= 1e-4
        assert torch.equal(out, ref)                # same kernel, same arithmetic


def test_noalloc_rejects_requests_beyond_its_scratch():
    w1 = wl.config1()
    fld = pdmp.DeviceField.from_host(w1.field)
    big = torch.zeros((1 << 20) + 1, 2, device="cuda")
    assert _call(fld, big, 3, 1e-3, big) == 3       # N above 2^20
    rff = pdmp.DeviceField.from_host(wl.random_field(1, wl.RFF, 7, 64))
    x7 = torch.zeros(16, 7, device="cuda")
    assert _call(rff, x7, 3, 1e-3, x7) == 8         # only the fast RBF path has a no-alloc variant
    assert pdmp.stream_status()[0] == 0
