"""The C ABI: the library loads without a GPU, exports every function the
header declares, and rejects bad arguments on the host before any launch."""
import ctypes
import os
import re

import pytest

import paper_2108_11775_gb300 as pdmp

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "pdmp.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(pdmp_[a-z_0-9]+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for must in ("pdmp_morph", "pdmp_morph_vjp", "pdmp_logdet", "pdmp_fit_occupancy", "pdmp_lipschitz_bound",
                 "pdmp_box_labels", "pdmp_occupancy_query", "pdmp_status_string", "pdmp_stream_status"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = pdmp.lib()
    for name in declared_functions():
        assert hasattr(L, name), f"{name} declared in pdmp.h but not exported"


def test_status_strings():
    L = pdmp.lib()
    for s in range(0, 9):
        assert L.pdmp_status_string(s)
    assert L.pdmp_status_string(12345) == b"unknown status"
    assert L.pdmp_version() >= 200


# Fake, never-dereferenced device addresses: every call below fails host
# validation before any CUDA call.  They run only where no GPU is visible, so
# that a validation gap can never turn into a launch on a bogus pointer.
import torch

nogpu = pytest.mark.skipif(torch.cuda.is_available(), reason="fake-pointer validation tests run without a GPU only")
A = 1 << 20          # 16-byte aligned
MIS = (1 << 20) + 4  # misaligned


def fld(kind=0, d=2, M=16, gamma=4.0, centres=A, w=A, phase=None, lipschitz=0.0):
    f = pdmp._Field()
    f.kind, f.d, f.M, f.gamma, f.bias, f.lipschitz = kind, d, M, gamma, 0.0, lipschitz
    f.centres, f.w, f.phase = centres, w, phase
    return f


def morph_call(f, x0=A, N=8, T=4, eta=0.01, xT=A, ckpt=None, k=0, ws=None, ws_bytes=0):
    return pdmp.lib().pdmp_morph(ctypes.byref(f), x0, N, T, eta, xT, ckpt, k, ws, ws_bytes, None)


@nogpu
@pytest.mark.parametrize("bad", [
    dict(M=0), dict(d=4), dict(d=0), dict(kind=2), dict(gamma=0.0), dict(gamma=float("nan")),
    dict(centres=None), dict(centres=MIS), dict(w=MIS), dict(phase=A), dict(lipschitz=-1.0),
])
def test_morph_rejects_bad_rbf_fields(bad):
    assert morph_call(fld(**bad)) == 1


@nogpu
def test_rff_field_needs_phase_and_allows_d8():
    assert morph_call(fld(kind=1, d=7, phase=None)) == 1
    assert morph_call(fld(kind=1, d=9, phase=A)) == 1
    assert morph_call(fld(kind=1, d=8, phase=MIS)) == 1


@nogpu
@pytest.mark.parametrize("kw,code", [
    (dict(N=-1), 1), (dict(T=-1), 1), (dict(eta=0.0), 1), (dict(eta=-1.0), 1), (dict(eta=float("inf")), 1),
    (dict(x0=MIS), 1), (dict(xT=None), 1), (dict(ckpt=A, k=3), 1), (dict(ckpt=A, k=0), 1), (dict(ckpt=MIS, k=2), 1),
])
def test_morph_rejects_bad_arguments(kw, code):
    assert morph_call(fld(), **kw) == code


@nogpu
def test_step_too_large_when_field_carries_L():
    assert morph_call(fld(lipschitz=100.0), eta=0.0101) == 2
    assert morph_call(fld(lipschitz=100.0), eta=0.5) == 2


@nogpu
def test_morph_workspace_size_and_checks():
    L = pdmp.lib()
    f = fld()
    need = L.pdmp_morph_workspace(ctypes.byref(f), 1 << 20)
    assert need > (1 << 20) * 8                       # keys + permutation at least
    # RFF, d = 8: the pair table (M records of 11 u64 pairs, padded to 16 bytes, 256 in all)
    pair8 = L.pdmp_morph_workspace(ctypes.byref(fld(kind=1, d=8, phase=A)), 1 << 20)
    assert pair8 == (16 * 12 * 8 + 255) // 256 * 256
    # RFF, d <= 7: the tensor-core table (k tiles of 8 features, 776 floats each, whole stages of 16)
    assert L.pdmp_morph_workspace(ctypes.byref(fld(kind=1, d=7, phase=A)), 1 << 20) == 16 * 776 * 4
    assert L.pdmp_morph_workspace(ctypes.byref(fld(kind=1, d=3, phase=A)), 1 << 20) == 16 * 776 * 4
    assert L.pdmp_morph_workspace(ctypes.byref(fld(kind=1, d=7, M=129, phase=A)), 1) == 32 * 776 * 4
    assert L.pdmp_morph_workspace(ctypes.byref(fld(d=1)), 1000) == 0
    assert morph_call(f, N=1 << 20, ws=A, ws_bytes=need - 1) == 3
    assert morph_call(f, N=1 << 20, ws=MIS, ws_bytes=need) == 1


@nogpu
def test_empty_batch_is_a_noop():
    assert morph_call(fld(), N=0, x0=None, xT=None) == 0


@nogpu
def test_vjp_validation():
    L = pdmp.lib()
    f = fld()
    # k must divide T and be at most the longest segment
    assert L.pdmp_morph_vjp(ctypes.byref(f), A, 8, 10, 0.01, 3, None, A, A, None, None, None, 0, None) == 1
    assert L.pdmp_morph_vjp(ctypes.byref(f), A, 8, 64, 0.01, 64, None, A, A, None, None, None, 0, None) == 1
    need = L.pdmp_morph_vjp_workspace(ctypes.byref(f), 1000, 10, 5, 2)   # the parameter gradient's rows
    assert need > 0
    # RBF, d = 2, k <= 16: the full size adds the sorted tiles' workspace (the morph's) after the rows
    assert (L.pdmp_morph_vjp_workspace(ctypes.byref(f), 1000, 10, 5, 1)
            == need + L.pdmp_morph_workspace(ctypes.byref(f), 1000))
    assert L.pdmp_morph_vjp_workspace(ctypes.byref(f), 1000, 32, 32, 1) == need   # segment too long: rows only
    # RBF, d = 2, no parameter gradient: the optional sorted-tile workspace (the morph's)
    assert L.pdmp_morph_vjp_workspace(ctypes.byref(f), 1000, 10, 5, 0) == L.pdmp_morph_workspace(ctypes.byref(f), 1000)
    assert L.pdmp_morph_vjp_workspace(ctypes.byref(fld(d=1)), 1000, 10, 5, 0) == 0
    assert L.pdmp_morph_vjp(ctypes.byref(f), A, 1000, 10, 0.01, 5, None, A, A, A, None, A, need - 1, None) == 3
    assert L.pdmp_morph_vjp(ctypes.byref(f), A, 1000, 10, 0.01, 5, None, A, A, A, None, None, need, None) == 1
    # RFF, d <= 7, k <= 16, no parameter gradient: the optional tensor-core table
    fr = fld(kind=1, d=7, M=16, phase=A)
    assert L.pdmp_morph_vjp_workspace(ctypes.byref(fr), 1000, 10, 5, 0) == 16 * 776 * 4
    assert L.pdmp_morph_vjp_workspace(ctypes.byref(fr), 1000, 32, 32, 0) == 0         # segment too long
    assert L.pdmp_morph_vjp_workspace(ctypes.byref(fld(kind=1, d=8, phase=A)), 1000, 10, 5, 0) == 0
    assert L.pdmp_morph_vjp(ctypes.byref(fr), A, 1000, 10, 0.01, 5, None, A, A, None, None, A,
                            16 * 776 * 4 - 1, None) == 3
    assert L.pdmp_morph_vjp(ctypes.byref(fr), A, 1000, 10, 0.01, 5, None, A, A, None, None, MIS,
                            16 * 776 * 4, None) == 1
    # with the parameter gradient: the per-block rows (8 blocks of 128 samples x (M + 1) floats, rounded
    # to 256 bytes), then the tensor-core table; the rows alone are the minimum
    rows = 256 * ((8 * 17 * 4 + 255) // 256)
    assert L.pdmp_morph_vjp_workspace(ctypes.byref(fr), 1000, 10, 5, 1) == rows + 16 * 776 * 4
    assert L.pdmp_morph_vjp_workspace(ctypes.byref(fr), 1000, 32, 32, 1) == rows
    assert L.pdmp_morph_vjp_workspace(ctypes.byref(fr), 1000, 10, 5, 2) == rows
    assert L.pdmp_morph_vjp(ctypes.byref(fr), A, 1000, 10, 0.01, 5, None, A, A, A, None, A, rows - 1, None) == 3
    assert L.pdmp_morph_vjp(ctypes.byref(fr), A, 1000, 10, 0.01, 5, None, A, A, None, A, MIS, rows, None) == 1


@nogpu
def test_fit_and_lipschitz_validation():
    L = pdmp.lib()
    f = fld()
    assert L.pdmp_fit_workspace(16, 100) > 0
    ws = L.pdmp_fit_workspace(16, 100)
    assert L.pdmp_fit_occupancy(ctypes.byref(f), A, A, 100, 1e-3, 0, 10, A, None, None, None, A, ws, None) == 1
    assert L.pdmp_fit_occupancy(ctypes.byref(f), A, A, 100, 1e-3, 5, 10, A, None, None, None, A, ws - 1, None) == 3
    assert L.pdmp_fit_occupancy(ctypes.byref(f), A, A, 0, 1e-3, 5, 10, A, None, None, None, A, ws, None) == 1
    Lo = ctypes.c_double(0)
    lo = (ctypes.c_double * 2)(0, 0)
    hi = (ctypes.c_double * 2)(10, 0)      # empty extent on axis 1
    assert L.pdmp_lipschitz_bound(ctypes.byref(f), lo, hi, 8, ctypes.byref(Lo), None, None) == 1
    hi = (ctypes.c_double * 2)(10, 10)
    assert L.pdmp_lipschitz_bound(ctypes.byref(f), lo, hi, 0, ctypes.byref(Lo), None, None) == 1
    assert L.pdmp_lipschitz_bound(ctypes.byref(f), lo, hi, 5000, ctypes.byref(Lo), None, None) == 1


@nogpu
def test_labels_validation():
    L = pdmp.lib()
    assert L.pdmp_box_labels(0, A, 1, A, 10, A, None) == 1
    assert L.pdmp_box_labels(9, A, 1, A, 10, A, None) == 1
    assert L.pdmp_box_labels(2, None, 3, A, 10, A, None) == 1
    assert L.pdmp_box_labels(2, A, 1, A, 0, A, None) == 0


@nogpu
def test_inverse_validation():
    L = pdmp.lib()
    fn = L.pdmp_morph_inverse
    f = ctypes.byref(fld())
    need = L.pdmp_morph_workspace(f, 8)
    assert need > 0
    assert fn(f, A, 8, 4, 0.01, 1e-6, 0, A, None, None, 0, None, None) == 1            # maxit < 1
    assert fn(f, A, 8, 4, 0.01, -1.0, 10, A, None, None, 0, None, None) == 1           # negative tolerance
    assert fn(f, A, 8, 4, 0.01, float("nan"), 10, A, None, None, 0, None, None) == 1
    assert fn(f, MIS, 8, 4, 0.01, 1e-6, 10, A, None, None, 0, None, None) == 1
    assert fn(f, A, 8, 4, 0.01, 1e-6, 10, A, MIS + 1, None, 0, None, None) == 1       # iters not 4-byte aligned
    assert fn(f, A, -1, 4, 0.01, 1e-6, 10, A, None, None, 0, None, None) == 1
    assert fn(f, A, 8, 4, 0.01, 1e-6, 10, A, None, A + 8192, need - 1, None, None) == 3   # workspace too small
    assert fn(f, A, 8, 4, 0.01, 1e-6, 10, A, None, MIS, need, None, None) == 1         # workspace misaligned
    assert fn(f, A, 8, 4, 0.01, 1e-6, 10, A, None, None, 0, A + 4, None) == 1          # work not 8-byte aligned
    assert fn(f, None, 0, 4, 0.01, 1e-6, 10, None, None, None, 0, None, None) == 0      # empty batch
    assert fn(ctypes.byref(fld(lipschitz=100.0)), A, 8, 4, 0.5, 1e-6, 10, A, None, None, 0, None, None) == 2


@nogpu
def test_log_density_validation():
    fn = pdmp.lib().pdmp_log_density
    lo = (ctypes.c_double * 2)(0, 0)
    hi = (ctypes.c_double * 2)(10, 10)
    flat = (ctypes.c_double * 2)(10, 0)
    f = ctypes.byref(fld())
    need = pdmp.lib().pdmp_morph_workspace(f, 8)
    P = lambda a: ctypes.cast(a, ctypes.POINTER(ctypes.c_double))
    assert fn(f, A, 8, 4, 0.01, P(lo), P(flat), 1e-6, 10, A + 4096, A, None, 0, None) == 1     # empty box
    assert fn(f, A, 8, 4, 0.01, None, P(hi), 1e-6, 10, A + 4096, A, None, 0, None) == 1
    assert fn(f, A, 8, 4, 0.01, P(lo), P(hi), 1e-6, 10, A, A + 4096, None, 0, None) == 1       # y aliases z
    assert fn(f, A, 8, 4, 0.01, P(lo), P(hi), 1e-6, 0, A + 4096, A + 8192, None, 0, None) == 1
    assert fn(f, A, 8, 4, 0.01, P(lo), P(hi), 1e-6, 10, A + 4096, A + 8192, A + 16384, need - 1, None) == 3
    assert fn(f, None, 0, 4, 0.01, P(lo), P(hi), 1e-6, 10, None, None, None, 0, None) == 0


@nogpu
def test_culled_validation():
    L = pdmp.lib()
    f = fld()
    need = L.pdmp_morph_culled_workspace(ctypes.byref(f), 1000)
    assert need > 1000 * 8
    assert L.pdmp_morph_culled_workspace(ctypes.byref(fld(kind=1, d=7, phase=A)), 1000) == 0
    call = lambda ff, **kw: L.pdmp_morph_culled(
        ctypes.byref(ff), kw.get("x0", A), kw.get("N", 1000), kw.get("T", 4), kw.get("eta", 0.01),
        kw.get("r", 1.0), kw.get("xT", A), None, 0, kw.get("ws", A), kw.get("ws_bytes", need), kw.get("work", None),
        None)
    assert call(fld(kind=1, d=7, phase=A)) == 8                 # RFF: unsupported
    assert call(fld(d=1)) == 8
    assert call(f, r=0.0) == 1
    assert call(f, r=float("inf")) == 1
    assert call(f, ws=None) == 1
    assert call(f, ws_bytes=need - 1) == 3
    assert call(f, work=A + 4) == 1                              # not 8-byte aligned
    assert call(f, N=0, x0=None, xT=None, ws=None) == 0
    r = ctypes.c_float(0)
    assert L.pdmp_cull_radius(ctypes.byref(f), 0.0, ctypes.byref(r), None, None) == 1
    assert L.pdmp_cull_radius(ctypes.byref(fld(kind=1, d=7, phase=A)), 1e-6, ctypes.byref(r), None, None) == 8


@nogpu
def test_tanh_net_validation():
    L = pdmp.lib()

    def net(d=2, H=64, W1=A, W2=A, b3=0.0, lipschitz=0.0):
        n = pdmp._TanhNet()
        n.d, n.H, n.W1, n.b1, n.W2, n.b2, n.w3, n.b3, n.lipschitz = d, H, W1, A, W2, A, A, b3, lipschitz
        return n

    call = lambda n, **kw: L.pdmp_tanh_net_morph(ctypes.byref(n), kw.get("x0", A), kw.get("N", 100),
                                                 kw.get("T", 4), kw.get("eta", 0.01), kw.get("xT", A),
                                                 kw.get("ckpt", None), kw.get("k", 0), None)
    assert call(net(d=4)) == 8 and call(net(H=48)) == 8          # unsupported shapes
    assert call(net(d=0)) == 1 and call(net(d=9)) == 1
    assert call(net(W1=None)) == 1 and call(net(W2=MIS)) == 1
    assert call(net(b3=float("nan"))) == 1
    assert call(net(lipschitz=-1.0)) == 1
    assert call(net(lipschitz=100.0), eta=0.011) == 2
    assert call(net(), eta=0.0) == 1 and call(net(), N=-1) == 1
    assert call(net(), ckpt=A, k=3) == 1
    assert call(net(), N=0, x0=None, xT=None) == 0
    assert L.pdmp_tanh_net_query(ctypes.byref(net()), MIS, 10, None, None, None, None) == 1
    assert L.pdmp_tanh_net_lipschitz(ctypes.byref(net()), None, None, None) == 1


@nogpu
def test_fast_paths_reject_sample_counts_past_int32():
    L = pdmp.lib()
    f = fld()
    big = (1 << 31) + 5
    assert morph_call(f, N=big, ws=A, ws_bytes=1 << 62) == 1
    assert L.pdmp_morph_culled(ctypes.byref(f), A, big, 4, 0.01, 1.0, A, None, 0, A, 1 << 62, None, None) == 1


@nogpu
def test_stream_wait_rejects_a_negative_timeout():
    assert pdmp.lib().pdmp_stream_wait(None, -1, None) == 1


@nogpu
def test_stage_wait_selftest_validation():
    L = pdmp.lib()
    assert L.pdmp_selftest_stage_wait(None, None, 0, 0, None) == 1                 # limit below 1 clock
    assert L.pdmp_selftest_stage_wait(None, None, (1 << 31) + 1, 0, None) == 1     # above 2^31 clocks
    assert L.pdmp_selftest_stage_wait(MIS, A, 1000, 1, None) == 1                  # src not 16-byte aligned
    assert L.pdmp_selftest_stage_wait(A, None, 1000, 1, None) == 1                 # copy without dst


def test_header_is_plain_c99():
    """The boundary header compiles as pedantic C99 (no C++ or CUDA types)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    r = subprocess.run(["gcc", "-fsyntax-only", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-x", "c",
                        HEADER], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
