"""torch.autograd through the Euler chain (forward pdmp_morph with
checkpoints, backward pdmp_morph_vjp): gradients against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_2108_11775_gb300 as pdmp
import workloads as wl
from gpu_util import rbf_eta, rff_eta_sampled, setup_oracle_threads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", [wl.RBF, wl.RFF])
def test_autograd_gradients_match_oracle(kind):
    assert torch.cuda.is_available()
    setup_oracle_threads()
    if kind == wl.RBF:
        f = wl.random_field(61, kind, 2, 200, lo=0, hi=4, gamma=3.0, wscale=1.5, bias=0.2)
        eta, _ = rbf_eta(f, np.full(2, -0.5), np.full(2, 4.5), cells=32)
        x0 = wl.uniform_box(61, 3, 300, np.zeros(2), np.full(2, 4.0))
        T, k = 8, 2
    else:
        f = wl.random_field(62, kind, 7, 128, wscale=5.0, bias=0.1)
        lo, hi = np.full(7, -np.pi), np.full(7, np.pi)
        eta, _ = rff_eta_sampled(f, lo, hi, n=500)
        x0 = wl.uniform_box(62, 3, 64, lo, hi)
        T, k = 10, 5
    fld = pdmp.DeviceField.from_host(f)
    x = torch.from_numpy(x0).cuda().requires_grad_(True)
    w = fld.w.clone().requires_grad_(True)
    b = torch.tensor(f.bias, device="cuda", requires_grad=True)
    xT = pdmp.morph_autograd(fld, x, T, eta, k=k, w=w, bias=b)
    gT = torch.from_numpy(wl.f32(wl.rng(63, 1).standard_normal(x0.shape))).cuda()
    (xT * gT).sum().backward()
    g0, gw, gb = oracle.morph_vjp(f, x0, T, eta, gT.cpu().numpy(), want_gw=True)
    assert np.linalg.norm(x.grad.cpu().numpy() - g0) <= 1e-4 * np.linalg.norm(g0)
    assert np.linalg.norm(w.grad.cpu().numpy() - gw) <= 1e-4 * np.linalg.norm(gw)
    assert abs(float(b.grad) - gb) <= 1e-4 * max(abs(gb), 1e-3)
    np.testing.assert_allclose(xT.detach().cpu().numpy(), oracle.morph(f, x0, T, eta), atol=1e-4)
