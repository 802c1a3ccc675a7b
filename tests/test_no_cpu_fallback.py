"""The product path has no CPU fallback: handed host (CPU) tensors, every
entry point of the binding refuses before the library computes anything,
rather than quietly computing on the host."""
import numpy as np
import pytest
import torch

import paper_2108_11775_gb300 as pdmp
import workloads as wl


def _host_case():
    f = wl.random_field(5, wl.RBF, 2, 64, lo=0.0, hi=4.0, gamma=4.0, wscale=1.0)
    fld = pdmp.DeviceField.from_host(f, device="cpu")
    x = torch.from_numpy(wl.uniform_box(5, 3, 32, np.zeros(2), np.full(2, 4.0)))
    return fld, x


@pytest.mark.parametrize("call", ["morph", "morph_vjp", "logdet", "morph_inverse", "occupancy_query"])
def test_host_tensors_are_refused(call):
    fld, x = _host_case()
    with pytest.raises(TypeError, match="CUDA tensor"):
        if call == "morph":
            pdmp.morph(fld, x, 4, 1e-3, fast=False)
        elif call == "morph_vjp":
            pdmp.morph_vjp(fld, x, 4, 1e-3, 2, torch.ones_like(x), fast=False)
        elif call == "logdet":
            pdmp.logdet(fld, x, 4, 1e-3, fast=False)
        elif call == "morph_inverse":
            pdmp.morph_inverse(fld, x, 4, 1e-3, fast=False)
        else:
            pdmp.occupancy_query(fld, x)
