"""A C program that uses only include/pdmp.h, libpdmp.so and the CUDA runtime
(examples/morph_c.c): built with nvcc and run; its samples move and the
status is clean."""
import os
import re
import subprocess

import pytest

import paper_2108_11775_gb300 as pdmp

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_on_the_boundary(tmp_path):
    lib = pdmp.lib()._name
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "morph_c")
    subprocess.run(["nvcc", "-o", exe, os.path.join(ROOT, "examples", "morph_c.c"), "-I", os.path.join(ROOT, "include"),
                    "-L", libdir, "-lpdmp", "-Xlinker", f"-rpath={libdir}"], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    m = re.search(r"checksum=([-0-9.e+]+) max_displacement=([-0-9.e+]+)", out)
    assert m, out
    assert float(m.group(2)) > 1e-4 and float(m.group(1)) == float(m.group(1))
