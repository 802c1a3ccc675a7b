"""The tcgen05 descriptors and operand layout of csrc/tc05.cuh, checked on the
host (g++ compiles the header's constexpr builders; no GPU).

Each descriptor is decoded here field by field with the bit ranges of the PTX
ISA's tcgen05 tables (instruction descriptor for kind::f16 / kind::tf32;
shared-memory descriptor), and every field must hold the intended value with
all reserved bits zero.  The canonical K-major layout (core matrices of
8 rows x 16 bytes, 128 contiguous bytes each) must map a whole operand onto
its bytes one to one."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2108_11775_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "tc05.cuh"
using namespace pdmp::tc05;
int main() {
  const int shapes[][2] = {{128, 128}, {128, 16}, {128, 256}, {64, 8}, {128, 32}};
  for (auto& s : shapes) {
    std::printf("idesc bf16 %d %d %u\n", s[0], s[1], idesc(kBF16, kBF16, s[0], s[1]));
    std::printf("idesc tf32 %d %d %u\n", s[0], s[1], idesc(kTF32, kTF32, s[0], s[1]));
  }
  const unsigned addrs[] = {0x0u, 0x400u, 0x12340u, 0x3fff0u, 0x1024f0u};
  for (unsigned a : addrs) std::printf("sdesc %u 128 2048 %llu\n", a, (unsigned long long)sdesc(a, 128, 2048));
  std::printf("sdesc %u 256 1536 %llu\n", 0x8000u, (unsigned long long)sdesc(0x8000u, 256, 1536));
  for (int kc = 1; kc <= 16; kc *= 2)
    for (int es = 2; es <= 4; es *= 2)
      for (int r = 0; r < 32; ++r)
        for (int k = 0; k < kc * 16 / es; ++k)
          std::printf("off %d %d %d %d %u\n", kc, es, r, k, kmajor_offset(r, k, kc, es));
  return 0;
}
"""


@pytest.fixture(scope="module")
def values(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("tc05")
    src = d / "t.cpp"
    src.write_text(PROGRAM)
    exe = d / "t"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    return [line.split() for line in out if line]


def field(v, lo, hi):
    """bits [lo, hi) of v"""
    return (v >> lo) & ((1 << (hi - lo)) - 1)


def test_instruction_descriptor_fields(values):
    rows = [r for r in values if r[0] == "idesc"]
    assert len(rows) == 10
    for _, kind, m, n, v in rows:
        m, n, v = int(m), int(n), int(v)
        fmt = 1 if kind == "bf16" else 2                  # kind::f16 BF16 = 1, kind::tf32 TF32 = 2
        assert field(v, 0, 2) == 0 and field(v, 2, 3) == 0 and field(v, 3, 4) == 0   # dense, no saturation
        assert field(v, 4, 6) == 1                        # D: F32
        assert field(v, 6, 7) == 0                        # reserved
        assert field(v, 7, 10) == fmt and field(v, 10, 13) == fmt
        assert field(v, 13, 14) == 0 and field(v, 14, 15) == 0   # no negation
        assert field(v, 15, 16) == 0 and field(v, 16, 17) == 0   # A and B K-major
        assert field(v, 17, 23) == n // 8
        assert field(v, 23, 24) == 0                      # reserved
        assert field(v, 24, 29) == m // 16
        assert field(v, 29, 32) == 0                      # reserved, no max shift
        assert v < (1 << 32)


def test_shared_memory_descriptor_fields(values):
    rows = [r for r in values if r[0] == "sdesc"]
    assert len(rows) == 6
    for _, addr, lbo, sbo, v in rows:
        addr, lbo, sbo, v = int(addr), int(lbo), int(sbo), int(v)
        assert field(v, 0, 14) == (addr & 0x3FFFF) >> 4   # start address, 16-byte units, 18-bit window
        assert field(v, 14, 16) == 0
        assert field(v, 16, 30) == lbo >> 4
        assert field(v, 30, 32) == 0
        assert field(v, 32, 46) == sbo >> 4
        assert field(v, 46, 48) == 1                      # descriptor version for tcgen05
        assert field(v, 48, 49) == 0
        assert field(v, 49, 52) == 0                      # base offset
        assert field(v, 52, 53) == 0                      # relative LBO
        assert field(v, 53, 61) == 0
        assert field(v, 61, 64) == 0                      # no swizzle


def test_kmajor_layout_is_a_bijection_of_core_matrices(values):
    by_shape = {}
    for _, kc, es, r, k, off in (x for x in values if x[0] == "off"):
        by_shape.setdefault((int(kc), int(es)), []).append((int(r), int(k), int(off)))
    assert len(by_shape) == 10
    for (kc, es), entries in by_shape.items():
        rows = 32
        total = rows * kc * 16                            # bytes of a 32-row operand
        starts = {}
        for r, k, off in entries:
            assert 0 <= off < total
            # byte (r, k) lies in core matrix (r // 8, k * es // 16) at row r % 8, byte (k * es) % 16
            core = (r // 8) * kc * 128 + (k * es // 16) * 128
            assert off == core + (r % 8) * 16 + (k * es) % 16
            starts[off] = (r, k)
        assert len(starts) == len(entries) == total // es  # one to one
