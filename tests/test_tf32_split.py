"""The two hi/lo splits the tensor-core kernels feed to TF32 MMAs, emulated
in float32 on the CPU: the head must be an exact TF32 value (its low 13
mantissa bits zero, so the tensor core uses it unchanged) and the tail small
enough that reading only its TF32 part costs at most about 2^-22."""
import numpy as np


def _tf32_exact(x):
    return (np.asarray(x, np.float32).view(np.uint32) & 0x1FFF) == 0


def test_veltkamp_split_gives_an_exact_tf32_head():
    rng = np.random.default_rng(3)
    a = (rng.standard_normal(200_000) * 10.0 ** rng.uniform(-6, 6, 200_000)).astype(np.float32)
    c = np.float32(8193.0)                                 # 2^13 + 1: 24 - 13 = 11 significant bits
    gm = (a * c).astype(np.float32)
    hi = (gm - (gm - a).astype(np.float32)).astype(np.float32)
    lo = (a - hi).astype(np.float32)
    assert _tf32_exact(hi).all()
    assert np.array_equal(hi.astype(np.float64) + lo.astype(np.float64), a.astype(np.float64))   # exact
    assert np.max(np.abs(lo / a)) <= 2.0 ** -11
    # 2^12 + 1 leaves a 12-bit head, which a TF32 operand cannot hold
    c12 = np.float32(4097.0)
    gm = (a * c12).astype(np.float32)
    hi12 = (gm - (gm - a).astype(np.float32)).astype(np.float32)
    assert not _tf32_exact(hi12).all()


def test_shift_split_of_values_in_the_unit_interval():
    rng = np.random.default_rng(4)
    a = np.concatenate([rng.uniform(-1, 1, 200_000), [-1.0, 1.0, 0.0, 2.0 ** -30]]).astype(np.float32)
    c = np.float32(6144.0)                                 # 1.5 * 2^12: rounds to a multiple of 2^-11
    hi = ((a + c).astype(np.float32) - c).astype(np.float32)
    lo = (a - hi).astype(np.float32)
    assert _tf32_exact(hi).all()
    assert np.array_equal(hi.astype(np.float64) + lo.astype(np.float64), a.astype(np.float64))
    assert np.max(np.abs(lo)) <= 2.0 ** -12
    # the tail read as TF32 (low 13 bits dropped) is within 2^-22 of it
    lo_t = (lo.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)
    assert np.max(np.abs(lo_t.astype(np.float64) - lo)) <= 2.0 ** -22
