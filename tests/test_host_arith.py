"""Arithmetic identities the kernels rely on, checked on the CPU in IEEE FP32 (numpy's float32
operations are correctly rounded, as the device's are with -prec-div / -prec-sqrt)."""
import numpy as np


def test_reciprocal_quotient_is_exact_below_2_16():
    """The voxel enumeration of the candidate kernels takes floor(i / n) as the integer part
    of (i + 0.5) * fl(1/n) in FP32, for ranges of at most 2^16 voxels.  The rounding error,
    at most (i / n) 2^-23, stays below the 0.5 / n margin.  Checked for every n up to 4096 and
    a spread of larger n, against every i < 2^16."""
    i = np.arange(65536, dtype=np.int64)
    fi = i.astype(np.float32) + np.float32(0.5)
    ns = list(range(1, 4097)) + list(range(4097, 65537, 97)) + [65535, 65536]
    for n in ns:
        inv = np.float32(1.0) / np.float32(n)
        q = (fi * inv).astype(np.int64)
        assert np.array_equal(q, i // n), n


def test_sign_of_rounded_difference_decides_the_order():
    """FP32 subtraction of finite values rounds to zero only for equal operands, so the sign
    of fl(a - b) is the sign of a - b (the per-row set and open tests of the capsule steps are
    comparisons against a budget; this is the identity their derivation uses)."""
    rng = np.random.default_rng(7)
    a = rng.standard_normal(200000).astype(np.float32) * np.float32(3.0)
    b = (a + rng.standard_normal(200000).astype(np.float32) * np.float32(1e-6)).astype(np.float32)
    d = a - b
    assert np.array_equal(d > 0, a > b) and np.array_equal(d < 0, a < b) and np.array_equal(d == 0, a == b)
