"""The reduce kernel drops a step-3 task when the sub-cell is separated from the capsule by
more than r + eta (a lower bound of their distance along one direction, with a margin for
the FP32 rounding of the bound and of the exact minimum).  Here the bound is restated in
numpy FP32 (one rounding per operation, as the kernels are built without contraction) and
checked against the oracle's capsule predicate on capsules grazing sub-cells: a dropped
sub-cell must be one the predicate rejects.  No GPU."""
import numpy as np

import oracle

f32 = np.float32


def separated(a, b, r, cell):
    """The kernel's capsule_local + segment_box_separated for one sub-cell (FP32)."""
    a = a.astype(f32); b = b.astype(f32); r = f32(r)
    d = (b - a).astype(f32)
    dd = f32(f32(f32(d[0] * d[0]) + f32(d[1] * d[1])) + f32(d[2] * d[2]))
    idd = f32(f32(1.0) / dd) if dd > 0 else f32(0.0)
    M = f32(max(np.abs(a).max(), np.abs(b).max(), 0.0))
    eta = f32(f32(2e-5) * f32(f32(M + r) + f32(3.0)))
    re = f32(r + eta)
    c = (np.array(cell, np.float64) * 0.125 + 0.0625).astype(f32)
    A = (a - c).astype(f32); B = (b - c).astype(f32)
    tc = f32(-f32(f32(f32(A[0] * d[0]) + f32(A[1] * d[1])) + f32(A[2] * d[2])) * idd)
    tc = f32(min(max(tc, f32(0.0)), f32(1.0)))
    v = (A + (tc * d).astype(f32)).astype(f32)
    sa = f32(f32(f32(v[0] * A[0]) + f32(v[1] * A[1])) + f32(v[2] * A[2]))
    sb = f32(f32(f32(v[0] * B[0]) + f32(v[1] * B[1])) + f32(v[2] * B[2]))
    l1 = f32(f32(abs(v[0]) + abs(v[1])) + abs(v[2]))
    sep = f32(min(sa, sb) - f32(f32(0.0625) * l1))
    vv = f32(f32(f32(v[0] * v[0]) + f32(v[1] * v[1])) + f32(v[2] * v[2]))
    return bool(sep > 0 and f32(sep * sep) > f32(f32(re * re) * vv))


def seg_box_dist(a, b, lo, hi):
    def g(t):
        p = a + t * (b - a)
        e = np.maximum(np.maximum(lo - p, p - hi), 0.0)
        return float(e @ e)
    l, h = 0.0, 1.0
    for _ in range(100):
        m1, m2 = l + (h - l) / 3, h - (h - l) / 3
        if g(m1) <= g(m2):
            h = m2
        else:
            l = m1
    return np.sqrt(g(0.5 * (l + h)))


def test_dropped_subcells_are_rejected_by_the_predicate():
    rng = np.random.default_rng(31)
    dropped = kept_near = 0
    for trial in range(1500):
        d = rng.normal(size=3); d /= np.linalg.norm(d)
        L = rng.uniform(0.05, 3.0)
        m = rng.uniform(-0.5, 1.5, 3)
        a = (m - 0.5 * L * d).astype(f32).astype(np.float64)
        b = (m + 0.5 * L * d).astype(f32).astype(np.float64)
        cell = rng.integers(0, 8, 3)
        lo = cell / 8.0; hi = lo + 0.125
        D = seg_box_dist(a, b, lo, hi)
        if D < 1e-3:
            continue
        # radii around the distance: most within the bound's margin, some far outside it
        for eps in (-3e-4, -3e-5, -1e-6, 0.0, 1e-6, 3e-5, 3e-4, -0.05, 0.05):
            r = f32(D * (1.0 + eps))
            if separated(a, b, r, cell):
                dropped += 1
                bit = oracle.capsule_box(a.astype(f32), b.astype(f32), f32(r * r),
                                         lo.astype(f32), hi.astype(f32))
                assert bit == 0, (a, b, r, cell, D)
            elif abs(eps) < 1e-3:
                kept_near += 1
    assert dropped > 500 and kept_near > 5000
