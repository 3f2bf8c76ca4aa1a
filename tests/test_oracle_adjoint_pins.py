"""Pins of the oracle's adjoints (no GPU).

The fiber adjoint is an analytic derivative of the clipped-length measure, the
triangle adjoint a complex-step derivative of the clipped area; both are checked
against what is fixed independently of them:
  - closed forms: with a uniform mass adjoint the per-voxel measures of a primitive
    lying inside the grid sum to its whole measure (pi r^2 |B - A| for a capsule axis,
    the triangle's area), so the gradient summed over voxels is the gradient of that
    whole measure; with a uniform moment adjoint the normal / tangent term has the
    closed form d (n^T G n) for the unit normal / tangent;
  - FP64 central finite differences of the oracle's own loss on stencils whose clip
    structure does not change;
  - the weight derivative is the per-primitive loss divided by its weight.
"""
import numpy as np
import pytest

import oracle
import synth


def all_keys(R):
    return np.array(sorted(oracle.morton(x, y, z) for x in range(R) for y in range(R) for z in range(R)), np.uint64)


def tri_area_grad(U):
    """d area / d U_k of one triangle (closed form): 0.5 * (U_k+1 - U_k+2) x n."""
    n = np.cross(U[1] - U[0], U[2] - U[0])
    J = np.linalg.norm(n)
    nh = n / J
    g = np.zeros((3, 3))
    for k in range(3):
        a, b = U[(k + 1) % 3], U[(k + 2) % 3]
        g[k] = 0.5 * np.cross(a - b, nh)
    return 0.5 * J, g


# ----------------------------------------------------------------------------
# triangles
# ----------------------------------------------------------------------------
def test_tri_adjoint_single_voxel_closed_form():
    R = 4
    grid = synth.Grid((0.0, 0.0, 0.0), 1.0 / R, R)
    U = np.array([[1.1, 1.1, 1.5], [1.6, 1.1, 1.5], [1.1, 1.6, 1.5]])   # inside voxel (1,1,1)
    tris = (U / R)[None]
    keys = all_keys(R)
    gm = np.ones(keys.shape[0])
    gM = np.zeros((keys.shape[0], 6))
    loss, d_t, d_w = oracle.tri_adjoint(tris, grid, keys, gm, gM, weights=np.array([2.0]))
    assert loss == pytest.approx(2.0 * 0.125, rel=1e-14)
    assert d_w[0] == pytest.approx(0.125, rel=1e-14)
    # moving U1 along +x lengthens the base: d area / d x1 = height / 2 = 0.25 (grid), x R (world)
    assert d_t[0, 1] == pytest.approx([2.0 * 0.25 * R, 0.0, 0.0], abs=1e-12)
    assert d_t[0, 2] == pytest.approx([0.0, 2.0 * 0.25 * R, 0.0], abs=1e-12)
    assert d_t[0, 0] == pytest.approx([-2.0 * 0.25 * R, -2.0 * 0.25 * R, 0.0], abs=1e-12)


def test_tri_adjoint_sum_over_voxels_is_area_gradient():
    """Clipped areas over all voxels sum to the area: the boundary terms of the clip
    planes cancel between neighbouring voxels, leaving the whole-triangle gradient."""
    R = 8
    grid = synth.Grid((0.0, 0.0, 0.0), 1.0 / R, R)
    rng = np.random.default_rng(3)
    keys = all_keys(R)
    for _ in range(6):
        U = rng.uniform(0.6, R - 0.6, size=(3, 3))
        tris = (U / R)[None]
        w = rng.uniform(0.5, 2.0)
        loss, d_t, d_w = oracle.tri_adjoint(tris, grid, keys, np.ones(keys.shape[0]), np.zeros((keys.shape[0], 6)),
                                            weights=np.array([w]))
        area, g = tri_area_grad(U)
        assert loss == pytest.approx(w * area, rel=1e-12)
        assert d_w[0] == pytest.approx(area, rel=1e-12)
        np.testing.assert_allclose(d_t[0], w * g * R, rtol=1e-9, atol=1e-9 * np.abs(g).max() * R)


def test_tri_adjoint_normal_term_closed_form():
    """Uniform moment adjoint B: the clipped pieces sum to area * n^T B n of the whole
    triangle, whose gradient is taken here by central differences of that closed form
    (no clipping involved)."""
    R = 8
    grid = synth.Grid((0.0, 0.0, 0.0), 1.0 / R, R)
    rng = np.random.default_rng(4)
    keys = all_keys(R)
    for _ in range(4):
        U = rng.uniform(0.6, R - 0.6, size=(3, 3))
        b = rng.uniform(-1, 1, 6)
        B = np.array([[b[0], b[3] / 2, b[4] / 2], [b[3] / 2, b[1], b[5] / 2], [b[4] / 2, b[5] / 2, b[2]]])
        gM = np.tile(b, (keys.shape[0], 1))
        loss, d_t, _ = oracle.tri_adjoint((U / R)[None], grid, keys, np.zeros(keys.shape[0]), gM)
        # reference by FP64 central differences of the closed-form total (no clipping involved)
        def total(V):
            n = np.cross(V[1] - V[0], V[2] - V[0])
            J = np.linalg.norm(n)
            nh = n / J
            return 0.5 * J * (nh @ B @ nh)
        assert loss == pytest.approx(total(U), rel=1e-12)
        ref = np.zeros((3, 3))
        for k in range(3):
            for i in range(3):
                e = np.zeros((3, 3)); e[k, i] = 1e-6
                ref[k, i] = (total(U + e) - total(U - e)) / 2e-6
        np.testing.assert_allclose(d_t[0], ref * R, rtol=1e-6, atol=1e-7 * R)


def test_tri_adjoint_finite_differences_random_weights():
    """Random per-voxel adjoints: complex-step gradient against FP64 central FD of the
    oracle's loss, on stencils whose clip structure is unchanged."""
    R = 8
    grid = synth.Grid((0.0, 0.0, 0.0), 1.0 / R, R)
    rng = np.random.default_rng(5)
    tris, _ = synth.random_triangles(12, R, seed=6, size=(0.5, 2.5))
    t64 = tris[..., :3].astype(np.float64)
    keys = all_keys(R)
    gm = rng.uniform(-1, 1, keys.shape[0])
    gM = rng.uniform(-1, 1, (keys.shape[0], 6))
    w = rng.uniform(0.5, 2.0, t64.shape[0])
    _, d_t, _ = oracle.tri_adjoint(t64, grid, keys, gm, gM, weights=w)
    h = 1e-6 / R
    checked = 0
    for p in range(t64.shape[0]):
        for k in range(3):
            for i in range(3):
                sig = set()
                for st in (-h, 0.0, h):
                    tt = t64.copy(); tt[p, k, i] += st
                    sig.add(oracle.tri_clip_signature(tt, grid, [p]))
                if len(sig) != 1:
                    continue
                tp = t64.copy(); tp[p, k, i] += h
                tm = t64.copy(); tm[p, k, i] -= h
                fp = oracle.tri_adjoint(tp, grid, keys, gm, gM, weights=w, prims=[p])[0]
                fm = oracle.tri_adjoint(tm, grid, keys, gm, gM, weights=w, prims=[p])[0]
                fd = (fp - fm) / (2 * h)
                assert abs(fd - d_t[p, k, i]) <= 1e-6 * max(abs(fd), 1.0), (p, k, i, fd, d_t[p, k, i])
                checked += 1
    assert checked >= 90


def test_tri_clip_signature_detects_plane_crossing():
    R = 4
    grid = synth.Grid((0.0, 0.0, 0.0), 1.0 / R, R)
    U = np.array([[1.1, 1.1, 1.5], [1.6, 1.1, 1.5], [1.1, 1.6, 1.5]])
    s0 = oracle.tri_clip_signature((U / R)[None], grid, [0])
    V = U.copy(); V[1, 0] = 2.3                       # vertex crosses the x = 2 plane
    assert oracle.tri_clip_signature((V / R)[None], grid, [0]) != s0
    V = U.copy(); V[1, 0] = 1.7                       # still inside
    assert oracle.tri_clip_signature((V / R)[None], grid, [0]) == s0


# ----------------------------------------------------------------------------
# fibers
# ----------------------------------------------------------------------------
def test_fiber_adjoint_sum_over_voxels_is_tube_gradient():
    """Uniform mass adjoint: sum of clipped lengths = |B - A|, so d loss / d A = -w pi r^2 t,
    d/dB = +w pi r^2 t, d/dr = 2 w pi r |B - A| (radius shared half-and-half by the two
    control points)."""
    R = 8
    grid = synth.Grid((0.0, 0.0, 0.0), 1.0 / R, R)
    rng = np.random.default_rng(7)
    keys = all_keys(R)
    for _ in range(6):
        A = rng.uniform(0.6, R - 0.6, 3)
        B = rng.uniform(0.6, R - 0.6, 3)
        r = rng.uniform(0.1, 0.6)
        ctrl = np.zeros((2, 4))
        ctrl[0, :3], ctrl[1, :3] = A / R, B / R
        ctrl[:, 3] = r / R
        w = rng.uniform(0.5, 2.0)
        loss, d_c, d_w = oracle.fiber_adjoint(ctrl, np.array([0, 2]), grid, keys, np.ones(keys.shape[0]),
                                              np.zeros((keys.shape[0], 6)), weights=np.array([w]))
        L = np.linalg.norm(B - A)
        t = (B - A) / L
        assert loss == pytest.approx(w * np.pi * r * r * L, rel=1e-12)
        assert d_w[0] == pytest.approx(np.pi * r * r * L, rel=1e-12)
        np.testing.assert_allclose(d_c[0, :3], -w * np.pi * r * r * t * R, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(d_c[1, :3], w * np.pi * r * r * t * R, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(d_c[:, 3], [w * np.pi * r * L * R] * 2, rtol=1e-9)


def test_fiber_adjoint_finite_differences_random_weights():
    R = 8
    grid = synth.Grid((0.0, 0.0, 0.0), 1.0 / R, R)
    rng = np.random.default_rng(8)
    ctrl, off, _ = synth.random_segments(3, 5, R, seed=9, radius=(0.1, 0.5), step=(0.5, 2.0))
    c64 = ctrl.astype(np.float64)
    keys = all_keys(R)
    gm = rng.uniform(-1, 1, keys.shape[0])
    gM = rng.uniform(-1, 1, (keys.shape[0], 6))
    _, d_c, _ = oracle.fiber_adjoint(c64, off, grid, keys, gm, gM)
    h = 1e-6 / R
    checked = 0
    nseg_before = lambda c: c - int(np.searchsorted(off, c, side="right") - 1)   # noqa: E731
    for c in range(c64.shape[0]):
        f = int(np.searchsorted(off, c, side="right") - 1)
        prims = ([nseg_before(c) - 1] if c > off[f] else []) + ([nseg_before(c)] if c + 1 < off[f + 1] else [])
        if not prims:
            continue
        for comp in range(4):
            sig = set()
            for st in (-h, 0.0, h):
                cc = c64.copy(); cc[c, comp] += st
                sig.add(oracle.clip_signature(cc, off, grid, prims))
            if len(sig) != 1:
                continue
            cp = c64.copy(); cp[c, comp] += h
            cm = c64.copy(); cm[c, comp] -= h
            fp = oracle.fiber_adjoint(cp, off, grid, keys, gm, gM, prims=np.array(prims))[0]
            fm = oracle.fiber_adjoint(cm, off, grid, keys, gm, gM, prims=np.array(prims))[0]
            fd = (fp - fm) / (2 * h)
            assert abs(fd - d_c[c, comp]) <= 1e-6 * max(abs(fd), 1.0), (c, comp, fd, d_c[c, comp])
            checked += 1
    assert checked >= 40
