"""Pins of the CPU oracle against what geometry and the paper fix (no GPU).

Each test checks the oracle against an independent statement: a different
algorithm (golden-section distance minimisation, an LP feasibility test,
supersampled point membership), a closed form (lengths, areas, rank-1 SGGX
matrices, uniform marginals of the sphere), or an invariant the paper states
(2x2x2 aggregation, dendrogram count, symmetric distance).
"""
import math

import numpy as np
import pytest

import oracle
import synth


# ----------------------------------------------------------------------------
# independent references
# ----------------------------------------------------------------------------
def seg_box_dist64(a, b, lo, hi, iters=200):
    """Distance from segment a-b to box [lo,hi] by golden-section search on t
    (the squared distance is convex in t).  FP64, independent of the oracle."""
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    lo = np.asarray(lo, np.float64); hi = np.asarray(hi, np.float64)
    d = b - a

    def f(t):
        p = a + t * d
        e = np.maximum(np.maximum(lo - p, 0.0), p - hi)
        return float(np.dot(e, e))
    gr = (math.sqrt(5) - 1) / 2
    x0, x1 = 0.0, 1.0
    c = x1 - gr * (x1 - x0); e_ = x0 + gr * (x1 - x0)
    fc, fe = f(c), f(e_)
    for _ in range(iters):
        if fc < fe:
            x1, e_, fe = e_, c, fc
            c = x1 - gr * (x1 - x0); fc = f(c)
        else:
            x0, c, fc = c, e_, fe
            e_ = x0 + gr * (x1 - x0); fe = f(e_)
    return math.sqrt(min(f(0.0), f(1.0), fc, fe, f(0.5 * (x0 + x1))))


def tri_box_margin(v, lo, hi):
    """LP: largest delta such that a point of the triangle lies in the box shrunk
    by delta.  > 0: overlap; < 0: disjoint.  Independent of the SAT."""
    from scipy.optimize import linprog
    v = np.asarray(v, np.float64)
    # variables: alpha0..2, delta ; maximise delta
    c = np.array([0, 0, 0, -1.0])
    A_ub, b_ub = [], []
    for i in range(3):
        # lo_i + delta - sum alpha_k v_ki <= 0
        A_ub.append([-v[0, i], -v[1, i], -v[2, i], 1.0]); b_ub.append(-lo[i])
        # sum alpha_k v_ki + delta - hi_i <= 0
        A_ub.append([v[0, i], v[1, i], v[2, i], 1.0]); b_ub.append(hi[i])
    res = linprog(c, A_ub=A_ub, b_ub=b_ub, A_eq=[[1, 1, 1, 0]], b_eq=[1.0],
                  bounds=[(0, None)] * 3 + [(None, None)], method="highs")
    assert res.status == 0
    return -res.fun


def sub_bounds(sx, sy, sz):
    lo = np.array([sx, sy, sz], np.float64) / 8.0
    return lo, lo + 0.125


# ----------------------------------------------------------------------------
# Morton keys
# ----------------------------------------------------------------------------
def test_morton_closed_form():
    assert oracle.morton(1, 0, 0) == 1
    assert oracle.morton(0, 1, 0) == 2
    assert oracle.morton(0, 0, 1) == 4
    # (3,5,7): x=011, y=101, z=111 -> triples (z y x) per bit: b0=(1,1,1)=7, b1=(1,0,1)=5, b2=(1,1,0)=6
    assert oracle.morton(3, 5, 7) == 7 | (5 << 3) | (6 << 6)
    assert oracle.morton(2047, 0, 0) == sum(1 << (3 * b) for b in range(11))


# ----------------------------------------------------------------------------
# capsule-box predicate: exact distance test
# ----------------------------------------------------------------------------
def test_capsule_box_matches_exact_distance():
    rng = np.random.default_rng(11)
    checked = amb = 0
    for _ in range(3000):
        a = rng.uniform(-0.6, 1.6, 3).astype(np.float32)
        if rng.uniform() < 0.2:
            b = a + rng.uniform(-0.05, 0.05, 3).astype(np.float32)   # short segments
        else:
            b = rng.uniform(-0.6, 1.6, 3).astype(np.float32)
        if rng.uniform() < 0.1:
            k = rng.integers(0, 3); b[k] = a[k]                        # axis-parallel
        r = np.float32(rng.uniform(0.01, 0.5))
        s = rng.integers(0, 8, 3)
        lo, hi = sub_bounds(*s)
        bit = oracle.capsule_box(a, b, np.float32(r) * np.float32(r), lo.astype(np.float32),
                                 hi.astype(np.float32))
        dist = seg_box_dist64(a, b, lo, hi)
        if abs(dist - float(r)) < 1e-5:
            amb += 1
            continue
        assert bit == (1 if dist < r else 0), (a, b, r, s, dist)
        checked += 1
    assert checked > 2900


def test_capsule_mask_supersampled():
    """Every sub-cell that contains a point of the capsule is set; every set
    sub-cell is within r of the segment (golden-section distance)."""
    rng = np.random.default_rng(5)
    for _ in range(12):
        A = rng.uniform(0.2, 1.8, 3).astype(np.float32)
        B = (A + rng.uniform(-1.2, 1.2, 3)).astype(np.float32)
        rg = np.float32(rng.uniform(0.05, 0.45))
        vijk = (1, 1, 1) if rng.uniform() < 0.5 else (0, 1, 0)
        m = oracle.capsule_mask(A, B, rg, vijk)
        loc_a = A.astype(np.float64) - vijk
        loc_b = B.astype(np.float64) - vijk
        # points on a 16^3 lattice per sub-cell (including faces)
        g = (np.arange(17) / 16.0) / 8.0
        for sz in range(8):
            for sy in range(8):
                for sx in range(8):
                    bit = (int(m[sz]) >> (sx + 8 * sy)) & 1
                    lo, hi = sub_bounds(sx, sy, sz)
                    dist = seg_box_dist64(loc_a, loc_b, lo, hi, iters=80)
                    if bit:
                        assert dist <= rg + 1e-5
                    else:
                        assert dist >= rg - 1e-5
                        if dist < rg + 0.02:   # near the surface: lattice check too
                            P = np.stack(np.meshgrid(lo[0] + g, lo[1] + g, lo[2] + g,
                                                     indexing="ij"), -1).reshape(-1, 3)
                            dd = loc_b - loc_a
                            t = np.clip(((P - loc_a) @ dd) / max(dd @ dd, 1e-30), 0, 1)
                            q = loc_a + t[:, None] * dd
                            assert np.min(np.linalg.norm(P - q, axis=1)) >= rg - 1e-5


# ----------------------------------------------------------------------------
# triangle-box SAT: LP feasibility + supersampling
# ----------------------------------------------------------------------------
def test_tri_mask_matches_lp():
    pytest.importorskip("scipy")
    rng = np.random.default_rng(7)
    checked = 0
    for _ in range(6):
        c = rng.uniform(0.3, 0.7, 3)
        V = (c + rng.standard_normal((3, 3)) * rng.uniform(0.1, 0.5)).astype(np.float32)
        U = V.reshape(9)
        m = oracle.tri_mask(U, (0, 0, 0))
        for sz in range(8):
            for sy in range(8):
                for sx in range(8):
                    lo, hi = sub_bounds(sx, sy, sz)
                    bit = (int(m[sz]) >> (sx + 8 * sy)) & 1
                    d = tri_box_margin(V.astype(np.float64), lo, hi)
                    if abs(d) < 1e-6:
                        continue
                    assert bit == (1 if d > 0 else 0), (V, sx, sy, sz, d)
                    checked += 1
    assert checked > 3000


def test_tri_mask_supersampled_points_covered():
    rng = np.random.default_rng(8)
    tris, grid = synth.random_triangles(20, 8, seed=3, size=(0.3, 2.0))
    U = tris[..., :3] * 8.0
    for t in range(U.shape[0]):
        V = U[t].astype(np.float64)
        ab = rng.uniform(0, 1, (4000, 2))
        flip = ab.sum(1) > 1
        ab[flip] = 1 - ab[flip]
        P = V[0] + ab[:, :1] * (V[1] - V[0]) + ab[:, 1:] * (V[2] - V[0])
        for p in P[:400]:
            vi = np.floor(p).astype(int)
            if np.any(vi < 0) or np.any(vi >= 8):
                continue
            loc = p - vi
            s = [int(x) for x in np.minimum((loc * 8).astype(int), 7)]
            m = oracle.tri_mask(U[t].reshape(9), tuple(int(x) for x in vi))
            assert (int(m[s[2]]) >> (s[0] + 8 * s[1])) & 1


# ----------------------------------------------------------------------------
# measures: closed forms
# ----------------------------------------------------------------------------
def test_fiber_mass_equals_tube_volume():
    ctrl, off, grid = synth.random_segments(6, 30, 16, seed=1, radius=(0.1, 0.4), step=(0.2, 1.2))
    # keep inside the grid
    ctrl[:, :3] = np.clip(ctrl[:, :3], 0.05, 0.95)
    rng = np.random.default_rng(2)
    nseg = synth.fiber_segment_count(off)
    w = rng.uniform(0.5, 2.0, nseg).astype(np.float32)
    L0 = oracle.voxelize_fibers(ctrl, off, grid, weights=w)
    s = 1.0 / grid.voxel_size
    tot = 0.0
    p = 0
    for f in range(len(off) - 1):
        for c in range(off[f], off[f + 1] - 1):
            a = ctrl[c, :3].astype(np.float64) * s
            b = ctrl[c + 1, :3].astype(np.float64) * s
            r = 0.5 * (float(ctrl[c, 3]) + float(ctrl[c + 1, 3])) * s
            tot += float(w[p]) * math.pi * r * r * float(np.linalg.norm(b - a))
            p += 1
    assert L0["mass64"].sum() == pytest.approx(tot, rel=1e-12)
    assert L0["mass"].astype(np.float64).sum() == pytest.approx(tot, rel=1e-5)


def test_triangle_mass_equals_area():
    tris, grid = synth.random_triangles(40, 16, seed=9, size=(0.3, 3.0))
    tris[..., :3] = np.clip(tris[..., :3], 0.02, 0.98)
    L0 = oracle.voxelize_tris(tris, grid)
    U = tris[..., :3].astype(np.float64) * 16
    area = 0.5 * np.linalg.norm(np.cross(U[:, 1] - U[:, 0], U[:, 2] - U[:, 0]), axis=1).sum()
    assert L0["mass64"].sum() == pytest.approx(area, rel=1e-12)
    assert L0["mass"].astype(np.float64).sum() == pytest.approx(area, rel=1e-5)


def test_fp32_chain_within_tolerance_of_fp64():
    """The FP32 definition stays within the stated tolerance of the FP64 sums:
    |m32 - m64| <= 1e-5 * m64 + 1e-6 * (largest primitive measure)."""
    w = synth.config1()
    L0 = oracle.voxelize(w)
    m32 = L0["mass"].astype(np.float64); m64 = L0["mass64"]
    floor = 1e-6 * 4.0
    assert np.all(np.abs(m32 - m64) <= 1e-5 * m64 + floor)
    M32 = L0["moment"].astype(np.float64); M64 = L0["moment64"]
    tr = M64[:, :3].sum(1)
    assert np.all(np.abs(M32 - M64) <= (1e-5 * tr + floor)[:, None])


# ----------------------------------------------------------------------------
# SGGX closed forms (Sec. 4.1): planar patch -> n n^T, straight fiber -> t t^T
# ----------------------------------------------------------------------------
def test_planar_patch_gives_rank1_normal():
    n = np.array([0.3, -0.2, 1.0]); n /= np.linalg.norm(n)
    xs = np.linspace(0.1, 0.9, 9)
    X, Y = np.meshgrid(xs, xs)
    Z = 0.5 + (-(n[0] * (X - 0.5) + n[1] * (Y - 0.5)) / n[2])
    P = np.stack([X, Y, Z], -1)
    tri = []
    for i in range(8):
        for j in range(8):
            tri.append([P[i, j], P[i, j + 1], P[i + 1, j + 1]])
            tri.append([P[i, j], P[i + 1, j + 1], P[i + 1, j]])
    tri = np.asarray(tri)
    T = np.zeros((tri.shape[0], 3, 4), np.float32); T[..., :3] = tri
    grid = synth.Grid((0.0, 0.0, 0.0), 1.0 / 16, 16)
    L0 = oracle.voxelize_tris(T, grid)
    ok = L0["lobe_count"] == 1
    assert ok.sum() > 50
    S = L0["lobes"][ok, 0, :6].astype(np.float64)
    nn = np.array([n[0] ** 2, n[1] ** 2, n[2] ** 2, n[0] * n[1], n[0] * n[2], n[1] * n[2]])
    # sign of the normal is irrelevant (second moment)
    assert np.max(np.abs(S - nn[None])) < 1e-5


def test_straight_fiber_gives_rank1_tangent():
    t = np.array([1.0, 0.7, 0.4]); t /= np.linalg.norm(t)
    p0 = np.array([0.1, 0.15, 0.2])
    pts = p0[None] + np.linspace(0, 0.8, 41)[:, None] * t[None]
    ctrl = np.zeros((41, 4), np.float32); ctrl[:, :3] = pts; ctrl[:, 3] = 0.02
    off = np.array([0, 41], np.int64)
    grid = synth.Grid((0.0, 0.0, 0.0), 1.0 / 32, 32)
    L0 = oracle.voxelize_fibers(ctrl, off, grid)
    ok = L0["lobe_count"] == 1
    assert ok.sum() > 20
    S = L0["lobes"][ok, 0, :6].astype(np.float64)
    tt = np.array([t[0] ** 2, t[1] ** 2, t[2] ** 2, t[0] * t[1], t[0] * t[2], t[1] * t[2]])
    assert np.max(np.abs(S - tt[None])) < 2e-5
    # trace 1, PSD
    for s in S:
        Sm = np.array([[s[0], s[3], s[4]], [s[3], s[1], s[5]], [s[4], s[5], s[2]]])
        assert abs(np.trace(Sm) - 1) < 1e-5
        assert np.linalg.eigvalsh(Sm).min() > -1e-6


def test_compact_roundtrip():
    rng = np.random.default_rng(3)
    for _ in range(50):
        Q = rng.standard_normal((3, 3))
        S = Q @ Q.T
        S /= np.trace(S)
        s6 = np.array([S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]], np.float32)
        c = oracle.compact(s6).astype(np.float64)
        back = np.array([c[0] ** 2, c[1] ** 2, c[2] ** 2, c[3] * c[0] * c[1], c[4] * c[0] * c[2],
                         c[5] * c[1] * c[2]])
        assert np.allclose(back, s6, atol=1e-6)
        assert np.all(np.abs(c[3:]) <= 1 + 1e-6)


# ----------------------------------------------------------------------------
# occupancy invariants (Sec. 3.5)
# ----------------------------------------------------------------------------
def test_occupancy_and_projection_invariants():
    L0 = oracle.voxelize(synth.config1())
    occ = L0["occ"].astype(int); proj = L0["proj"].astype(int)
    pc = np.array([[bin(int(x)).count("1") for x in row] for row in L0["mask"][:500]]).sum(1)
    assert np.array_equal(pc, occ[:500])
    assert np.all(occ >= 1)
    assert np.all(proj <= 64)
    assert np.all(proj.max(1) <= occ)
    assert np.all(occ <= 8 * proj.min(1))


# ----------------------------------------------------------------------------
# LoD (Sec. 4.2-4.3): 2x2x2 aggregation equals direct coarse evaluation
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["fibers", "triangles"])
def test_lod_masks_equal_direct_coarse_voxelization(kind, dirs5000):
    R = 16
    if kind == "fibers":
        ctrl, off, grid = synth.random_segments(5, 25, R, seed=4, radius=(0.1, 0.5))
        L0 = oracle.voxelize_fibers(ctrl, off, grid)
    else:
        tris, grid = synth.random_triangles(30, R, seed=5)
        L0 = oracle.voxelize_tris(tris, grid)
    pyr = oracle.build_pyramid(L0, R, 1, dirs5000)
    assert len(pyr) == 4
    for lvl, L in enumerate(pyr, start=1):
        g2 = synth.Grid(grid.origin, grid.voxel_size * 2 ** lvl, R >> lvl)
        if kind == "fibers":
            D = oracle.voxelize_fibers(ctrl, off, g2)
            scale = 8.0 ** lvl
        else:
            D = oracle.voxelize_tris(tris, g2)
            scale = 4.0 ** lvl
        assert np.array_equal(L["keys"], D["keys"])
        assert np.array_equal(L["mask"], D["mask"])
        assert np.array_equal(L["occ"], D["occ"])
        assert np.array_equal(L["proj"], D["proj"])
        assert np.allclose(L["mass64"], D["mass64"] * scale, rtol=1e-9, atol=1e-12)
        assert np.allclose(L["moment64"], D["moment64"] * scale, rtol=1e-9, atol=1e-9)


def test_lod_conservation_and_parents(dirs5000):
    L0 = oracle.voxelize(synth.config1())
    pyr = oracle.build_pyramid(L0, 128, 1, dirs5000)
    assert len(pyr) == 7
    assert pyr[-1]["keys"].shape[0] == 1 and pyr[-1]["keys"][0] == 0
    prev = L0
    for L in pyr:
        assert L["mass64"].sum() == pytest.approx(L0["mass64"].sum(), rel=1e-12)
        assert np.allclose(L["moment64"].sum(0), L0["moment64"].sum(0), rtol=1e-12, atol=1e-9)
        assert np.array_equal(np.unique(prev["keys"] >> np.uint64(3)), L["keys"])
        prev = L


# ----------------------------------------------------------------------------
# SGGX-H (Sec. 4.4)
# ----------------------------------------------------------------------------
def test_sqrtm_matches_eigh():
    rng = np.random.default_rng(4)
    for _ in range(200):
        Q = rng.standard_normal((3, 3))
        lam = rng.uniform(0, 1, 3) ** 4
        V, _ = np.linalg.qr(Q)
        S = V @ np.diag(lam) @ V.T
        S /= np.trace(S)
        S += 1e-6 * np.eye(3)
        s6 = np.array([S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]], np.float32)
        R = oracle.sqrtm3(s6).astype(np.float64)
        S64 = np.array([[s6[0], s6[3], s6[4]], [s6[3], s6[1], s6[5]], [s6[4], s6[5], s6[2]]], np.float64)
        w, U = np.linalg.eigh(S64)
        Rref = U @ np.diag(np.sqrt(np.maximum(w, 0))) @ U.T
        assert np.max(np.abs(R - Rref)) < 2e-5
        assert np.max(np.abs(R - R.T)) < 1e-6


def test_isotropic_lobe_histogram_is_uniform_marginal(dirs5000):
    """Uniform directions on the sphere have uniform coordinate marginals on [-1,1]
    (Archimedes), so P(|w_a| >= 0.6) = 0.4 and P(|w_a| >= 0.2) = 0.8."""
    S = np.array([1 / 3, 1 / 3, 1 / 3, 0, 0, 0], np.float32)
    h, M = oracle.sample_lobe(S, dirs5000)
    N = 5000
    assert np.all(np.abs(h[:3] / N - 0.4) < 0.01)
    assert np.all(np.abs(h[3:] / N - 0.8) < 0.01)
    assert np.allclose(M, [1 / 3, 1 / 3, 1 / 3, 0, 0, 0], atol=2e-3)


def test_rank1_lobe_concentrates(dirs5000):
    t = np.array([0.8, 0.5, 0.33]); t /= np.linalg.norm(t)
    S = np.array([t[0] ** 2, t[1] ** 2, t[2] ** 2, t[0] * t[1], t[0] * t[2], t[1] * t[2]], np.float32)
    h, M = oracle.sample_lobe(S, dirs5000)
    N = 5000
    exp_o = [N if abs(x) >= 0.6 else 0 for x in t]
    exp_mo = [N if abs(x) >= 0.2 else 0 for x in t]
    # S' = S + 1e-6 tr(S) I: directions with |t.u| below ~1e-3 (a few per thousand of
    # a uniform set) are not pulled onto +-t.
    assert np.all(np.abs(h[:3] - exp_o) <= 0.005 * N)
    assert np.all(np.abs(h[3:] - exp_mo) <= 0.005 * N)
    assert np.allclose(M, S, atol=5e-3)


def test_hist_distance_properties(dirs5000):
    rng = np.random.default_rng(6)
    H = []
    for _ in range(8):
        Q = rng.standard_normal((3, 3)); S = Q @ Q.T; S /= np.trace(S)
        s6 = np.array([S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]], np.float32)
        H.append(oracle.sample_lobe(s6, dirs5000)[0])
    for i in range(8):
        assert oracle.hist_dist(H[i], H[i]) == 0
        for j in range(8):
            assert oracle.hist_dist(H[i], H[j]) == oracle.hist_dist(H[j], H[i]) >= 0
            for k in range(8):
                assert oracle.hist_dist(H[i], H[k]) <= oracle.hist_dist(H[i], H[j]) + oracle.hist_dist(H[j], H[k])


def _s6(v):
    v = np.asarray(v, np.float64); v /= np.linalg.norm(v)
    return [v[0] ** 2, v[1] ** 2, v[2] ** 2, v[0] * v[1], v[0] * v[2], v[1] * v[2]]


def test_sggx_h_count_and_weights(dirs5000):
    """D_{L-1} = D_L minus {S_i, S_j} plus S_n: one lobe fewer per merge, weights add."""
    rng = np.random.default_rng(8)
    groups = [[1, 0.05, 0], [0, 1, 0.05], [0.05, 0, 1]]
    cand, gw = [], [0.0, 0.0, 0.0]
    for gi, g in enumerate(groups):
        for _ in range(3):
            v = np.asarray(g) + 0.02 * rng.standard_normal(3)
            w = float(rng.uniform(0.5, 2))
            cand.append(_s6(v) + [w]); gw[gi] += np.float32(w)
    cand = np.asarray(cand, np.float32)
    for K in (1, 2, 3, 5, 9, 12):
        out, merges = oracle.sggx_h(cand, K, dirs5000)
        assert out.shape[0] == min(K, 9)
        assert len(merges) == 9 - out.shape[0]
        assert out[:, 6].sum() == pytest.approx(cand[:, 6].sum(), rel=1e-6)
        assert np.all(np.diff(out[:, 6]) <= 0)
    out, _ = oracle.sggx_h(cand, 3, dirs5000)
    # the three groups survive: weights and principal directions
    assert sorted(out[:, 6]) == pytest.approx(sorted(gw), rel=1e-6)
    for o in out:
        S = np.array([[o[0], o[3], o[4]], [o[3], o[1], o[5]], [o[4], o[5], o[2]]])
        ev = np.linalg.eigh(S)[1][:, -1]
        assert max(abs(ev @ (np.asarray(g) / np.linalg.norm(g))) for g in groups) > 0.99
        assert np.trace(S) == pytest.approx(1.0, abs=1e-3)
        assert np.linalg.eigvalsh(S).min() > -1e-6


def test_sggx_h_tie_break_and_identical_merge(dirs5000):
    s = _s6([0.2, 0.9, 0.3])
    cand = np.asarray([s + [1.0]] * 4, np.float32)
    out, merges = oracle.sggx_h(cand, 3, dirs5000)
    assert merges == [(1, 0)]
    # merging a lobe with itself keeps its sample second moment
    _, M = oracle.sample_lobe(np.asarray(s, np.float32), dirs5000)
    merged = [o for o in out if o[6] == 2.0][0]
    assert np.allclose(merged[:6], M, atol=1e-7)


def test_sggx_h_copies_when_few(dirs5000):
    cand = np.asarray([_s6([1, 0, 0]) + [0.5], _s6([0, 1, 0]) + [2.0]], np.float32)
    out, merges = oracle.sggx_h(cand, 4, dirs5000)
    assert merges == []
    assert np.allclose(out[0], cand[1]) and np.allclose(out[1], cand[0])


# ----------------------------------------------------------------------------
# 8-bit compact SGGX (Sec. 4.3): closed-form byte values and the round-trip bound
# ----------------------------------------------------------------------------
def test_compact8_closed_form_values():
    c = np.array([[0.0, 1.0, 0.5, -1.0, 1.0, 0.0],              # 0.5 * 255 = 127.5 -> 128 (even)
                  [1.0 / 255, 2.0 / 255, 0.999, -0.5, 0.5, 1.0 / 127.5 - 1.0],
                  [1.2, -0.1, 0.25, -1.3, 1.3, 0.3]], np.float32)  # clamped
    q = oracle.compact8(c)
    assert q.dtype == np.uint8
    assert q[0].tolist() == [0, 255, 128, 0, 255, 128]            # 127.5 r + 127.5 at r = 0: 127.5 -> 128
    assert q[1].tolist() == [1, 2, 255, 64, 191, 1]               # 63.75 -> 64, 191.25 -> 191
    assert q[2].tolist() == [255, 0, 64, 0, 255, 166]             # 63.75 -> 64, 165.75 -> 166
    # an isotropic lobe S = I/3: sigma = sqrt(1/3) -> 147.2 -> 147, r = 0 -> 128
    iso = oracle.compact(np.array([1 / 3, 1 / 3, 1 / 3, 0, 0, 0], np.float32))
    assert oracle.compact8(iso).tolist() == [147, 147, 147, 128, 128, 128]


def test_compact8_round_trip_bound():
    rng = np.random.default_rng(12)
    c = np.concatenate([rng.uniform(0, 1, (5000, 3)), rng.uniform(-1, 1, (5000, 3))], axis=1).astype(np.float32)
    q = oracle.compact8(c).astype(np.float64)
    sig = q[:, :3] / 255.0
    r = q[:, 3:] / 127.5 - 1.0
    assert np.abs(sig - c[:, :3]).max() <= 0.5 / 255 + 1e-6
    assert np.abs(r - c[:, 3:]).max() <= 0.5 / 127.5 + 1e-6


# ----------------------------------------------------------------------------
# Catmull-Rom spline fibers (Sec. 3.2): independent FP64 matrix form, linear precision
# ----------------------------------------------------------------------------
CR_BASIS = 0.5 * np.array([[0, 2, 0, 0], [-1, 0, 1, 0], [2, -5, 4, -1], [-1, 3, -3, 1]], np.float64)


def cr_reference(nodes, S):
    """FP64 reference: [1 t t^2 t^3] M [P0 P1 P2 P3]^T with reflected end nodes."""
    P = nodes[:, :3].astype(np.float64)
    n = P.shape[0]
    ext = np.concatenate([2 * P[:1] - P[1:2], P, 2 * P[-1:] - P[-2:-1]]) if n > 1 else P
    pts = []
    for i in range(n - 1):
        G = ext[i: i + 4]
        for j in range(S):
            t = j / S
            pts.append(np.array([1, t, t * t, t ** 3]) @ CR_BASIS @ G)
    pts.append(P[-1])
    return np.array(pts)


def test_catmull_rom_matches_matrix_form():
    rng = np.random.default_rng(21)
    sizes = [2, 3, 7, 1, 12]
    nodes = np.concatenate([np.concatenate([rng.uniform(0, 4, (k, 3)), rng.uniform(0.1, 0.5, (k, 1))], 1)
                            for k in sizes]).astype(np.float32)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    S = 6
    ctrl, out_off = oracle.catmull_rom(nodes, off, S)
    assert out_off.tolist() == [int((off[f] - f) * S + f) for f in range(len(sizes) + 1)]
    for f, k in enumerate(sizes):
        got = ctrl[out_off[f]: out_off[f + 1]]
        assert got.shape[0] == (k - 1) * S + 1
        ref = cr_reference(nodes[off[f]: off[f + 1]], S)
        np.testing.assert_allclose(got[:, :3], ref, rtol=0, atol=1e-5)
        # nodes are passed exactly (t = 0 of each span, and the closing node)
        assert np.array_equal(got[::S, :3], nodes[off[f]: off[f + 1], :3])
        # radius: linear between consecutive nodes
        r = nodes[off[f]: off[f + 1], 3].astype(np.float64)
        if k > 1:
            t = (np.arange((k - 1) * S) % S) / S
            i = np.arange((k - 1) * S) // S
            np.testing.assert_allclose(got[:-1, 3], r[i] + t * (r[i + 1] - r[i]), rtol=1e-6)


def test_catmull_rom_linear_precision():
    # equally spaced nodes on a line: every sample is on the line at its uniform parameter
    a = np.array([0.3, -1.2, 2.0]); d = np.array([0.7, 0.2, -0.4])
    k, S = 9, 5
    nodes = np.concatenate([a + np.arange(k)[:, None] * d, np.full((k, 1), 0.25)], 1).astype(np.float32)
    ctrl, _ = oracle.catmull_rom(nodes, np.array([0, k]), S)
    u = np.arange((k - 1) * S + 1) / S
    np.testing.assert_allclose(ctrl[:, :3], a + u[:, None] * d, rtol=0, atol=2e-6)


# ----------------------------------------------------------------------------
# SGGX-H merge rules (C12 and the mass-weighted option)
# ----------------------------------------------------------------------------
def test_sggx_h_merge_rules_two_lobes():
    """Two lobes merged into one: the pooled rule gives (M^_1 + M^_2) / 2, the mass-weighted
    rule (w_1 M^_1 + w_2 M^_2) / (w_1 + w_2), with M^ each lobe's own sample moment."""
    dirs = synth.sample_directions(5000)
    S1 = np.array([0.8, 0.15, 0.05, 0.1, 0.0, 0.02], np.float32)
    S2 = np.array([0.1, 0.2, 0.7, 0.0, -0.05, 0.1], np.float32)
    w1, w2 = 3.0, 0.5
    cand = np.array([list(S1) + [w1], list(S2) + [w2]], np.float32)
    _, M1 = oracle.sample_lobe(S1, dirs)
    _, M2 = oracle.sample_lobe(S2, dirs)
    pooled, _ = oracle.sggx_h(cand, 1, dirs, merge=0)
    mass, _ = oracle.sggx_h(cand, 1, dirs, merge=1)
    np.testing.assert_allclose(pooled[0, :6], (M1.astype(np.float64) + M2) / 2, rtol=0, atol=1e-7)
    np.testing.assert_allclose(mass[0, :6], (w1 * M1.astype(np.float64) + w2 * M2) / (w1 + w2), rtol=0, atol=1e-6)
    assert pooled[0, 6] == mass[0, 6] == np.float32(w1 + w2)
    # the mass-weighted lobe leans towards the heavier lobe
    assert abs(mass[0, 0] - M1[0]) < abs(pooled[0, 0] - M1[0])


# ----------------------------------------------------------------------------
# Sample-based voxelization (Sec. 3.2-3.3, comparison workload)
# ----------------------------------------------------------------------------
def test_sampled_fibers_closed_form_and_subset_of_exact():
    grid = synth.Grid((0.0, 0.0, 0.0), 1.0 / 8, 8)
    # a segment along x through voxel centres (y = z = 0.5 voxel), 4 voxels long, 16 samples:
    # 4 samples per voxel at x = 1/8, 3/8, 5/8, 7/8 -> sub-cells sx = 1, 3, 5, 7 of row (4, 4)
    r = 0.01
    ctrl = np.array([[0.0, 0.5 / 8, 0.5 / 8, r], [4.0 / 8, 0.5 / 8, 0.5 / 8, r]], np.float32)
    L = oracle.voxelize_fibers_sampled(ctrl, np.array([0, 2]), grid, 16)
    assert L["keys"].tolist() == [oracle.morton(i, 0, 0) for i in range(4)]
    assert L["occ"].tolist() == [4, 4, 4, 4]
    row = sum(1 << (sx + 8 * 4) for sx in (1, 3, 5, 7))
    assert all(int(m[4]) == row and int(m[:4].sum()) == 0 for m in L["mask"])
    mu = np.pi * (r * 8) ** 2 * 4.0
    np.testing.assert_allclose(L["mass"], mu / 4, rtol=1e-6)
    np.testing.assert_allclose(L["moment"][:, 0], mu / 4, rtol=1e-6)        # t = x: only xx
    assert np.abs(L["moment"][:, 1:]).max() == 0.0
    # random fibers: the mass of the samples inside the grid, and every sampled sub-cell is one
    # the exact capsule test sets (a sample lies on the axis, inside the capsule)
    ctrl, off, grid = synth.random_segments(6, 12, 16, seed=4, radius=(0.2, 1.0), step=(0.3, 2.0))
    S = 6
    Ls = oracle.voxelize_fibers_sampled(ctrl, off, grid, S)
    Le = oracle.voxelize(synth.Workload("e", "fibers", grid, ctrl=ctrl, fiber_offsets=off))
    idx = {int(k): i for i, k in enumerate(Le["keys"])}
    for k, m in zip(Ls["keys"], Ls["mask"]):
        e = Le["mask"][idx[int(k)]]
        assert np.all((m & ~e) == 0)
    assert Ls["occ"].sum() < Le["occ"].sum()


def test_sampled_triangles_counts_mass_and_subset():
    grid = synth.Grid((0.0, 0.0, 0.0), 1.0, 16)
    # two right triangles in the plane z = 2.5: legs 4 (area 8) and legs 2.19 (area ~2.4, 0.3 of
    # the largest), far apart; S = 10 -> 10 and ceil(3.0) = 3 samples
    big = np.array([[1.0, 1.0, 2.5, 0], [5.0, 1.0, 2.5, 0], [1.0, 5.0, 2.5, 0]], np.float32)
    leg = np.float32(np.sqrt(2 * 8 * 0.3))
    small = np.array([[9.0, 9.0, 2.5, 0], [9.0 + leg, 9.0, 2.5, 0], [9.0, 9.0 + leg, 2.5, 0]], np.float32)
    tris = np.stack([big, small])
    L = oracle.voxelize_tris_sampled(tris, grid, 10)
    keys = L["keys"]
    def x_of(k):   # x bits of a Morton key (bit 0 of every triple)
        return sum(((int(k) >> (3 * i)) & 1) << i for i in range(21))
    x = np.array([x_of(k) for k in keys])
    small_sel = x >= 8
    assert L["occ"][small_sel].sum() <= 3 and L["occ"][~small_sel].sum() <= 10
    area_small = 0.5 * float(leg) * float(leg)
    np.testing.assert_allclose(L["mass"][small_sel].sum(), area_small, rtol=1e-5)
    np.testing.assert_allclose(L["mass"][~small_sel].sum(), 8.0, rtol=1e-6)
    # the normal moment: plane z = const -> only zz
    np.testing.assert_allclose(L["moment"][:, 2], L["mass"], rtol=1e-6)
    assert np.abs(L["moment"][:, [0, 1, 3, 4, 5]]).max() == 0.0
    # every sampled sub-cell is one the exact test sets (the sample lies on the triangle)
    tris, grid = synth.random_triangles(60, 16, seed=2, size=(0.5, 4.0))
    Ls = oracle.voxelize_tris_sampled(tris, grid, 24)
    Le = oracle.voxelize(synth.Workload("t", "triangles", grid, tri_verts=tris))
    pos = np.searchsorted(Le["keys"], Ls["keys"])
    assert np.array_equal(Le["keys"][pos], Ls["keys"])
    assert np.all((Ls["mask"] & ~Le["mask"][pos]) == 0)


def test_vdb_leaves_hand_made():
    # voxels (0,0,0), (1,0,0), (7,7,7) in leaf 0; (8,0,0) in leaf 1; (0,9,0) in leaf 2
    pts = [(0, 0, 0), (1, 0, 0), (7, 7, 7), (8, 0, 0), (0, 9, 0)]
    keys = np.array(sorted(oracle.morton(*p) for p in pts), np.uint64)
    lk, masks, first = oracle.vdb_leaves(keys)
    assert lk.tolist() == [0, 1, 2]              # Morton keys of leaves (0,0,0), (1,0,0), (0,1,0)
    assert first.tolist() == [0, 3, 4, 5]
    assert int(masks[0, 0]) == 1 | (1 << 0) and int(masks[0, 1]) == (1 << 0)   # x=1 -> bit 64
    assert int(masks[0, 7]) == 1 << 63                                       # (7,7,7) -> bit 511
    assert int(masks[1, 0]) == 1 and int(masks[2, 0]) == 1 << 8              # (0,9,0) -> y & 7 = 1
    assert oracle.demorton(oracle.morton(5, 3, 6)) == (5, 3, 6)


# ----------------------------------------------------------------------------
# SGGX-H statistics against a literal FP64 restatement (Sec. 4.4, Eq. similarity)
# ----------------------------------------------------------------------------
def _fp64_lobe_directions(s6, dirs):
    """omega_k = normalize(S'^(1/2) u_k) in FP64 with numpy's eigh, S' = S + 1e-6 tr(S) I
    (the regularised lobe, its diagonal formed in FP32 as the method forms it)."""
    s6 = np.asarray(s6, np.float32)
    tr = np.float32(np.float32(s6[0] + s6[1]) + s6[2])
    eps = np.float32(1e-6) * tr
    S = np.array([[s6[0] + eps, s6[3], s6[4]], [s6[3], s6[1] + eps, s6[5]], [s6[4], s6[5], s6[2] + eps]],
                 np.float32).astype(np.float64)
    w, U = np.linalg.eigh(S)
    R = U @ np.diag(np.sqrt(np.maximum(w, 0.0))) @ U.T
    v = np.asarray(dirs, np.float64) @ R.T
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _literal_histogram(om):
    """The 5 x 5 x 5 histogram over [-1, 1]^3 of the 2N entries omega and -omega, bin
    min(4, floor((c + 1) * 2.5)) per axis, normalised to 1."""
    pts = np.concatenate([om, -om])
    b = np.minimum(4, np.floor((pts + 1.0) * 2.5).astype(np.int64))
    H = np.zeros((5, 5, 5))
    np.add.at(H, (b[:, 0], b[:, 1], b[:, 2]), 1.0)
    return H / pts.shape[0]


def _sliced_w1(Ha, Hb):
    """Sum over the three axes of the Wasserstein-1 distance between the axis marginals
    (bin width 0.4): sum_a sum_k |CDF_a(k) - CDF_b(k)| * 0.4."""
    d = 0.0
    for ax in range(3):
        other = tuple(i for i in range(3) if i != ax)
        ca = np.cumsum(Ha.sum(axis=other))
        cb = np.cumsum(Hb.sum(axis=other))
        d += 0.4 * np.abs(ca - cb)[:4].sum()
    return d


def _near_edges(om, tol=1e-5):
    """Samples whose |omega_a| is within tol of a bin edge (0.2 or 0.6): FP32 and FP64 may
    bin them differently."""
    c = np.abs(om)
    return ((np.abs(c - 0.6) < tol) | (np.abs(c - 0.2) < tol)).sum(axis=0)


def _random_lobes(rng, n):
    out = []
    for t in range(n):
        Q = rng.standard_normal((3, 3))
        lam = rng.uniform(0, 1, 3) ** (1 + 3 * (t % 3))     # isotropic to nearly rank 1
        V, _ = np.linalg.qr(Q)
        S = V @ np.diag(lam) @ V.T
        S /= np.trace(S)
        out.append(np.array([S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]], np.float32))
    return out


def test_sample_lobe_matches_fp64_directions(dirs5000):
    """The oracle's histogram counts and sample second moment against directions computed in
    FP64 with numpy's eigh: counts exact (up to samples within 1e-5 of a bin edge), M^ within
    1e-6 (measured worst case 5.6e-7, for nearly rank-1 lobes)."""
    rng = np.random.default_rng(11)
    for s6 in _random_lobes(rng, 15):
        h, M = oracle.sample_lobe(s6, dirs5000)
        om = _fp64_lobe_directions(s6, dirs5000)
        c = np.abs(om)
        near = _near_edges(om)
        assert np.all(np.abs(h[:3] - (c >= 0.6).sum(axis=0)) <= near)
        assert np.all(np.abs(h[3:] - (c >= 0.2).sum(axis=0)) <= near)
        Mref = np.array([np.mean(om[:, a] * om[:, b]) for a, b in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))])
        assert np.max(np.abs(M - Mref)) <= 1e-6


def test_hist_dist_equals_sliced_wasserstein_of_literal_histogram(dirs5000):
    """The oracle stores a lobe's 5^3 histogram as six counts and its distance as an integer
    sum of count differences, in units of 0.4 / N.  Against the literal statement (the
    125-bin histogram of omega and -omega, the Wasserstein-1 distance of each axis marginal,
    summed over the axes) the two agree up to samples within 1e-5 of a bin edge.  A wrong
    edge, a wrong weight on the middle band or a dropped factor for the +-omega doubling
    moves the distance by far more than that tolerance (asserted below)."""
    rng = np.random.default_rng(12)
    lobes = _random_lobes(rng, 10)
    N = dirs5000.shape[0]
    oms = [_fp64_lobe_directions(s6, dirs5000) for s6 in lobes]
    Hs = [_literal_histogram(om) for om in oms]
    hs = [oracle.sample_lobe(s6, dirs5000)[0] for s6 in lobes]
    for H in Hs:
        # the symmetric histogram: each marginal is mirror-symmetric
        for ax in range(3):
            m = H.sum(axis=tuple(i for i in range(3) if i != ax))
            assert np.allclose(m, m[::-1], atol=1e-12)
    checked = 0
    for i in range(len(lobes)):
        for j in range(len(lobes)):
            lit = _sliced_w1(Hs[i], Hs[j])
            orc = oracle.hist_dist(hs[i], hs[j]) * 0.4 / N
            tol = 0.4 / N * (int(_near_edges(oms[i]).sum()) + int(_near_edges(oms[j]).sum())) * 2 + 1e-12
            assert abs(lit - orc) <= tol, (i, j, lit, orc)
            if i != j:
                assert lit > 50 * tol   # the pin can see a factor of 2 or a moved edge
                checked += 1
    assert checked == 90
