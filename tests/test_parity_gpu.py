"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar: keys, sub-cell masks, occupancy, projections and lobe counts bit-exact; mass and
moments bit-exact with the oracle's FP32 chain and within the stated tolerance of its
FP64 reference; lobes (S, weight) within 1e-5 (trace-1 matrices, so absolute).
Tolerance (FP32 vs FP64 reference), with mu_max the larger of the largest voxel mass
and the largest whole-primitive measure w * pi r^2 L (fibers) or w * area (triangles):
    |m - m64| <= 1e-5 |m64| + 1e-6 mu_max          (mass)
    |M - M64| <= 1e-5 tr(M64) + 1e-6 mu_max        (moment entries)
The absolute floor covers FP32 clipping: a clip parameter carries an absolute error of a
few 2^-24 of the primitive's parameter range, so a clipped piece's measure is exact only
to ~1e-7 of the whole primitive's measure, whatever the size of the piece.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2604_13191_gb300 as vx  # noqa: E402

DEV = torch.device("cuda", 0)
LOBE_TOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    c = vx.Context(DEV)
    yield c
    c.close()


def run_gpu(ctx, w, K=None, dirs=None, num_levels=0, lod=True):
    K = w.K if K is None else K
    if w.kind == "triangles":
        L0 = ctx.voxelize(w.grid, tri_verts=torch.from_numpy(w.tri_verts).to(DEV),
                          weights=None if w.weights is None else torch.from_numpy(w.weights).to(DEV))
    else:
        L0 = ctx.voxelize(w.grid, ctrl=torch.from_numpy(w.ctrl).to(DEV),
                          fiber_offsets=torch.from_numpy(w.fiber_offsets).to(DEV),
                          weights=None if w.weights is None else torch.from_numpy(w.weights).to(DEV))
    pyr = []
    if lod:
        d = None if dirs is None else torch.from_numpy(dirs).to(DEV)
        pyr = ctx.build_lod(L0, K=K, dirs=d, num_levels=num_levels)
    torch.cuda.synchronize()
    return [L0.host()] + [p.host() for p in pyr]


def prim_measure_max(w) -> float:
    """Largest whole-primitive measure in level-0 voxel units."""
    s = 1.0 / w.grid.voxel_size
    wt = np.ones(w.num_prims) if w.weights is None else w.weights.astype(np.float64)
    if w.kind == "triangles":
        U = w.tri_verts[..., :3].astype(np.float64) * s
        mu = 0.5 * np.linalg.norm(np.cross(U[:, 1] - U[:, 0], U[:, 2] - U[:, 0]), axis=1)
    else:
        off = w.fiber_offsets
        mu = []
        for f in range(len(off) - 1):
            c = w.ctrl[off[f]: off[f + 1]].astype(np.float64)
            if c.shape[0] < 2:
                continue
            L = np.linalg.norm(np.diff(c[:, :3], axis=0), axis=1) * s
            r = 0.5 * (c[:-1, 3] + c[1:, 3]) * s
            mu.append(np.pi * r * r * L)
        mu = np.concatenate(mu) if mu else np.zeros(0)
    return float((wt[: mu.shape[0]] * mu).max()) if mu.size else 0.0


def compare_level(g, r, name="", lobes=True, mu_max=0.0):
    assert np.array_equal(g["keys"], r["keys"]), f"{name}: keys differ ({g['keys'].shape} vs {r['keys'].shape})"
    assert np.array_equal(g["mask"], r["mask"]), f"{name}: masks differ"
    assert np.array_equal(g["occ"], r["occ"]), f"{name}: occ differs"
    assert np.array_equal(g["proj"], r["proj"]), f"{name}: projections differ"
    m64, M64 = r["mass64"], r["moment64"]
    if m64.size:
        floor = 1e-6 * max(float(m64.max()), mu_max, 1e-30)
        assert np.all(np.abs(g["mass"] - m64) <= 1e-5 * np.abs(m64) + floor), f"{name}: mass tolerance"
        tr = M64[:, :3].sum(1)
        assert np.all(np.abs(g["moment"] - M64) <= (1e-5 * tr + floor)[:, None]), f"{name}: moment tolerance"
    # the FP32 chain is evaluated in the same order on both sides
    assert np.array_equal(g["mass"].view(np.uint32), r["mass"].view(np.uint32)), f"{name}: FP32 mass not bit-exact"
    assert np.array_equal(g["moment"].view(np.uint32), r["moment"].view(np.uint32)), f"{name}: FP32 moment not bit-exact"
    if lobes:
        assert np.array_equal(g["lobe_count"], r["lobe_count"]), f"{name}: lobe counts differ"
        K = r["lobes"].shape[1]
        for k in range(K):
            sel = r["lobe_count"] > k
            if not sel.any():
                continue
            gl, rl = g["lobes"][sel, k], r["lobes"][sel, k]
            assert np.max(np.abs(gl[:, :6] - rl[:, :6])) <= LOBE_TOL, f"{name}: lobe {k} S"
            assert np.all(np.abs(gl[:, 6] - rl[:, 6]) <= 1e-5 * np.abs(rl[:, 6]) + 1e-30), f"{name}: lobe {k} weight"
            gc, rc = g["compact"][sel, k], r["compact"][sel, k]
            assert np.max(np.abs(gc - rc)) <= 1e-5, f"{name}: compact params of lobe {k}"


# ----------------------------------------------------------------------------
# heightfield (7,938 triangles, 128^3, K = 1): the whole pyramid
# ----------------------------------------------------------------------------
def test_heightfield_full_pyramid(ctx, dirs5000):
    w = synth.config1()
    got = run_gpu(ctx, w, dirs=dirs5000)
    ref0 = oracle.voxelize(w)
    refs = [ref0] + oracle.build_pyramid(ref0, 128, 1, dirs5000)
    assert len(got) == len(refs) == 8
    mu = prim_measure_max(w)
    for lvl, (g, r) in enumerate(zip(got, refs)):
        compare_level(g, r, f"level {lvl}", mu_max=mu)
    # mass conservation across the pyramid (FP64 sums of FP32 outputs)
    tot = got[0]["mass"].astype(np.float64).sum()
    for g in got[1:]:
        assert g["mass"].astype(np.float64).sum() == pytest.approx(tot, rel=1e-5)


@pytest.mark.parametrize("seed,R,rad,pts", [(1, 32, (0.05, 0.4), 30), (2, 64, (0.3, 2.5), 20),
                                            (3, 16, (0.01, 0.2), 30), (4, 128, (1.0, 3.0), 8)])
def test_random_fibers(ctx, dirs5000, seed, R, rad, pts):
    ctrl, off, grid = synth.random_segments(8, pts, R, seed=seed, radius=rad, step=(0.05, 2.0))
    rng = np.random.default_rng(seed)
    n = synth.fiber_segment_count(off)
    w = synth.Workload("rf", "fibers", grid, ctrl=ctrl, fiber_offsets=off,
                       weights=rng.uniform(0.1, 3.0, n).astype(np.float32), K=1)
    got = run_gpu(ctx, w, dirs=dirs5000)
    ref0 = oracle.voxelize(w)
    refs = [ref0] + oracle.build_pyramid(ref0, R, 1, dirs5000)
    for lvl, (g, r) in enumerate(zip(got, refs)):
        compare_level(g, r, f"seed {seed} level {lvl}", mu_max=prim_measure_max(w))


def test_dense_bundle_batches_and_voxel_groups(ctx, dirs5000):
    """A bundle of 72 thick parallel fibers through one region: voxels near its axis hold over
    a hundred capsules (several batches of 32 in the reduce), voxels at its rim a few (packed
    several to a batch).  Every level equals the oracle's, bit for bit."""
    R = 32
    h = 1.0 / R
    rng = np.random.default_rng(21)
    ctrl, off = [], [0]
    for f in range(72):
        y0, z0 = 16.0 + rng.uniform(-1.5, 1.5), 16.0 + rng.uniform(-1.5, 1.5)
        r = rng.uniform(0.6, 1.6)
        for k in range(41):
            x = 4.0 + 0.5 * k + rng.uniform(-0.05, 0.05)
            y, z = y0 + rng.uniform(-0.1, 0.1), z0 + rng.uniform(-0.1, 0.1)
            ctrl.append([x * h, y * h, z * h, r * h])
        off.append(len(ctrl))
    ctrl = np.asarray(ctrl, np.float32)
    off = np.asarray(off, np.int64)
    n = synth.fiber_segment_count(off)
    w = synth.Workload("bundle", "fibers", synth.Grid((0.0, 0.0, 0.0), h, R), ctrl=ctrl, fiber_offsets=off,
                       weights=rng.uniform(0.5, 2.0, n).astype(np.float32), K=4)
    got = run_gpu(ctx, w, dirs=dirs5000)
    ref0 = oracle.voxelize(w)
    refs = [ref0] + oracle.build_pyramid(ref0, R, 4, dirs5000)
    # the case reaches what it is for: voxels of more than 32 capsules next to small ones
    # (capsules counted by their midpoint within r + 1 of the voxel centre)
    A = np.concatenate([ctrl[off[f]:off[f + 1] - 1, :3] for f in range(len(off) - 1)]) * R
    B = np.concatenate([ctrl[off[f] + 1:off[f + 1], :3] for f in range(len(off) - 1)]) * R
    rr = np.concatenate([0.5 * (ctrl[off[f]:off[f + 1] - 1, 3] + ctrl[off[f] + 1:off[f + 1], 3])
                         for f in range(len(off) - 1)]) * R
    mid = 0.5 * (A + B)
    vox = np.stack(np.meshgrid(np.arange(R), np.arange(R), np.arange(R), indexing="ij"), -1).reshape(-1, 3) + 0.5
    near = vox[(np.abs(vox[:, 1] - 16) < 4) & (np.abs(vox[:, 2] - 16) < 4) & (vox[:, 0] > 6) & (vox[:, 0] < 22)]
    counts = np.array([(np.linalg.norm(mid - c, axis=1) < rr + 1.0).sum() for c in near])
    assert counts.max() > 32 and (counts[counts > 0] <= 16).any()
    for lvl, (g, r) in enumerate(zip(got, refs)):
        compare_level(g, r, f"bundle level {lvl}", mu_max=prim_measure_max(w))


def _seg_box_dist(a, b, lo, hi):
    """FP64 distance from segment a-b to box [lo, hi] (ternary search of a convex function)."""
    def g(t):
        p = a + t * (b - a)
        e = np.maximum(np.maximum(lo - p, p - hi), 0.0)
        return float(e @ e)
    l, h = 0.0, 1.0
    for _ in range(200):
        m1, m2 = l + (h - l) / 3, h - (h - l) / 3
        if g(m1) <= g(m2):
            h = m2
        else:
            l = m1
    return np.sqrt(g(0.5 * (l + h)))


def test_grazing_capsules(ctx):
    """Capsules whose radius is within a relative 3e-4 of the distance from their axis to
    one sub-cell, whose nearest point lies inside the segment (so steps 1-2 leave it to the
    exact minimum): the sub-cell decision sits at the edge of step 3 and inside the
    margin of the separation test that drops step-3 work.  One capsule per 8^3 block of a
    64^3 grid, so that no other capsule can set the grazed sub-cells."""
    R = 64
    grid = synth.Grid((0.0, 0.0, 0.0), 1.0 / R, R)
    rng = np.random.default_rng(17)
    eps = [-3e-4, -1e-4, -3e-5, -1e-5, -3e-6, -1e-6, -3e-7, -1e-7, 0.0, 1e-7, 3e-7, 1e-6, 3e-6, 1e-5, 3e-5,
           1e-4, 3e-4]
    ctrl = []
    n = 0
    for bx in range(8):
        for by in range(8):
            for bz in range(8):
                base = np.array([bx, by, bz], np.float64) * 8 + 2.0
                # a segment crossing the block's middle voxel, a target sub-cell beside its middle
                d = rng.normal(size=3)
                d /= np.linalg.norm(d)
                L = rng.uniform(0.5, 3.0)
                m = base + 2.0 + rng.uniform(-0.3, 0.3, 3)
                a = np.float32(m - 0.5 * L * d).astype(np.float64)
                b = np.float32(m + 0.5 * L * d).astype(np.float64)
                side = np.cross(d, rng.normal(size=3))
                side /= np.linalg.norm(side)
                q = 0.5 * (a + b) + side * rng.uniform(0.3, 1.2)
                lo = np.floor(q * 8) / 8
                D = _seg_box_dist(a, b, lo, lo + 0.125)
                if D < 0.05:
                    continue
                r = np.float32(D * (1.0 + eps[n % len(eps)]) / R)
                n += 1
                ctrl += [[*(a / R), r], [*(b / R), r]]
    ctrl = np.array(ctrl, np.float32)
    off = np.arange(0, ctrl.shape[0] + 1, 2, dtype=np.int64)
    w = synth.Workload("graze", "fibers", grid, ctrl=ctrl, fiber_offsets=off, K=1)
    got = run_gpu(ctx, w, lod=False)
    compare_level(got[0], oracle.voxelize(w), "grazing", lobes=False, mu_max=prim_measure_max(w))
    assert n > 400


@pytest.mark.parametrize("seed,R,size", [(1, 16, (0.2, 3.0)), (2, 32, (0.05, 0.5)), (3, 64, (2.0, 12.0))])
def test_random_triangles(ctx, dirs5000, seed, R, size):
    tris, grid = synth.random_triangles(60, R, seed=seed, size=size)
    rng = np.random.default_rng(seed)
    w = synth.Workload("rt", "triangles", grid, tri_verts=tris,
                       weights=rng.uniform(0.1, 3.0, tris.shape[0]).astype(np.float32), K=1)
    got = run_gpu(ctx, w, dirs=dirs5000)
    ref0 = oracle.voxelize(w)
    refs = [ref0] + oracle.build_pyramid(ref0, R, 1, dirs5000)
    for lvl, (g, r) in enumerate(zip(got, refs)):
        compare_level(g, r, f"seed {seed} level {lvl}", mu_max=prim_measure_max(w))


def test_yarn_reduced_sggx_h(ctx, dirs5000):
    """Twisted-ply yarn (3 plies x 8 fibers x 500 segments) at 128^3 with K = 4 SGGX-H."""
    w = synth.config2(fibers_per_ply=8, segments=500, R=128, K=4)
    got = run_gpu(ctx, w, dirs=dirs5000)
    ref0 = oracle.voxelize(w)
    refs = [ref0] + oracle.build_pyramid(ref0, 128, 4, dirs5000)
    clustered = 0
    for lvl, (g, r) in enumerate(zip(got, refs)):
        compare_level(g, r, f"level {lvl}", mu_max=prim_measure_max(w))
        if lvl:
            clustered += int((r["lobe_count"] == 4).sum())
    assert clustered > 100


def test_sggx_h_mass_weighted_merge(ctx, dirs5000):
    """The mass-weighted merge option on the reduced yarn: every level against the oracle
    run with the same rule."""
    w = synth.config2(fibers_per_ply=8, segments=500, R=128, K=4)
    L0 = ctx.voxelize(w.grid, ctrl=torch.from_numpy(w.ctrl).to(DEV),
                      fiber_offsets=torch.from_numpy(w.fiber_offsets).to(DEV))
    pyr = ctx.build_lod(L0, K=4, dirs=torch.from_numpy(dirs5000).to(DEV), merge="mass")
    torch.cuda.synchronize()
    got = [L0.host()] + [p.host() for p in pyr]
    ref0 = oracle.voxelize(w)
    refs = [ref0] + oracle.build_pyramid(ref0, 128, 4, dirs5000, merge=1)
    for lvl, (g, r) in enumerate(zip(got, refs)):
        compare_level(g, r, f"level {lvl}", mu_max=prim_measure_max(w))
    with pytest.raises(ValueError):
        ctx.build_lod(L0, K=4, dirs=torch.from_numpy(dirs5000).to(DEV), merge="median")


def test_sggx_h_more_directions_than_one_pass(ctx):
    """The same yarn with N = 33,000 directions: above 32 x 1024, so the warp tier (levels
    1-2 here, over 2,432 parents) samples through its general loop with 64-bit partial sums,
    while the block tiers keep the paired loop.  Lobes and counts must still match."""
    w = synth.config2(fibers_per_ply=8, segments=500, R=128, K=4)
    dirs = synth.sample_directions(33000)
    got = run_gpu(ctx, w, dirs=dirs)
    ref0 = oracle.voxelize(w)
    refs = [ref0] + oracle.build_pyramid(ref0, 128, 4, dirs)
    assert refs[1]["keys"].shape[0] > 152 * 16
    for lvl, (g, r) in enumerate(zip(got, refs)):
        compare_level(g, r, f"level {lvl}", mu_max=prim_measure_max(w))


@pytest.mark.parametrize("n_dirs", [4999, 33001])
def test_sggx_h_odd_direction_count(ctx, n_dirs):
    """An odd number of directions: the paired sampling loop leaves one sample over, taken
    by a single thread.  4,999 puts every tier on the paired loop; 33,001 puts the warp tier
    on its general loop and the block tiers on the paired loop.  Lobes and counts must match."""
    w = synth.config2(fibers_per_ply=8, segments=500, R=128, K=4)
    dirs = synth.sample_directions(n_dirs)
    got = run_gpu(ctx, w, dirs=dirs)
    ref0 = oracle.voxelize(w)
    refs = [ref0] + oracle.build_pyramid(ref0, 128, 4, dirs)
    for lvl, (g, r) in enumerate(zip(got, refs)):
        compare_level(g, r, f"level {lvl}", mu_max=prim_measure_max(w))


def test_catmull_rom_splines(ctx, dirs5000):
    """Spline fibers: the device tessellation equals the oracle's bit for bit, and the
    tessellated fibers voxelize to the oracle's pyramid (a yarn whose polylines are
    subsampled to every 8th node and re-tessellated with 8 points per span)."""
    w = synth.config2(fibers_per_ply=6, segments=480, R=128, K=4)
    off = w.fiber_offsets
    keep = []
    for f in range(len(off) - 1):
        idx = np.arange(off[f], off[f + 1])
        keep.append(np.unique(np.concatenate([idx[::8], idx[-1:]])))
    nodes = np.concatenate([w.ctrl[k] for k in keep]).astype(np.float32)
    noff = np.concatenate([[0], np.cumsum([len(k) for k in keep])]).astype(np.int64)
    S = 8
    ctrl_d, off_d = ctx.tessellate_catmull_rom(torch.from_numpy(nodes).to(DEV), torch.from_numpy(noff).to(DEV), S)
    ctrl_o, off_o = oracle.catmull_rom(nodes, noff, S)
    assert np.array_equal(off_d.cpu().numpy(), off_o)
    assert np.array_equal(ctrl_d.cpu().numpy().view(np.uint32), ctrl_o.view(np.uint32))
    ws = synth.Workload("spl", "fibers", w.grid, ctrl=ctrl_o, fiber_offsets=off_o, K=4)
    L0 = ctx.voxelize(ws.grid, ctrl=ctrl_d, fiber_offsets=off_d)
    pyr = ctx.build_lod(L0, K=4, dirs=torch.from_numpy(dirs5000).to(DEV))
    torch.cuda.synchronize()
    got = [L0.host()] + [p.host() for p in pyr]
    ref0 = oracle.voxelize(ws)
    refs = [ref0] + oracle.build_pyramid(ref0, 128, 4, dirs5000)
    for lvl, (g, r) in enumerate(zip(got, refs)):
        compare_level(g, r, f"splines level {lvl}", mu_max=prim_measure_max(ws))
    # a spline without nodes is rejected, and so are offsets that do not run from 0 to the
    # node count (the last spline would read past the nodes)
    for bad in ([0, 3, 3, len(nodes)], [0, 3, len(nodes) + 2], [1, 3, len(nodes)]):
        with pytest.raises(vx.VxError) as e:
            ctx.tessellate_catmull_rom(torch.from_numpy(nodes).to(DEV),
                                       torch.tensor(bad, dtype=torch.int64, device=DEV), S)
        assert e.value.status == 1


def test_sampled_fibers(ctx):
    """The sample-based level 0 (4 axis samples per segment) of the reduced yarn against the
    oracle's, and its sub-cells inside the exact path's (a sample lies inside its capsule)."""
    w = synth.config2(fibers_per_ply=8, segments=500, R=128, K=1)
    ctrl = torch.from_numpy(w.ctrl).to(DEV)
    off = torch.from_numpy(w.fiber_offsets).to(DEV)
    Ls = ctx.voxelize_sampled(w.grid, ctrl=ctrl, fiber_offsets=off, samples=4)
    Le = ctx.voxelize(w.grid, ctrl=ctrl, fiber_offsets=off)
    torch.cuda.synchronize()
    gs, ge = Ls.host(), Le.host()
    rs = oracle.voxelize_fibers_sampled(w.ctrl, w.fiber_offsets, w.grid, 4)
    compare_level(gs, rs, "sampled", mu_max=prim_measure_max(w))
    pos = np.searchsorted(ge["keys"], gs["keys"])
    assert np.array_equal(ge["keys"][pos], gs["keys"])
    assert np.all((gs["mask"] & ~ge["mask"][pos]) == 0)
    assert gs["occ"].sum() < ge["occ"].sum()


def test_sampled_triangles(ctx):
    """The sample-based level 0 of the heightfield (up to 16 samples per triangle by area)
    against the oracle's, and inside the exact path's sub-cells."""
    w = synth.config1()
    tv = torch.from_numpy(w.tri_verts).to(DEV)
    Ls = ctx.voxelize_sampled(w.grid, tri_verts=tv, samples=16)
    Le = ctx.voxelize(w.grid, tri_verts=tv)
    torch.cuda.synchronize()
    gs, ge = Ls.host(), Le.host()
    rs = oracle.voxelize_tris_sampled(w.tri_verts, w.grid, 16)
    compare_level(gs, rs, "sampled triangles", mu_max=prim_measure_max(w))
    pos = np.searchsorted(ge["keys"], gs["keys"])
    assert np.array_equal(ge["keys"][pos], gs["keys"])
    assert np.all((gs["mask"] & ~ge["mask"][pos]) == 0)


def test_export_vdb_leaves(ctx, dirs5000):
    """OpenVDB-style leaf tables of the reduced yarn's level 0 and level 2 against the oracle's
    tables of its own levels."""
    w = synth.config2(fibers_per_ply=8, segments=500, R=128, K=1)
    L0 = ctx.voxelize(w.grid, ctrl=torch.from_numpy(w.ctrl).to(DEV),
                      fiber_offsets=torch.from_numpy(w.fiber_offsets).to(DEV))
    pyr = ctx.build_lod(L0, K=1, num_levels=2)
    ref0 = oracle.voxelize(w)
    refs = [ref0] + oracle.build_pyramid(ref0, 128, 1, dirs5000, num_levels=2)
    for lvl, lv in ((0, L0), (2, pyr[1])):
        k, m, f = ctx.export_leaves(lv)
        rk, rm, rf = oracle.vdb_leaves(refs[lvl]["keys"])
        assert np.array_equal(k.cpu().numpy().view(np.uint64), rk), f"level {lvl}: leaf keys"
        assert np.array_equal(m.cpu().numpy().view(np.uint64), rm), f"level {lvl}: value masks"
        assert np.array_equal(f.cpu().numpy().astype(np.int64), rf), f"level {lvl}: first voxels"


def test_export_compact8(ctx, dirs5000):
    """8-bit compact SGGX export of every level of the K = 4 yarn pyramid against the
    oracle's quantization of its own compact parameters.  Level 0 (S = M/m, bit-exact
    inputs) must match byte for byte; on coarser levels the lobes agree to 1e-5, so a byte
    may differ by one only where the oracle's scaled value lies within 1e-3 of a rounding
    boundary.  Lobes past lobe_count are zero."""
    w = synth.config2(fibers_per_ply=8, segments=500, R=128, K=4)
    L0 = ctx.voxelize(w.grid, ctrl=torch.from_numpy(w.ctrl).to(DEV),
                      fiber_offsets=torch.from_numpy(w.fiber_offsets).to(DEV))
    pyr = ctx.build_lod(L0, K=4, dirs=torch.from_numpy(dirs5000).to(DEV))
    got = [ctx.export_compact8(lv).cpu().numpy() for lv in [L0] + pyr]
    ref0 = oracle.voxelize(w)
    refs = [ref0] + oracle.build_pyramid(ref0, 128, 4, dirs5000)
    scale = np.array([255.0] * 3 + [127.5] * 3)
    bias = np.array([0.0] * 3 + [127.5] * 3)
    for lvl, (g, r) in enumerate(zip(got, refs)):
        # (the oracle's level 0 is stored with the pyramid's K; it holds at most one lobe)
        K = g.shape[1]
        assert g.shape[0] == r["keys"].shape[0] and r["lobe_count"].max() <= K
        comp = r["compact"][:, :K]
        q = oracle.compact8(comp)
        live = np.arange(K)[None, :] < r["lobe_count"][:, None]
        q[~live] = 0
        if lvl == 0:
            assert np.array_equal(g, q), "level 0: bytes differ"
            continue
        x = comp.astype(np.float64) * scale + bias
        near = np.abs(x - np.floor(x) - 0.5) < 1e-3
        diff = g.astype(np.int32) - q.astype(np.int32)
        assert np.abs(diff).max() <= 1, f"level {lvl}"
        assert np.all((diff == 0) | (near & live[..., None])), f"level {lvl}: bytes differ away from a boundary"


# ----------------------------------------------------------------------------
# edge cases
# ----------------------------------------------------------------------------
def test_empty_and_outside(ctx):
    grid = synth.Grid((0.0, 0.0, 0.0), 1.0 / 16, 16)
    ctrl = np.array([[2.0, 2.0, 2.0, 0.01], [2.5, 2.0, 2.0, 0.01]], np.float32)   # outside
    off = np.array([0, 2], np.int64)
    w = synth.Workload("out", "fibers", grid, ctrl=ctrl, fiber_offsets=off)
    got = run_gpu(ctx, w, K=1, lod=True)
    assert all(g["keys"].shape[0] == 0 for g in got)
    tris = np.zeros((0, 3, 4), np.float32)
    w = synth.Workload("none", "triangles", grid, tri_verts=tris)
    got = run_gpu(ctx, w, K=1, lod=False)
    assert got[0]["keys"].shape[0] == 0


def test_degenerate_primitives(ctx, dirs5000):
    grid = synth.Grid((0.0, 0.0, 0.0), 1.0 / 8, 8)
    # zero-length segment (a sphere), a segment along a grid line, fibers with 1 point
    ctrl = np.array([[0.3, 0.3, 0.3, 0.05], [0.3, 0.3, 0.3, 0.05],
                     [0.5, 0.5, 0.1, 0.02], [0.5, 0.5, 0.9, 0.02],
                     [0.7, 0.7, 0.7, 0.1]], np.float32)
    off = np.array([0, 2, 4, 5], np.int64)
    w = synth.Workload("deg", "fibers", grid, ctrl=ctrl, fiber_offsets=off)
    got = run_gpu(ctx, w, K=1, dirs=dirs5000)
    ref0 = oracle.voxelize(w)
    refs = [ref0] + oracle.build_pyramid(ref0, 8, 1, dirs5000)
    for lvl, (g, r) in enumerate(zip(got, refs)):
        compare_level(g, r, f"level {lvl}", mu_max=prim_measure_max(w))
    # degenerate triangles: a line and a point, plus a triangle in a grid plane
    tris = np.zeros((3, 3, 4), np.float32)
    tris[0, :, :3] = [[0.1, 0.1, 0.1], [0.6, 0.6, 0.6], [0.35, 0.35, 0.35]]
    tris[1, :, :3] = [[0.4, 0.2, 0.7]] * 3
    tris[2, :, :3] = [[0.1, 0.1, 0.5], [0.9, 0.1, 0.5], [0.1, 0.9, 0.5]]
    w = synth.Workload("degt", "triangles", grid, tri_verts=tris)
    got = run_gpu(ctx, w, K=1, dirs=dirs5000)
    ref0 = oracle.voxelize(w)
    refs = [ref0] + oracle.build_pyramid(ref0, 8, 1, dirs5000)
    for lvl, (g, r) in enumerate(zip(got, refs)):
        compare_level(g, r, f"tri level {lvl}", mu_max=prim_measure_max(w))


def test_single_voxel_grid_and_max_resolution(ctx, dirs5000):
    for R in (1, 1024):
        # radii and steps in voxel units of the grid itself: a few voxels per primitive
        ctrl, off, grid = synth.random_segments(2, 5, R, seed=9, radius=(0.1, 1.5), step=(0.3, 2.0))
        w = synth.Workload("r", "fibers", grid, ctrl=ctrl, fiber_offsets=off, K=1)
        got = run_gpu(ctx, w, K=1, dirs=dirs5000, num_levels=min(3, int(np.log2(R))))
        ref0 = oracle.voxelize(w)
        refs = [ref0] + (oracle.build_pyramid(ref0, R, 1, dirs5000, num_levels=3) if R > 1 else [])
        for lvl, (g, r) in enumerate(zip(got, refs)):
            compare_level(g, r, f"R={R} level {lvl}", mu_max=prim_measure_max(w))


def test_invalid_arguments(ctx):
    grid = synth.Grid((0.0, 0.0, 0.0), 1.0 / 16, 16)
    ctrl = torch.zeros((4, 4), dtype=torch.float32, device=DEV)
    off = torch.tensor([0, 4], dtype=torch.int64, device=DEV)
    with pytest.raises(vx.VxError) as e:
        ctx.voxelize(grid, ctrl=ctrl, fiber_offsets=off, num_prims=7)   # wrong segment count
    assert e.value.status == 1
    with pytest.raises(vx.VxError) as e:
        ctx.voxelize(synth.Grid((0.0, 0.0, 0.0), 1.0 / 12, 12), ctrl=ctrl, fiber_offsets=off)
    assert e.value.status == 1
    with pytest.raises(vx.VxError) as e:
        ctx.voxelize(synth.Grid((0.0, 0.0, 0.0), 1.0 / 4096, 4096), ctrl=ctrl, fiber_offsets=off)
    assert e.value.status == 6
    # non-finite coordinates and negative weights or radii are rejected (the ranges of such
    # records are empty, so nothing runs on them before the error is read back)
    bad = ctrl.clone()
    bad[1, 0] = float("nan")
    with pytest.raises(vx.VxError) as e:
        ctx.voxelize(grid, ctrl=bad, fiber_offsets=off)
    assert e.value.status == 1
    bad = ctrl.clone()
    bad[2, 3] = -1.0
    with pytest.raises(vx.VxError) as e:
        ctx.voxelize(grid, ctrl=bad, fiber_offsets=off)
    assert e.value.status == 1
    tris = torch.full((2, 3, 4), 0.5, dtype=torch.float32, device=DEV)
    with pytest.raises(vx.VxError) as e:
        ctx.voxelize(grid, tri_verts=tris, weights=torch.tensor([1.0, -2.0], device=DEV))
    assert e.value.status == 1
    tris[1, 2, 1] = float("inf")
    with pytest.raises(vx.VxError) as e:
        ctx.voxelize(grid, tri_verts=tris)
    assert e.value.status == 1
    # offsets that reach past ctrl[num_ctrl - 1], or start below 0, are flagged before any
    # control point outside the array is read (the buffer is sliced so that the bytes past
    # num_ctrl exist and belong to this test)
    big = torch.zeros((8, 4), dtype=torch.float32, device=DEV)
    P = vx.api.VxPrimitives()
    P.kind, P.num_prims, P.ctrl, P.num_ctrl = vx.api.VX_FIBERS, 4, big.data_ptr(), 4
    for bad_off in ([0, 5], [-1, 4], [3, 1, 4]):
        o = torch.tensor(bad_off, dtype=torch.int64, device=DEV)
        P.fiber_offsets, P.num_fibers = o.data_ptr(), len(bad_off) - 1
        P.num_prims = sum(max(b - a - 1, 0) for a, b in zip(bad_off[:-1], bad_off[1:]))
        out = vx.api.VxLevel()
        st = ctx.lib.vx_voxelize(ctx.h, C.byref(P), C.byref(vx.api._grid(grid)), vx.api._stream(None),
                                 C.byref(out))
        assert st == 1, bad_off
    L0 = ctx.voxelize(grid, ctrl=ctrl, fiber_offsets=off)
    with pytest.raises(vx.VxError) as e:
        ctx.build_lod(L0, K=9)
    assert e.value.status == 6
    with pytest.raises(vx.VxError) as e:
        ctx.build_lod(L0, K=4)          # K > 1 needs the direction set
    assert e.value.status == 1


def test_deterministic(ctx, dirs5000):
    w = synth.config2(fibers_per_ply=4, segments=400, R=64, K=4)
    a = run_gpu(ctx, w, dirs=dirs5000)
    b = run_gpu(ctx, w, dirs=dirs5000)
    for x, y in zip(a, b):
        for k in ("keys", "mask", "mass", "moment", "lobes", "lobe_count", "compact"):
            assert np.array_equal(np.asarray(x[k]).view(np.uint8), np.asarray(y[k]).view(np.uint8)), k


def test_tiled_2048_grid(ctx, dirs5000):
    """A 2048^3 grid runs as eight 1024^3 tiles: fibers crossing the tile planes at 1024."""
    R = 2048
    rng = np.random.default_rng(12)
    h = 1.0 / R
    ctrl, off = [], [0]
    for f in range(12):
        p = np.array([1024.0, 1024.0, 1024.0]) + rng.uniform(-6, 6, 3)
        d = rng.standard_normal(3); d /= np.linalg.norm(d)
        r = rng.uniform(0.3, 2.0)
        for k in range(12):
            ctrl.append([p[0] * h, p[1] * h, p[2] * h, r * h])
            d = d + 0.5 * rng.standard_normal(3); d /= np.linalg.norm(d)
            p = p + d * rng.uniform(0.3, 1.5)
        off.append(len(ctrl))
    w = synth.Workload("t2048", "fibers", synth.Grid((0.0, 0.0, 0.0), h, R),
                       ctrl=np.asarray(ctrl, np.float32), fiber_offsets=np.asarray(off, np.int64), K=1)
    got = run_gpu(ctx, w, dirs=dirs5000, num_levels=4)
    ref0 = oracle.voxelize(w)
    refs = [ref0] + oracle.build_pyramid(ref0, R, 1, dirs5000, num_levels=4)
    tiles = np.unique(got[0]["keys"] >> np.uint64(30))
    assert tiles.size == 8, tiles
    for lvl, (g, r) in enumerate(zip(got, refs)):
        compare_level(g, r, f"level {lvl}", mu_max=prim_measure_max(w))


@pytest.mark.parametrize("kind", ["fibers", "triangles"])
def test_windows_split_by_pair_limit(ctx, dirs5000, kind):
    """A per-pass pair limit far below the total splits the grid into octant windows,
    recursively; the concatenated level is bit-identical to the oracle and to one pass."""
    R = 64
    if kind == "fibers":
        ctrl, off, grid = synth.random_segments(6, 10, R, seed=21, radius=(0.2, 1.5), step=(0.5, 2.5))
        w = synth.Workload("split-f", "fibers", grid, ctrl=ctrl, fiber_offsets=off, K=4)
    else:
        tris, grid = synth.random_triangles(60, R, seed=22, size=(0.5, 4.0))
        w = synth.Workload("split-t", "triangles", grid, tri_verts=tris, K=4)
    one = run_gpu(ctx, w, dirs=dirs5000, num_levels=3)
    try:
        ctx.set_max_pairs_per_pass(97)
        split = run_gpu(ctx, w, dirs=dirs5000, num_levels=3)
        if kind == "fibers":
            ctx.set_max_pairs_per_pass(1)       # the voxel of a joint holds two segments' pairs
            with pytest.raises(vx.VxError) as e:
                run_gpu(ctx, w, lod=False)
            assert e.value.status == 3
    finally:
        ctx.set_max_pairs_per_pass(2 ** 31 - 1)
    ref0 = oracle.voxelize(w)
    refs = [ref0] + oracle.build_pyramid(ref0, R, 4, dirs5000, num_levels=3)
    for lvl, (a, b, r) in enumerate(zip(one, split, refs)):
        for k in ("keys", "mask", "mass", "moment", "lobes", "lobe_count", "compact"):
            assert np.array_equal(np.asarray(a[k]).view(np.uint8), np.asarray(b[k]).view(np.uint8)), (lvl, k)
        compare_level(b, r, f"level {lvl}", mu_max=prim_measure_max(w))


# ----------------------------------------------------------------------------
# the windowed pyramid (vx_voxelize_lod_windowed) against the whole one
# ----------------------------------------------------------------------------
FIELDS = ("keys", "mask", "mass", "moment", "occ", "proj", "lobe_count", "lobes", "compact")


def _cat_levels(parts):
    out = {}
    for f in FIELDS:
        out[f] = np.concatenate([p[f] for p in parts]) if parts else None
    return out


@pytest.mark.parametrize("kind,w_log2,K", [("fibers", 4, 4), ("fibers", 6, 1), ("triangles", 5, 1),
                                           ("triangles", 3, 4)])
def test_windowed_pyramid_equals_whole(ctx, dirs5000, kind, w_log2, K):
    """Every window's levels 0 .. w-1, concatenated in window order, and the levels built
    from the windows' roots equal vx_voxelize + vx_build_lod bit for bit (all fields)."""
    if kind == "fibers":
        w = synth.config2(fibers_per_ply=6, segments=480, R=128, K=K)
        geom = dict(ctrl=torch.from_numpy(w.ctrl).to(DEV), fiber_offsets=torch.from_numpy(w.fiber_offsets).to(DEV))
    else:
        w = synth.config1()
        geom = dict(tri_verts=torch.from_numpy(w.tri_verts).to(DEV))
    dirs = torch.from_numpy(dirs5000).to(DEV) if K > 1 else None
    L0 = ctx.voxelize(w.grid, **geom)
    whole = [L0.host()] + [p.host() for p in ctx.build_lod(L0, K=K, dirs=dirs)]
    per_level = [[] for _ in range(w_log2)]
    seen = []

    def on_window(win, levels):
        assert len(levels) == w_log2 and win["log2_size"] == w_log2
        seen.append(win)
        for l, lv in enumerate(levels):
            per_level[l].append(lv.host())

    top = ctx.voxelize_lod_windowed(w.grid, window_log2=w_log2, on_window=on_window, K=K, dirs=dirs, **geom)
    torch.cuda.synchronize()
    assert len(seen) > 1 and [s["index"] for s in seen] == list(range(len(seen)))
    assert len(top) == len(whole) - w_log2
    got = [_cat_levels(p) for p in per_level] + [t.host() for t in top]
    roots = np.asarray(got[w_log2]["keys"]).astype(np.uint64)
    assert len(roots) == len(seen)
    for win in seen:   # a window's index is its root's row in the top level
        finest = np.asarray(per_level[w_log2 - 1][win["index"]]["keys"]).astype(np.uint64)
        assert np.all((finest >> np.uint64(3)) == roots[win["index"]])
    for l, (g, r) in enumerate(zip(got, whole)):
        for f in FIELDS:
            assert np.array_equal(np.asarray(g[f]).view(np.uint8), np.asarray(r[f]).view(np.uint8)), (l, f)


def test_windowed_callback_error_stops_the_call(ctx):
    w = synth.config2(fibers_per_ply=2, segments=200, R=64, K=1)
    geom = dict(ctrl=torch.from_numpy(w.ctrl).to(DEV), fiber_offsets=torch.from_numpy(w.fiber_offsets).to(DEV))
    calls = []

    def on_window(win, levels):
        calls.append(win["index"])
        if len(calls) == 2:
            raise KeyError("stop")

    with pytest.raises(KeyError):
        ctx.voxelize_lod_windowed(w.grid, window_log2=3, on_window=on_window, **geom)
    assert calls == [0, 1]
    with pytest.raises(vx.VxError) as e:
        ctx.voxelize_lod_windowed(w.grid, window_log2=7, on_window=on_window, **geom)   # w > log2 R
    assert e.value.status == 1


def test_windowed_pyramid_with_split_windows_equals_whole(ctx, dirs5000):
    """A pass limit below a window's pairs splits each window further inside the windowed
    call (its level 0 then takes the two-pass path); the result is still the whole pyramid."""
    w = synth.config2(fibers_per_ply=6, segments=480, R=128, K=4)
    geom = dict(ctrl=torch.from_numpy(w.ctrl).to(DEV), fiber_offsets=torch.from_numpy(w.fiber_offsets).to(DEV))
    dirs = torch.from_numpy(dirs5000).to(DEV)
    L0 = ctx.voxelize(w.grid, **geom)
    whole = [L0.host()] + [p.host() for p in ctx.build_lod(L0, K=4, dirs=dirs)]
    per_level = [[] for _ in range(5)]

    def on_window(win, levels):
        for l, lv in enumerate(levels):
            per_level[l].append(lv.host())

    ctx.set_max_pairs_per_pass(20_000)
    try:
        top = ctx.voxelize_lod_windowed(w.grid, window_log2=5, on_window=on_window, K=4, dirs=dirs, **geom)
        torch.cuda.synchronize()
    finally:
        ctx.set_max_pairs_per_pass(2**31 - 1)
    got = [_cat_levels(p) for p in per_level] + [t.host() for t in top]
    assert len(got) == len(whole)
    for l, (g, r) in enumerate(zip(got, whole)):
        for f in FIELDS:
            assert np.array_equal(np.asarray(g[f]).view(np.uint8), np.asarray(r[f]).view(np.uint8)), (l, f)


def test_build_lod_while_level0_downloads(ctx, dirs5000):
    """vx_build_lod's sizing readback is a kernel store into mapped memory, so the call runs
    beside a large download of its input on another stream; the pyramid and the downloaded
    level are unchanged by the overlap."""
    w = synth.config2(fibers_per_ply=6, segments=480, R=128, K=4)
    geom = dict(ctrl=torch.from_numpy(w.ctrl).to(DEV), fiber_offsets=torch.from_numpy(w.fiber_offsets).to(DEV))
    dirs = torch.from_numpy(dirs5000).to(DEV)
    L0 = ctx.voxelize(w.grid, **geom)
    ref = [p.host() for p in ctx.build_lod(L0, K=4, dirs=dirs)]
    torch.cuda.synchronize()
    host = torch.empty(L0.block.numel(), dtype=torch.uint8).pin_memory()
    side = torch.cuda.Stream(DEV)
    ev = torch.cuda.Event()
    ev.record()
    with torch.cuda.stream(side):
        side.wait_event(ev)
        host.copy_(L0.block, non_blocking=True)
    got = [p.host() for p in ctx.build_lod(L0, K=4, dirs=dirs)]
    torch.cuda.synchronize()
    assert torch.equal(host, L0.block.cpu())
    assert len(got) == len(ref)
    for l, (g, r) in enumerate(zip(got, ref)):
        for f in FIELDS:
            assert np.array_equal(np.asarray(g[f]).view(np.uint8), np.asarray(r[f]).view(np.uint8)), (l, f)
    prof_names = ctx.profile_read().keys()
    assert "readback" in prof_names
    # the levels downloaded on the side stream, each after its completion event
    evs = [torch.cuda.Event() for _ in ref]
    lv = ctx.build_lod(L0, K=4, dirs=dirs, events=evs)
    hosts = [torch.empty(x.block.numel(), dtype=torch.uint8).pin_memory() for x in lv]
    with torch.cuda.stream(side):
        for x, h, ev in zip(lv, hosts, evs):
            side.wait_event(ev)
            h.copy_(x.block, non_blocking=True)
    torch.cuda.synchronize()
    for l, (x, h, r) in enumerate(zip(lv, hosts, ref)):
        assert torch.equal(h, x.block.cpu()), l
        g = x.host()
        for f in FIELDS:
            assert np.array_equal(np.asarray(g[f]).view(np.uint8), np.asarray(r[f]).view(np.uint8)), (l, f)
