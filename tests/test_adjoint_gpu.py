"""Adjoint (vx_backward / VoxelizeLoD) against the oracle's FP64 analytic gradient and
FP64 central finite differences.

Loss: sum over levels 0..L and voxels of alpha * m + beta . M with U(-1,1) weights
drawn per (level, key, component) by a counter-based generator, so both sides draw the
same weights from their own key sets.  Parameters: control-point xyz, radii, weights.
Tolerance: |g32 - g64| <= 1e-4 * max(|g64|, median |g64|) against the analytic gradient;
against FD, 1e-4 relative to max(|FD|, 1% of the summed magnitudes of the parameter's
per-pair terms) (FP32 per-pair terms carry ~1e-6 relative error, so the rounding of a sum
of cancelling terms scales with the terms, not with the total).
FD: central, FP64, h = 1e-4 in voxel units (the method's coordinates after the grid
normalisation of Sec. 3.1; 1e-4 / 256 in world units here), on 64 random parameters whose
stencil does not cross a kink (a clipped piece changing its entering or leaving plane
between -h and +h, detected exactly from the oracle's active sets); skipped draws are
counted and reported.  (A world-unit step of 1e-4 is 1/40 voxel: it rotates the 0.13-voxel
segments of this yarn by ~0.2 rad, and the central difference's own h^2 error reaches ~0.5%.)
"""
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


@pytest.fixture(scope="module")
def ctx():
    c = vx.Context(DEV)
    yield c
    c.close()


def gpu_forward_backward(ctx, w, levels, weights):
    ctrl = torch.from_numpy(w.ctrl).to(DEV).requires_grad_(True)
    wt = torch.from_numpy(weights).to(DEV).requires_grad_(True)
    off = torch.from_numpy(w.fiber_offsets).to(DEV)
    outs = vx.VoxelizeLoD.apply(ctrl, wt, off, w.grid, levels, ctx)
    # level keys for the loss weights: rebuild them from the forward's level 0
    L0 = ctx.voxelize(w.grid, ctrl=ctrl.detach(), fiber_offsets=off, weights=wt.detach())
    pyr = ctx.build_lod(L0, K=1, num_levels=levels)
    keys = [lv.keys.cpu().numpy().view(np.uint64) for lv in [L0] + pyr]
    loss = 0.0
    for l in range(levels + 1):
        a, b = synth.loss_weights(keys[l], l)
        loss = loss + (outs[2 * l] * torch.from_numpy(a).to(DEV)).sum() + \
            (outs[2 * l + 1] * torch.from_numpy(b).to(DEV)).sum()
    loss.backward()
    torch.cuda.synchronize()
    return ctrl.grad.cpu().numpy(), wt.grad.cpu().numpy(), keys


def _floor_report(name, got, ref, floor):
    """Entries that pass 1e-4 only through the floor, and the cap: every entry whose |ref|
    is at least 1e-3 of the floor is within 1e-3 of |ref|."""
    err = np.abs(got - ref)
    only_floor = int(np.sum((err > 1e-4 * np.abs(ref)) & (err <= 1e-4 * np.maximum(np.abs(ref), floor))))
    big = np.abs(ref) >= 1e-3 * floor
    worst = float(np.max(err[big] / np.abs(ref[big]))) if big.any() else 0.0
    print(f"{name}: {ref.size} entries, {only_floor} within 1e-4 only through the floor, "
          f"{int((~big).sum())} below 1e-3 of the floor, worst relative error above it {worst:.2e}")
    assert worst <= 1e-3, (name, worst)


def test_adjoint_matches_oracle_gradient(ctx):
    w = synth.config2(fibers_per_ply=4, segments=300, R=64, K=1)
    levels = 4
    rng = np.random.default_rng(51)
    weights = rng.uniform(0.5, 2.0, w.num_prims).astype(np.float32)
    g_ctrl, g_w, keys = gpu_forward_backward(ctx, w, levels, weights)
    ref0 = oracle.voxelize_fibers(w.ctrl, w.fiber_offsets, w.grid, weights)
    refs = [ref0] + oracle.build_pyramid(ref0, 64, 1, synth.sample_directions(16), num_levels=levels)
    for l in range(levels + 1):
        assert np.array_equal(refs[l]["keys"], keys[l])
    ab = [synth.loss_weights(r["keys"], l) for l, r in enumerate(refs)]
    gm0, gM0 = oracle.broadcast_adjoints(ref0["keys"], [r["keys"] for r in refs], [a for a, _ in ab],
                                         [b for _, b in ab])
    _, d_ctrl, d_w = oracle.fiber_adjoint(w.ctrl, w.fiber_offsets, w.grid, ref0["keys"], gm0, gM0, weights=weights)
    scale = np.median(np.abs(d_ctrl[:, :3]))
    err = np.abs(g_ctrl[:, :3] - d_ctrl[:, :3])
    assert np.all(err <= 1e-4 * np.maximum(np.abs(d_ctrl[:, :3]), scale)), err.max()
    rs = np.median(np.abs(d_ctrl[:, 3]))
    assert np.all(np.abs(g_ctrl[:, 3] - d_ctrl[:, 3]) <= 1e-4 * np.maximum(np.abs(d_ctrl[:, 3]), rs))
    ws = np.median(np.abs(d_w))
    assert np.all(np.abs(g_w - d_w) <= 1e-4 * np.maximum(np.abs(d_w), ws))
    _floor_report("ctrl xyz", g_ctrl[:, :3], d_ctrl[:, :3], scale)
    _floor_report("radius", g_ctrl[:, 3], d_ctrl[:, 3], rs)
    _floor_report("weight", g_w, d_w, ws)


def test_adjoint_finite_differences_yarn_256(ctx):
    """Config 5: the yarn at 256^3 with 4 LoD levels, 64 random parameters."""
    w = synth.config5()
    levels = w.levels
    weights = np.ones(w.num_prims, np.float32)
    g_ctrl, g_w, keys = gpu_forward_backward(ctx, w, levels, weights)
    rng = np.random.default_rng(w.extra["seed"])
    off = w.fiber_offsets
    P = w.ctrl.shape[0]
    c64 = w.ctrl.astype(np.float64)
    h = 1e-4 * w.grid.voxel_size
    checked, kinks, worst, floored, worst_fd = 0, 0, 0.0, 0, 0.0
    while checked < w.extra["n_params"]:
        assert kinks < 10 * w.extra["n_params"], "too many stencils cross a kink"
        c = int(rng.integers(0, P))
        comp = int(rng.integers(0, 4))
        f = int(np.searchsorted(off, c, side="right") - 1)
        # segments touching control point c (segment ids count c - f for >= 1-point fibers)
        prims = []
        if c > off[f]:
            prims.append(c - f - 1)
        if c + 1 < off[f + 1]:
            prims.append(c - f)
        # exclude stencils on which a clipped piece changes its entering/leaving plane
        sig = []
        for step in (-h, 0.0, h):
            cc = c64.copy(); cc[c, comp] += step
            sig.append(oracle.clip_signature(cc, off, w.grid, prims))
        if len(set(sig)) != 1:
            kinks += 1
            continue
        # occupied voxels near the affected segments (brute force over every primitive)
        s = 1.0 / w.grid.voxel_size
        pts = c64[max(c - 1, 0): c + 2, :3] * s
        lo = np.maximum(np.floor(pts.min(0) - 2.5).astype(int), 0)
        hi = np.minimum(np.floor(pts.max(0) + 2.5).astype(int), w.grid.resolution - 1)
        g = np.stack(np.meshgrid(*[np.arange(lo[i], hi[i] + 1) for i in range(3)], indexing="ij"), -1).reshape(-1, 3)
        cand = np.array([oracle.morton(int(x), int(y), int(z)) for x, y, z in g], np.uint64)
        vox = oracle.fiber_voxels(w.ctrl, off, w.grid, cand)
        occ = cand[vox["mask"].any(1)]
        occ.sort()
        gm0 = np.zeros(occ.shape[0]); gM0 = np.zeros((occ.shape[0], 6))
        for l in range(levels + 1):
            a, b = synth.loss_weights(occ >> np.uint64(3 * l), l)
            gm0 += a; gM0 += b

        def local_loss(cc):
            return oracle.fiber_adjoint(cc, off, w.grid, occ, gm0, gM0, prims=np.array(prims))[0]

        def fd(step):
            cp = c64.copy(); cp[c, comp] += step
            cm = c64.copy(); cm[c, comp] -= step
            return (local_loss(cp) - local_loss(cm)) / (2 * step)
        f1 = fd(h)
        _, d_ctrl, _, d_abs = oracle.fiber_adjoint(c64, off, w.grid, occ, gm0, gM0, prims=np.array(prims),
                                                   with_abs=True)
        ref = d_ctrl[c, comp]
        # scale: |gradient| or 1% of its summed per-pair term magnitudes (FP32 rounding of the
        # sum scales with the terms, not with their possibly cancelling total)
        scale = max(abs(f1), 0.01 * d_abs[c, comp], 1e-3)
        assert abs(ref - f1) <= 1e-4 * scale, (c, comp, ref, f1)
        err = abs(g_ctrl[c, comp] - f1) / scale
        worst = max(worst, err)
        assert err <= 1e-4, (c, comp, g_ctrl[c, comp], f1)
        # the floor is capped: relative to |FD| itself every parameter is within 1e-3
        rel = abs(g_ctrl[c, comp] - f1) / max(abs(f1), 1e-30)
        floored += rel > 1e-4
        worst_fd = max(worst_fd, rel)
        assert rel <= 1e-3, (c, comp, g_ctrl[c, comp], f1)
        checked += 1
    print(f"FD checked {checked}, stencils across a kink skipped {kinks}, worst rel {worst:.2e}; "
          f"{floored} within 1e-4 only through the floor, worst relative to |FD| {worst_fd:.2e}")


# ----------------------------------------------------------------------------
# triangles: the config-1 heightfield
# ----------------------------------------------------------------------------
def gpu_tri_forward_backward(ctx, w, levels, weights):
    tv = torch.from_numpy(w.tri_verts).to(DEV).requires_grad_(True)
    wt = torch.from_numpy(weights).to(DEV).requires_grad_(True)
    outs = vx.VoxelizeLoD.apply(tv, wt, None, w.grid, levels, ctx)
    L0 = ctx.voxelize(w.grid, tri_verts=tv.detach(), weights=wt.detach())
    pyr = ctx.build_lod(L0, K=1, num_levels=levels)
    keys = [lv.keys.cpu().numpy().view(np.uint64) for lv in [L0] + pyr]
    loss = 0.0
    for l in range(levels + 1):
        a, b = synth.loss_weights(keys[l], l)
        loss = loss + (outs[2 * l] * torch.from_numpy(a).to(DEV)).sum() + \
            (outs[2 * l + 1] * torch.from_numpy(b).to(DEV)).sum()
    loss.backward()
    torch.cuda.synchronize()
    return tv.grad.cpu().numpy(), wt.grad.cpu().numpy(), keys


@pytest.fixture(scope="module")
def heightfield_grads(ctx):
    w = synth.config1()
    levels = 4
    rng = np.random.default_rng(52)
    weights = rng.uniform(0.5, 2.0, w.num_prims).astype(np.float32)
    g_t, g_w, keys = gpu_tri_forward_backward(ctx, w, levels, weights)
    ref0 = oracle.voxelize_tris(w.tri_verts, w.grid, weights)
    refs = [ref0] + oracle.build_pyramid(ref0, w.grid.resolution, 1, synth.sample_directions(16), num_levels=levels)
    for l in range(levels + 1):
        assert np.array_equal(refs[l]["keys"], keys[l])
    ab = [synth.loss_weights(r["keys"], l) for l, r in enumerate(refs)]
    gm0, gM0 = oracle.broadcast_adjoints(ref0["keys"], [r["keys"] for r in refs], [a for a, _ in ab],
                                         [b for _, b in ab])
    return w, weights, g_t, g_w, ref0["keys"], gm0, gM0


def grid_coords32(w):
    """Grid coordinates as the method computes them (Sec. 3.1 normalisation in FP32):
    U = (p - origin) * (1 / h), each operation rounded to FP32."""
    o = np.asarray(w.grid.origin, np.float32)
    s = np.float32(1.0) / np.float32(w.grid.voxel_size)
    return (w.tri_verts[..., :3].astype(np.float32) - o) * s, float(s)


def test_tri_adjoint_matches_oracle_gradient(heightfield_grads):
    """GPU analytic (reference-domain) gradient against the oracle's complex-step one, both
    taken at the FP32 grid coordinates the method works on (a heightfield triangle almost
    parallel to a voxel plane has a gradient that moves by ~1e-4 relative under the
    ~1e-5-voxel rounding of the normalisation, so the two sides must see the same input)."""
    w, weights, g_t, g_w, keys0, gm0, gM0 = heightfield_grads
    U, s = grid_coords32(w)
    unit = synth.Grid((0.0, 0.0, 0.0), 1.0, w.grid.resolution)
    _, d_u, d_w = oracle.tri_adjoint(U.astype(np.float64), unit, keys0, gm0, gM0, weights=weights)
    d_t = d_u * s
    assert g_t.shape == (w.num_prims, 3, 4)
    assert np.all(g_t[..., 3] == 0.0)
    scale = np.median(np.abs(d_t))
    err = np.abs(g_t[..., :3] - d_t)
    assert np.all(err <= 1e-4 * np.maximum(np.abs(d_t), scale)), err.max()
    ws = np.median(np.abs(d_w))
    assert np.all(np.abs(g_w - d_w) <= 1e-4 * np.maximum(np.abs(d_w), ws))
    _floor_report("vertex xyz", g_t[..., :3], d_t, scale)
    _floor_report("weight", g_w, d_w, ws)


def test_tri_adjoint_finite_differences_heightfield(heightfield_grads):
    """FP64 central FD (h = 1e-4 voxel units) of the heightfield loss, as a function of the
    FP32 grid coordinates, on 64 random vertex coordinates whose stencil keeps every
    clipped polygon's structure."""
    w, weights, g_t, _, keys0, gm0, gM0 = heightfield_grads
    rng = np.random.default_rng(53)
    U, s = grid_coords32(w)
    u64 = U.astype(np.float64)
    unit = synth.Grid((0.0, 0.0, 0.0), 1.0, w.grid.resolution)
    w64 = weights.astype(np.float64)
    h = 1e-4
    checked, kinks, worst, floored, worst_fd = 0, 0, 0.0, 0, 0.0
    while checked < 64:
        assert kinks < 640, "too many stencils cross a kink"
        p, k, i = int(rng.integers(0, u64.shape[0])), int(rng.integers(0, 3)), int(rng.integers(0, 3))
        sig = set()
        for st in (-h, 0.0, h):
            tt = u64.copy(); tt[p, k, i] += st
            sig.add(oracle.tri_clip_signature(tt, unit, [p]))
        if len(sig) != 1:
            kinks += 1
            continue

        def local_loss(step):
            tt = u64.copy(); tt[p, k, i] += step
            return oracle.tri_adjoint(tt, unit, keys0, gm0, gM0, weights=w64, prims=[p])[0]
        fd = (local_loss(h) - local_loss(-h)) / (2 * h)
        _, d_u, _, d_abs = oracle.tri_adjoint(u64, unit, keys0, gm0, gM0, weights=w64, prims=[p], with_abs=True)
        scale = max(abs(fd), 0.01 * d_abs[p, k, i], 1e-3)
        assert abs(d_u[p, k, i] - fd) <= 1e-4 * scale, (p, k, i, d_u[p, k, i], fd)
        err = abs(g_t[p, k, i] / s - fd) / scale
        worst = max(worst, err)
        assert err <= 1e-4, (p, k, i, g_t[p, k, i] / s, fd)
        rel = abs(g_t[p, k, i] / s - fd) / max(abs(fd), 1e-30)
        floored += rel > 1e-4
        worst_fd = max(worst_fd, rel)
        assert rel <= 1e-3, (p, k, i, g_t[p, k, i] / s, fd)
        checked += 1
    print(f"FD checked {checked}, stencils across a kink skipped {kinks}, worst rel {worst:.2e}; "
          f"{floored} within 1e-4 only through the floor, worst relative to |FD| {worst_fd:.2e}")


def _fiber_grads(ctx, ctrl, off, grid, weights, levels):
    """GPU forward, the loss weights of every level, and vx_backward's gradients."""
    c = torch.from_numpy(ctrl).to(DEV)
    o = torch.from_numpy(off).to(DEV)
    wt = torch.from_numpy(weights).to(DEV)
    L0 = ctx.voxelize(grid, ctrl=c, fiber_offsets=o, weights=wt)
    pyr = ctx.build_lod(L0, K=1, num_levels=levels)
    keys = [lv.keys.cpu().numpy().view(np.uint64) for lv in [L0] + pyr]
    ab = [synth.loss_weights(k, l) for l, k in enumerate(keys)]
    gm = [torch.from_numpy(a).to(DEV) for a, _ in ab]
    gM = [torch.from_numpy(b).to(DEV) for _, b in ab]
    g_c, g_w = ctx.backward(grid, ctrl=c, fiber_offsets=o, keys0=L0.keys, grad_mass=gm, grad_moment=gM,
                            weights=wt)
    torch.cuda.synchronize()
    return g_c.cpu().numpy(), g_w.cpu().numpy(), keys, ab


def test_adjoint_windows_match_one_pass(ctx):
    """Windows forced by a low pass limit (several octant windows, each adding its pairs' terms)
    give the gradients of one pass up to the FP64 summation order."""
    w = synth.config2(fibers_per_ply=4, segments=300, R=64, K=1)
    rng = np.random.default_rng(54)
    weights = rng.uniform(0.5, 2.0, w.num_prims).astype(np.float32)
    ref_c, ref_w, _, _ = _fiber_grads(ctx, w.ctrl, w.fiber_offsets, w.grid, weights, 3)
    ctx.set_max_pairs_per_pass(5_000)
    try:
        got_c, got_w, _, _ = _fiber_grads(ctx, w.ctrl, w.fiber_offsets, w.grid, weights, 3)
    finally:
        ctx.set_max_pairs_per_pass(2**31 - 1)
    sc = np.max(np.abs(ref_c))
    assert np.max(np.abs(got_c - ref_c)) <= 1e-6 * sc
    assert np.max(np.abs(got_w - ref_w)) <= 1e-6 * np.max(np.abs(ref_w))


def test_adjoint_at_2048_matches_oracle_gradient(ctx):
    """A 2048^3 grid (the fibers cross the 1024^3 windows' planes): vx_backward, window by
    window, against the oracle's FP64 analytic gradient, tolerance of the 64^3 test."""
    ctrl, off, grid = synth.random_segments(10, 30, 2048, seed=55, radius=(0.3, 1.5), step=(0.5, 2.0))
    # move the walks onto the window corner (1024, 1024, 1024) so that they cross its planes
    shift = np.float32(1024.0 / 2048.0) - ctrl[:, :3].mean(axis=0)
    ctrl = ctrl.copy()
    ctrl[:, :3] += shift
    nseg = synth.fiber_segment_count(off)
    weights = np.random.default_rng(56).uniform(0.5, 2.0, nseg).astype(np.float32)
    g_c, g_w, keys, ab = _fiber_grads(ctx, ctrl, off, grid, weights, 2)
    assert len(np.unique(keys[0] >> np.uint64(30))) > 1          # voxels in several 1024^3 windows
    ref0 = oracle.voxelize_fibers(ctrl, off, grid, weights)
    assert np.array_equal(ref0["keys"], keys[0])
    gm0, gM0 = oracle.broadcast_adjoints(ref0["keys"], keys, [a for a, _ in ab], [b for _, b in ab])
    _, d_ctrl, d_w = oracle.fiber_adjoint(ctrl, off, grid, ref0["keys"], gm0, gM0, weights=weights)
    for got, ref in ((g_c[:, :3], d_ctrl[:, :3]), (g_c[:, 3], d_ctrl[:, 3]), (g_w, d_w)):
        scale = np.median(np.abs(ref))
        assert np.all(np.abs(got - ref) <= 1e-4 * np.maximum(np.abs(ref), scale))
