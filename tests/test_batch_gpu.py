"""Batched path (vx_batch_*): every instance's levels equal the plain path's on that
instance alone, bit for bit (K = 1 and K = 4 with SGGX-H), on the first run and on graph
replays; an overflow of the planned capacities is reported, not written past."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2604_13191_gb300 as vx  # noqa: E402

DEV = torch.device("cuda", 0)
FIELDS = ("keys", "mask", "mass", "moment", "occ", "proj", "lobe_count", "lobes", "compact")


def instances(seed=4, n=12):
    ws = synth.config4(seed=seed, n_instances=n, min_tris=200, max_tris=20000, min_segs=500, max_segs=30000)
    out = []
    for w in ws:
        if w.kind == "triangles":
            out.append({"kind": "triangles", "grid": w.grid, "tri_verts": torch.from_numpy(w.tri_verts).to(DEV)})
        else:
            out.append({"kind": "fibers", "grid": w.grid, "ctrl": torch.from_numpy(w.ctrl).to(DEV),
                        "fiber_offsets": torch.from_numpy(w.fiber_offsets).to(DEV)})
    return out


def plain(ctx, inst, K=1, dirs=None):
    if inst["kind"] == "triangles":
        L0 = ctx.voxelize(inst["grid"], tri_verts=inst["tri_verts"])
    else:
        L0 = ctx.voxelize(inst["grid"], ctrl=inst["ctrl"], fiber_offsets=inst["fiber_offsets"])
    pyr = ctx.build_lod(L0, K=K, dirs=dirs)
    torch.cuda.synchronize()
    return [L0.host()] + [p.host() for p in pyr]


def check_batch(ctx, b, insts, K=1, dirs=None):
    for i, inst in enumerate(insts):
        ref = plain(ctx, inst, K, dirs)
        for l, r in enumerate(ref):
            g = b.level(i, l).host()
            for f in FIELDS:
                assert np.array_equal(np.asarray(g[f]).view(np.uint8), np.asarray(r[f]).view(np.uint8)), (i, l, f)


def test_batch_matches_plain_instances():
    ctx = vx.Context(DEV)
    insts = instances()
    b = ctx.batch(insts)
    b.run()
    check_batch(ctx, b, insts)
    b.run()          # graph replay
    b.run()
    check_batch(ctx, b, insts)
    b.close()
    ctx.close()


def test_batch_capacity_overflow_is_reported():
    ctx = vx.Context(DEV)
    insts = [i for i in instances(seed=5, n=4) if i["kind"] == "fibers"]
    b = ctx.batch(insts, headroom=0.0)
    b.run()
    b.level(0, 0)
    # thicker fibers produce more candidate pairs than planned
    b.keep[0][:, 3] *= 4.0
    b.run()
    with pytest.raises(vx.VxError) as e:
        b.level(0, 0)
    assert e.value.status == 3
    b.close()
    ctx.close()


def test_batch_with_sggx_h_matches_plain_instances(dirs5000):
    """K = 4: every level above 0 clustered with SGGX-H inside the captured graph."""
    ctx = vx.Context(DEV)
    insts = instances(seed=6, n=8)
    dirs = torch.from_numpy(dirs5000).to(DEV)
    b = ctx.batch(insts, K=4, dirs=dirs)
    b.run()
    check_batch(ctx, b, insts, K=4, dirs=dirs)
    b.run()          # graph replay
    check_batch(ctx, b, insts, K=4, dirs=dirs)
    assert any(int(b.level(i, 1).lobe_count.max()) > 1 for i in range(len(insts)))
    b.close()
    ctx.close()


def _oracle_instances():
    """Two heightfields (512 and 2,048 triangles at 64^3 and 128^3) and two yarn patches
    (1,200 and 1,080 segments, fibers 1.5 voxels thick, at 64^3 and 32^3): sizes the oracle
    finishes in seconds, with clustered parents at every level above 0."""
    ws = []
    for n, R, seed in ((17, 64, 1), (33, 128, 2)):
        ws.append(synth.Workload(f"hf{n}", "triangles", synth.Grid((0.0, 0.0, -0.5), 1.0 / R, R),
                                 tri_verts=synth.heightfield(n, seed), K=1))
    for fpp, segs, R, seed in ((2, 200, 64, 3), (3, 120, 32, 4)):
        c, o = synth.yarn(3, fpp, segs, fiber_radius=1.5 / R, seed=seed)
        ws.append(synth.Workload(f"yarn{fpp}", "fibers", synth.Grid((0.0, 0.0, 0.0), 1.0 / R, R), ctrl=c,
                                 fiber_offsets=o, K=1))
    return ws


def _as_instance(w):
    if w.kind == "triangles":
        return {"kind": "triangles", "grid": w.grid, "tri_verts": torch.from_numpy(w.tri_verts).to(DEV)}
    return {"kind": "fibers", "grid": w.grid, "ctrl": torch.from_numpy(w.ctrl).to(DEV),
            "fiber_offsets": torch.from_numpy(w.fiber_offsets).to(DEV)}


@pytest.mark.parametrize("K,which", [(1, (0, 3)), (4, (0, 1, 2, 3))])
def test_batch_matches_oracle(K, which, dirs5000):
    """Each batched instance against the CPU oracle directly (not through the plain CUDA
    path): keys, masks, occupancy, projections and the FP32 sums bit-exact, the FP64
    tolerance of the parity tests, and the SGGX-H lobes within 1e-5 (K = 4)."""
    import oracle
    from test_parity_gpu import compare_level, prim_measure_max
    ws = [_oracle_instances()[i] for i in which]
    ctx = vx.Context(DEV)
    dirs = torch.from_numpy(dirs5000).to(DEV) if K > 1 else None
    b = ctx.batch([_as_instance(w) for w in ws], K=K, dirs=dirs)
    refs = []
    for w in ws:
        ref0 = oracle.voxelize(w, K=1)
        refs.append([ref0] + oracle.build_pyramid(ref0, w.grid.resolution, K, dirs5000))
    for rep in range(2):      # first run, then a graph replay
        b.run()
        torch.cuda.synchronize()
        for i, w in enumerate(ws):
            for l, r in enumerate(refs[i]):
                compare_level(b.level(i, l).host(), r, f"{w.name} K={K} level {l} run {rep}",
                              mu_max=prim_measure_max(w))
    b.close()
    ctx.close()


@pytest.mark.parametrize("K", [1, 4])
def test_batch_groups_by_pass_limit(K, dirs5000):
    """With a per-pass pair limit below a kind's total, its instances run as several
    consecutive groups sharing one set of pair buffers; every instance still equals the plain
    path bit for bit, on the first run and on a replay.  An instance that alone is over the
    limit is reported (VX_ERR_CAPACITY)."""
    ctx = vx.Context(DEV)
    insts = instances(seed=7, n=10)
    dirs = torch.from_numpy(dirs5000).to(DEV) if K > 1 else None
    ref = vx.Context(DEV)
    refs = [plain(ref, inst, K, dirs) for inst in insts]
    whole = ctx.batch(insts, K=K, dirs=dirs).query()
    total = max(whole["fibers"]["max_group_pairs"], whole["triangles"]["max_group_pairs"])
    assert whole["fibers"]["groups"] == 1 and whole["triangles"]["groups"] == 1
    b = None
    for frac in (0.8, 0.65, 0.5):
        ctx.set_max_pairs_per_pass(int(frac * total))
        try:
            b = ctx.batch(insts, K=K, dirs=dirs)
        except vx.VxError as e:          # one instance over this limit: try a larger one
            assert e.status == 3
            continue
        break
    assert b is not None
    q = b.query()
    assert max(q["fibers"]["groups"], q["triangles"]["groups"]) > 1, q
    for _ in range(2):
        b.run()
        for i in range(len(insts)):
            for l, r in enumerate(refs[i]):
                g = b.level(i, l).host()
                for f in FIELDS:
                    assert np.array_equal(np.asarray(g[f]).view(np.uint8), np.asarray(r[f]).view(np.uint8)), (i, l, f)
    b.close()
    ctx.set_max_pairs_per_pass(20_000)
    with pytest.raises(vx.VxError) as e:
        ctx.batch(insts, K=K, dirs=dirs)
    assert e.value.status == 3
    ctx.close()
    ref.close()


def test_batch_autotuner_records_its_choices(dirs5000):
    """The plan times every candidate launch shape on its own data and keeps the fastest:
    the reduce grid per kind and the clustering tier per level (K = 4)."""
    ctx = vx.Context(DEV)
    insts = instances(seed=6, n=8)
    b = ctx.batch(insts, K=4, dirs=torch.from_numpy(dirs5000).to(DEV))
    q = b.query()
    for kind in ("triangles", "fibers"):
        r = q[kind]
        assert r["groups"] == 1 and r["max_group_pairs"] > 0
        assert len(r["reduce_ms"]) == 5 and all(v > 0 for v in r["reduce_ms"].values())
        assert r["reduce_ms"][r["reduce_blocks_per_sm"]] == min(r["reduce_ms"].values())
        assert r["cluster_tier"] and all(t in (0, 1, 2) for t in r["cluster_tier"].values())
        for l, t in r["cluster_tier"].items():
            assert r["cluster_ms"][l][t] == min(r["cluster_ms"][l])
    print(q)
    b.close()
    ctx.close()
