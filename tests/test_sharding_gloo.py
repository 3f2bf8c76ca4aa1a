"""Sharding by Morton tile ranges, emulated with two gloo ranks on CPU (oracle only).

The grid's octants are aligned blocks of Morton keys, so a parent never has children in two
octants.  Each rank voxelizes the octants it owns and builds its pyramid up to the octant's
root level (one voxel per octant) on its own; the only exchange is an all-gather of those
root records, from which the remaining levels are built.  The result must equal the
single-process pyramid bit for bit, SGGX-H lobes included.  The GPU library runs replicas
(one box, one GPU); this checks that the decomposition it would shard along is exact.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
R = 32                  # grid resolution; octants are 16^3, their roots are level 4
OCT_SHIFT = 12          # key >> 12 = octant (3 bits per level, 4 levels below the octant root)
K = 4
FIELDS = ("keys", "mask", "mass", "moment", "mass64", "moment64", "occ", "proj", "lobe_count", "lobes", "compact")


def _workload():
    sys.path.insert(0, ROOT)
    import synth
    ctrl, off, grid = synth.random_segments(10, 14, R, seed=31, radius=(0.3, 1.5), step=(0.8, 3.0))
    return synth.Workload("shard", "fibers", grid, ctrl=ctrl, fiber_offsets=off, K=1)


def _subset(level, sel):
    out = dict(level)
    for f in FIELDS:
        if f in level and hasattr(level[f], "shape") and level[f].shape[:1] == level["keys"].shape[:1]:
            out[f] = level[f][sel]
    return out


def _concat(levels):
    out = dict(levels[0])
    for f in FIELDS:
        if f in out and hasattr(out[f], "shape"):
            out[f] = np.concatenate([lv[f] for lv in levels])
    return out


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    w = _workload()
    dirs = synth.sample_directions(600)
    full0 = oracle.voxelize(w)
    # this rank's octants: a contiguous range of Morton keys
    octs = (full0["keys"] >> np.uint64(OCT_SHIFT)).astype(np.int64)
    mine = (octs * ws) // 8 == rank
    cur = _subset(full0, mine)
    local = [cur]
    for _ in range(4):                      # levels 1..4 stay inside the octants
        cur = oracle.lod_step(cur, K, dirs)
        local.append(cur)
    # the one exchange: every rank's octant roots (level 4)
    roots = [None] * ws
    dist.all_gather_object(roots, local[-1])
    top = [_concat([r for r in roots if r["keys"].shape[0] > 0])]
    top.append(oracle.lod_step(top[0], K, dirs))      # level 5: the 1^3 root
    out[rank] = {"local": local, "top": top}
    dist.barrier()
    dist.destroy_process_group()


def test_octant_shards_with_one_gather_equal_the_whole_pyramid():
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    w = _workload()
    dirs = synth.sample_directions(600)
    whole = [oracle.voxelize(w)] + oracle.build_pyramid(oracle.voxelize(w), R, K, dirs)
    # levels 0..4: the ranks' local levels, concatenated in rank (= Morton) order
    for lvl in range(5):
        parts = [res[r]["local"][lvl] for r in range(ws)]
        assert all(p["keys"].shape[0] > 0 for p in parts), "both ranks must own voxels"
        got = _concat(parts)
        for f in ("keys", "mask", "mass", "moment", "occ", "proj", "lobe_count", "lobes", "compact"):
            assert np.array_equal(np.asarray(got[f]).view(np.uint8), np.asarray(whole[lvl][f]).view(np.uint8)), \
                (lvl, f)
    # levels 4 (gathered) and 5, identical on both ranks and to the whole pyramid
    for r in range(ws):
        for lvl, top in zip((4, 5), res[r]["top"]):
            for f in ("keys", "mask", "mass", "moment", "lobe_count", "lobes"):
                assert np.array_equal(np.asarray(top[f]).view(np.uint8), np.asarray(whole[lvl][f]).view(np.uint8)), \
                    (r, lvl, f)
    assert (whole[4]["lobe_count"] > 1).any() or (whole[3]["lobe_count"] > 1).any()
