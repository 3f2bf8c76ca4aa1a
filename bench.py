"""Benchmark: sparse voxelization + full LoD pyramid with SGGX-H (K = 4) of a fiber yarn.

Workload (seeded, synthetic): 3 plies x 64 fibers, each a helical polyline of 4,000
FP32 segments (768,000 capsule primitives, radius 0.004), voxelized into a sparse
512^3 grid with 8^3 sub-cells, then the pyramid down to 1^3 with K = 4 lobes per voxel
and N = 5000 sampled directions per lobe histogram.  One step = vx_voxelize +
vx_build_lod (all levels).  `value` is primitives voxelized per second of the whole
step with the inputs resident on the device; `e2e` is the same metric through the
public API from pinned host buffers, with the input upload and the download of every
level inside the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs an independent replica (the path does not
exchange data between GPUs); value = all ranks' primitives / max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "primitives voxelized/s (voxelize + full LoD build with SGGX-H)"
UNIT = "prims/s"
WORKLOAD = "fiber yarn 3x64 fibers x 4000 segments (768k capsules), 512^3, 8^3 sub-cells, LoD to 1^3, K=4, N=5000"
K_LOBES = 4
N_SAMPLES = 5000
L2_FLUSH_BYTES = 256 << 20
FP32_LANES_PER_SM = 128
N_SMS = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-splines", action="store_true")
    ap.add_argument("--no-heightfield", action="store_true")
    ap.add_argument("--no-sampled", action="store_true")
    ap.add_argument("--woven", type=int, default=16,
                    help="also time the woven patch at 2048^3 with this many warp and weft yarns (16 = the "
                         "full patch, 0 = skip)")
    ap.add_argument("--fibers-per-ply", type=int, default=64,
                    help="smaller yarns for profiling captures (64 = the benchmark workload)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------------
# replicas: every rank runs the whole workload on its own GPU; the job's time is the
# slowest rank's and its throughput counts every rank's primitives
# ----------------------------------------------------------------------------------
def max_over_ranks(x, ws, device):
    """The maximum of x over the ranks of the default process group (x itself when alone)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(ws, prims_per_rank, steps, total_ms):
    """Primitives of all ranks over `steps` steps divided by the slowest rank's time."""
    return ws * prims_per_rank * steps / (total_ms / 1e3)


# ----------------------------------------------------------------------------------
# CPU oracle timings (the reference arm and the cpu_baseline leg)
# ----------------------------------------------------------------------------------
SEGMENTS_PER_PROC = 1000


def usable_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_worker(args):
    """One oracle process: voxelize + full LoD of its fibers (segments, seconds)."""
    ctrl, off, grid, barrier = args
    import oracle
    dirs = synth.sample_directions(N_SAMPLES)
    barrier.wait()
    t = time.perf_counter()
    L0 = oracle.voxelize_fibers(ctrl, off, grid, K=1)
    oracle.build_pyramid(L0, grid.resolution, K_LOBES, dirs)
    return synth.fiber_segment_count(off), time.perf_counter() - t


def time_oracle_parallel(w, procs):
    """The oracle as it stands (single-threaded C) run as `procs` concurrent processes, one
    per usable host core, process p on the first 1,000 segments of fiber p of the yarn:
    voxelize + full LoD with K = 4, N = 5000.  Returns (segments, wall seconds of the slowest
    process, processes).  Processes are spawned (never forked after CUDA is initialised)."""
    import multiprocessing as mp
    mpc = mp.get_context("spawn")
    off = w.fiber_offsets
    procs = max(1, min(procs, len(off) - 1))
    with mpc.Manager() as m:
        barrier = m.Barrier(procs)
        jobs = []
        for p in range(procs):
            c0 = int(off[p])
            jobs.append((w.ctrl[c0: c0 + SEGMENTS_PER_PROC + 1].copy(), np.array([0, SEGMENTS_PER_PROC + 1], np.int64),
                         w.grid, barrier))
        with mpc.Pool(procs) as pool:
            res = pool.map(_oracle_worker, jobs)
    return sum(r[0] for r in res), max(r[1] for r in res), procs


def cpu_sample_text(procs, n, secs):
    return (f"{procs} concurrent oracle processes (one per usable host core), process p on the first "
            f"{SEGMENTS_PER_PROC} segments of fiber p of the same yarn ({n} segments in all), voxelize + full LoD "
            f"K={K_LOBES}, N={N_SAMPLES}, 512^3; single-threaded C oracle per process; wall {secs:.1f} s of the "
            f"slowest")


def cpu_baseline(w, dirs=None):
    n, secs, procs = time_oracle_parallel(w, usable_cores())
    return {"value": n / secs, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": cpu_sample_text(procs, n, secs)}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    w = synth.config2()
    cores = usable_cores()
    for _ in range(args.warmup):
        time_oracle_parallel(w, cores)
    tot, n = 0.0, 0
    procs = 1
    for _ in range(args.steps):
        k, secs, procs = time_oracle_parallel(w, cores)
        tot += secs
        n += k
    value = n / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": cpu_sample_text(procs, n // max(args.steps, 1), tot / max(args.steps, 1)) +
                             " (per step)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None
        # the raw samples: VX_CLOCK_LOG if set, else a file in the temporary directory
        self.path = os.environ.get("VX_CLOCK_LOG") or os.path.join(tempfile.gettempdir(),
                                                                   f"vx_clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.fh, stderr=subprocess.DEVNULL)
            # the sampler's own start (driver and NVML initialisation) stays out of the timed
            # region: wait, at most 3 s, for its first sample before the steps begin
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 3.0 and self.p.poll() is None:
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.02)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.fh.close()
        with open(self.path) as fh:
            return self.summarize(fh)

    @staticmethod
    def summarize(lines):
        """Median SM clock, the maximum clock and the throttle reasons seen active in
        nvidia-smi CSV lines (the FIELDS order); None without a sample."""
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------------
# native arm
# ----------------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import paper_2604_13191_gb300 as vx

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    assert args.warmup >= 3, "at least 3 warm-up steps"

    w = synth.config2(fibers_per_ply=args.fibers_per_ply)
    dirs_np = synth.sample_directions(N_SAMPLES)
    n_prims = w.num_prims
    ctx = vx.Context(dev)
    ctrl = torch.from_numpy(w.ctrl).to(dev)
    off = torch.from_numpy(w.fiber_offsets).to(dev)
    dirs = torch.from_numpy(dirs_np).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step():
        L0 = ctx.voxelize(w.grid, ctrl=ctrl, fiber_offsets=off, num_prims=n_prims)
        pyr = ctx.build_lod(L0, K=K_LOBES, dirs=dirs)
        return L0, pyr

    for _ in range(args.warmup):
        out = step()
    torch.cuda.synchronize()
    levels = [out[0]] + out[1]
    level_sizes = [lv.num_voxels for lv in levels]
    pairs_hint = None
    del out, levels

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- timed region: device-resident inputs --------------------------------------
    clocks = ClockSampler(torch.cuda.current_device())
    ctx.profile(True)
    clocks.start()
    barrier()
    t_ms = []
    for _ in range(args.steps):
        flush.fill_(1)                       # L2 flush between timed steps (outside the events)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        res = step()
        b.record()
        torch.cuda.synchronize()
        t_ms.append(a.elapsed_time(b))
        del res
    barrier()
    clk = clocks.stop()
    prof = ctx.profile_read()
    ctx.profile(False)
    total_ms = max_over_ranks(sum(t_ms), ws, dev)
    value = replica_throughput(ws, n_prims, args.steps, total_ms)
    launches = sum(v[0] for v in prof.values())
    prof = {k: v for k, v in prof.items() if v[0]}

    # ---- vx_voxelize alone on a warm stream: median of 10 calls -----------------------------
    vox_ms = []
    for _ in range(10):
        flush.fill_(1)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        L0 = ctx.voxelize(w.grid, ctrl=ctrl, fiber_offsets=off, num_prims=n_prims)
        b.record()
        torch.cuda.synchronize()
        vox_ms.append(a.elapsed_time(b))
        del L0
    voxelize = {"median_ms": statistics.median(vox_ms), "prims_per_s": n_prims / (statistics.median(vox_ms) * 1e-3),
                "calls": len(vox_ms)}

    # ---- e2e: same calls from pinned host buffers, outputs downloaded ------------------
    e2e = None
    if not args.no_e2e:
        h_ctrl = torch.from_numpy(w.ctrl).pin_memory()
        h_off = torch.from_numpy(w.fiber_offsets).pin_memory()
        h_dirs = torch.from_numpy(dirs_np).pin_memory()
        L0, pyr = step()
        sizes = [lv.block.numel() for lv in [L0] + pyr]
        del L0, pyr
        h_out = torch.empty(sum(sizes) + 4096 * len(sizes), dtype=torch.uint8).pin_memory()
        h2d = h_ctrl.numel() * 4 + h_off.numel() * 8 + h_dirs.numel() * 4
        side = torch.cuda.Stream(dev)
        level_done = [torch.cuda.Event() for _ in sizes[1:]]

        def e2e_step():
            c = h_ctrl.to(dev, non_blocking=True)
            o = h_off.to(dev, non_blocking=True)
            d = h_dirs.to(dev, non_blocking=True)
            L0 = ctx.voxelize(w.grid, ctrl=c, fiber_offsets=o, num_prims=n_prims)
            # level 0 downloads on a second stream while the pyramid is built from it
            done0 = torch.cuda.Event()
            done0.record()
            n0 = L0.block.numel()
            with torch.cuda.stream(side):
                side.wait_event(done0)
                h_out[0: n0].copy_(L0.block, non_blocking=True)
            # every coarser level downloads on the second stream as soon as it is complete
            pyr = ctx.build_lod(L0, K=K_LOBES, dirs=d, events=level_done)
            pos, nbytes = n0, n0
            with torch.cuda.stream(side):
                for lv, ev in zip(pyr, level_done):
                    side.wait_event(ev)
                    n = lv.block.numel()
                    h_out[pos: pos + n].copy_(lv.block, non_blocking=True)
                    pos += n
                    nbytes += n
            torch.cuda.synchronize()
            return nbytes

        for _ in range(2):
            e2e_step()
        barrier()
        e_ms = []
        d2h = 0
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d2h = e2e_step()
            e_ms.append(1e3 * (time.perf_counter() - t0))
        barrier()
        etot = max_over_ranks(sum(e_ms), ws, dev)
        # this box's device-to-host rate, for reading the e2e time (one level-0 download alone,
        # after the timed steps)
        L0x = ctx.voxelize(w.grid, ctrl=ctrl, fiber_offsets=off, num_prims=n_prims)
        torch.cuda.synchronize()
        nx = L0x.block.numel()
        ta = time.perf_counter()
        h_out[0: nx].copy_(L0x.block, non_blocking=True)
        torch.cuda.synchronize()
        d2h_gbs = nx / (time.perf_counter() - ta) / 1e9
        del L0x
        e2e = {"value": replica_throughput(ws, n_prims, args.steps, etot), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": etot / args.steps, "d2h_gbs": d2h_gbs,
               "note": "inputs uploaded from pinned host memory, every level downloaded to pinned host "
                       "memory on a second stream: level 0 while the pyramid is built, every coarser level "
                       "once its event (vx_build_lod_events) is recorded"}

    # ---- batched path vs per-instance plain calls (64 instances of uneven size) ------------
    batched = None
    if not args.no_batched:
        batched = batched_vs_plain(ctx, dev, args.steps, dirs)

    # ---- the woven patch at 2048^3 (optional) ---------------------------------------------
    woven = None
    if args.woven > 0:
        woven = woven_patch(ctx, dev, args.woven, dirs)

    # ---- the triangle path (heightfields) ----------------------------------------------------
    heightfield = None
    if not args.no_heightfield:
        heightfield = heightfield_record(ctx, dev, args.steps)

    # ---- spline input (Catmull-Rom nodes tessellated on the device) --------------------------
    splines = None
    if not args.no_splines:
        splines = spline_fibers(ctx, dev, args.steps, dirs)

    # ---- the paper's sample-based level 0 against the exact one -----------------------------
    sampled = None
    if not args.no_sampled:
        sampled = sampled_vs_exact(ctx, dev, args.steps)

    # ---- adjoint vs forward on the differentiation workload ---------------------------------
    adjoint = None
    if not args.no_adjoint:
        adjoint = adjoint_vs_forward(ctx, dev, args.steps)

    # ---- roofline of the dominant kernel -------------------------------------------------
    roof = roofline(prof, w, level_sizes, args.steps)

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline(w)
    stages = {k: {"launches": v[0] // args.steps, "ms_per_step": v[1] / args.steps,
                  "units_per_step": v[2] // args.steps}
              for k, v in prof.items() if v[0]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.fibers_per_ply == 64 else
                   f"{WORKLOAD} [profiling variant: {args.fibers_per_ply} fibers per ply]", "prims": n_prims, "resolution": w.grid.resolution,
                   "K": K_LOBES, "n_samples": N_SAMPLES, "levels": len(level_sizes),
                   "voxels_per_level": level_sizes, "parallelism": f"replicas x{ws}",
                   "l2": "flushed between timed steps (256 MiB write)",
                   "timing": "the timed steps carry a CUDA event pair around every library launch (the "
                             "stage times and the roofline's launch durations); e2e runs without them"},
        "lod_ms": sum(v["ms_per_step"] for k, v in stages.items() if k.startswith(("lod", "sggx"))),
        "voxelize": voxelize,
        "stages": stages,
        "gpu_launches": int(launches),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "batched": batched,
        "heightfield": heightfield,
        "splines": splines,
        "sampled": sampled,
        "adjoint": adjoint,
    }
    if woven is not None:
        line["woven"] = woven
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ----------------------------------------------------------------------------------
ADJ_WORKLOAD = ("yarn 3x64 fibers x 4000 segments (768k capsules) at 256^3, level 0 + 4 LoD levels (K=1); "
                "loss = sum of U(-1,1) weights times every level's m and M")
BATCH_WORKLOAD = ("64 instances: 32 heightfields of 2k-2M triangles and 32 yarn patches of 10k-4M "
                  "segments (log-uniform), grids 64^3-1024^3, all LoD levels, K=4, N=5000")


def batched_vs_plain(ctx, dev, steps, dirs):
    """One graph replay of the batched path against a loop of plain vx_voxelize +
    vx_build_lod calls over the same instances (same GPU, CUDA events), K = 4 on every
    level; the plan's groups and the launch shapes its autotuner picked are reported."""
    import torch
    ws = synth.config4(seed=4, n_instances=64)
    insts = []
    for w in ws:
        if w.kind == "triangles":
            insts.append({"kind": "triangles", "grid": w.grid, "tri_verts": torch.from_numpy(w.tri_verts).to(dev)})
        else:
            insts.append({"kind": "fibers", "grid": w.grid, "ctrl": torch.from_numpy(w.ctrl).to(dev),
                          "fiber_offsets": torch.from_numpy(w.fiber_offsets).to(dev),
                          "num_prims": w.num_prims})
    nprims = sum(w.num_prims for w in ws)
    t0 = time.perf_counter()
    b = ctx.batch(insts, K=K_LOBES, dirs=dirs)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    plan = b.query()

    def run_batch():
        b.run()

    def run_plain():
        outs = []
        for inst in insts:
            if inst["kind"] == "triangles":
                L0 = ctx.voxelize(inst["grid"], tri_verts=inst["tri_verts"])
            else:
                L0 = ctx.voxelize(inst["grid"], ctrl=inst["ctrl"], fiber_offsets=inst["fiber_offsets"],
                                  num_prims=inst["num_prims"])
            outs.append((L0, ctx.build_lod(L0, K=K_LOBES, dirs=dirs)))
        return outs

    def timed(fn, n):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(n):
            fn()
        e.record()
        torch.cuda.synchronize()
        return a.elapsed_time(e) / n

    tb = timed(run_batch, steps)
    tp = timed(run_plain, steps)
    # kernels per replay: the kernel nodes of the captured graph (the library's launch count)
    ctx.profile(True)
    b.run()
    torch.cuda.synchronize()
    graph_kernels = ctx.profile_read().get("batched_graph", (0, 0.0, 0))[0]
    ctx.profile(False)
    b.close()
    for k in plan.values():
        k.pop("cluster_ms", None)
    return {"workload": BATCH_WORKLOAD, "prims": int(nprims),
            "triangles": int(sum(w.num_prims for w in ws if w.kind == "triangles")),
            "segments": int(sum(w.num_prims for w in ws if w.kind == "fibers")),
            "batched_ms": tb, "plain_ms": tp, "speedup": tp / tb, "batched_prims_per_s": nprims / (tb * 1e-3),
            "plan_s": plan_s, "plan": plan, "graph_kernels": int(graph_kernels),
            "note": "batched = one captured graph per run (groups of instances whose pairs fit one pass, run in "
                    "sequence per kind, the two kinds on two branches); plain = per-instance vx_voxelize + "
                    "vx_build_lod; plan_s includes the autotuner's timing runs"}


VOX_STAGES = ("prep", "candidates_count", "candidates_emit", "scan", "sort_hist", "sort_scatter", "segment_heads",
              "reduce_fibers", "reduce_tris", "finalize")
LOD_STAGES = ("lod_counts", "lod_heads", "lod_reduce", "sggx_cluster")


def woven_patch(ctx, dev, n_yarns, dirs, window_log2=9, steps=2):
    """The woven patch (n_yarns warp x n_yarns weft yarns of 3 x 80 fibers, 2,000 segments
    per span, r = 0.002) at 2048^3 with K = 4, through vx_voxelize_lod_windowed (512^3
    windows: the pyramid of the full patch does not fit in device memory at once).  Each
    window's levels are handed to a callback that drops them.  One warm-up step, `steps`
    timed steps (CUDA events around the call), then one step with per-stage event timing
    for the voxelize / LoD split; peak device memory from torch's allocator."""
    import torch
    import paper_2604_13191_gb300 as vx
    w = synth.config3(n_yarns=n_yarns)
    ctrl = torch.from_numpy(w.ctrl).to(dev)
    off = torch.from_numpy(w.fiber_offsets).to(dev)
    info = {"windows": 0, "voxels": [0] * window_log2}
    # a context of its own, so that the peak below includes the workspace the call grows
    ctx = vx.Context(dev)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats(dev)
    base = torch.cuda.memory_allocated(dev)

    def on_window(win, levels):
        info["windows"] += 1
        for l, lv in enumerate(levels):
            info["voxels"][l] += lv.num_voxels

    def step():
        info["windows"] = 0
        info["voxels"] = [0] * window_log2
        top = ctx.voxelize_lod_windowed(w.grid, window_log2=window_log2, on_window=on_window, K=K_LOBES, dirs=dirs,
                                        ctrl=ctrl, fiber_offsets=off, num_prims=w.num_prims)
        return info["voxels"] + [t.num_voxels for t in top]

    step()
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        sizes = step()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    peak = torch.cuda.max_memory_allocated(dev) - base
    ctx.profile(True)
    step()
    prof = ctx.profile_read()
    ctx.profile(False)
    ctx.close()
    vox_ms = sum(prof[k][1] for k in VOX_STAGES if k in prof)
    lod_ms = sum(prof[k][1] for k in LOD_STAGES if k in prof)
    pairs = prof.get("reduce_fibers", (0, 0.0, 0))[2]
    t = statistics.mean(ms)
    return {"workload": f"woven patch {n_yarns}x{n_yarns} yarns x 3 plies x 80 fibers x 2000 segments "
                        f"({w.num_prims} capsules, r = 0.002), 2048^3, K=4, N=5000, windows of "
                        f"{1 << window_log2}^3 (vx_voxelize_lod_windowed, every window's levels dropped by the "
                        f"callback)",
            "prims": int(w.num_prims), "ms_per_step": t, "prims_per_s": w.num_prims / (t * 1e-3),
            "voxelize_ms": vox_ms, "lod_ms": lod_ms, "stage_split_note": "device time of the library's "
            "voxelize and LoD stages in one extra step with per-launch event timing",
            "windows": info["windows"], "candidate_pairs": int(pairs), "voxels_per_level": sizes,
            "peak_device_bytes": int(peak), "peak_note": "device memory the call held at its peak (levels, "
            "workspace), over the inputs already resident", "steps": steps}


def heightfield_record(ctx, dev, steps):
    """The triangle path: vx_voxelize + vx_build_lod (K = 1) of the config-1 heightfield
    (64 x 64 vertices, 7,938 triangles, 128^3) and of a 1024 x 1024-vertex heightfield
    (2,093,058 triangles, the largest size of the batching workload) at 1024^3; CUDA events
    over `steps` steps after 2 warm-up steps, per-stage device times from one profiled step;
    k_reduce_tris's pairs per second (its pipe and issue fractions are ncu counters, in the
    profile summary of that kernel)."""
    import torch
    out = {}
    for name, n, R in (("config1_128", 64, 128), ("hf1024_1024", 1024, 1024)):
        tris = synth.heightfield(n, 1)
        grid = synth.Grid((0.0, 0.0, -0.5), 1.0 / R, R)
        tv = torch.from_numpy(tris).to(dev)

        def step():
            L0 = ctx.voxelize(grid, tri_verts=tv)
            pyr = ctx.build_lod(L0, K=1)
            return L0, pyr
        for _ in range(2):
            step()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            L0, pyr = step()
        e.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(e) / steps
        nvox = L0.num_voxels
        del L0, pyr
        ctx.profile(True)
        step()
        prof = ctx.profile_read()
        ctx.profile(False)
        red = prof.get("reduce_tris", (0, 0.0, 0))
        lod_ms = sum(prof[k][1] for k in LOD_STAGES if k in prof)
        vox_ms = sum(prof[k][1] for k in VOX_STAGES if k in prof)
        out[name] = {"triangles": int(tris.shape[0]), "resolution": R, "ms_per_step": ms,
                     "prims_per_s": tris.shape[0] / (ms * 1e-3), "voxelize_ms": vox_ms, "lod_ms": lod_ms,
                     "level0_voxels": int(nvox), "candidate_pairs": int(red[2]), "reduce_tris_ms": red[1],
                     "reduce_tris_pairs_per_s": red[2] / (red[1] * 1e-3) if red[1] > 0 else None}
    out["note"] = ("voxelize + full LoD K=1; stage times from one extra step with per-launch event timing; "
                   "k_reduce_tris's FP32-pipe and issue fractions are ncu counters "
                   "(profiles/k_reduce_tris_heightfield.md)")
    return out


def spline_fibers(ctx, dev, steps, dirs):
    """Spline input: the bench yarn's fibers given as Catmull-Rom splines through every 10th
    node (401 nodes per fiber), tessellated on the device with 10 points per span (the same
    768k capsules), then vx_voxelize + vx_build_lod, K = 4; CUDA events."""
    import torch
    w = synth.config2()
    off = w.fiber_offsets
    keep = [np.arange(off[f], off[f + 1], 10) for f in range(len(off) - 1)]
    nodes = torch.from_numpy(np.concatenate([w.ctrl[k] for k in keep]).astype(np.float32)).to(dev)
    noff = torch.from_numpy(np.concatenate([[0], np.cumsum([len(k) for k in keep])]).astype(np.int64)).to(dev)
    S = 10
    tess, total = [], []
    for i in range(steps + 2):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        m = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        ctrl, coff = ctx.tessellate_catmull_rom(nodes, noff, S)
        m.record()
        L0 = ctx.voxelize(w.grid, ctrl=ctrl, fiber_offsets=coff)
        pyr = ctx.build_lod(L0, K=K_LOBES, dirs=dirs)
        b.record()
        torch.cuda.synchronize()
        if i >= 2:
            tess.append(a.elapsed_time(m))
            total.append(a.elapsed_time(b))
        n_caps = int(ctrl.shape[0] - (coff.shape[0] - 1))
        del L0, pyr, ctrl, coff
    return {"workload": "the bench yarn as Catmull-Rom splines: 192 fibers x 401 nodes, 10 points per span "
                        "(768k capsules), 512^3, K=4, N=5000",
            "nodes": int(nodes.shape[0]), "subdiv": S, "prims": n_caps, "tessellate_ms": statistics.mean(tess),
            "ms_per_step": statistics.mean(total), "prims_per_s": n_caps / (statistics.mean(total) * 1e-3)}


def sampled_vs_exact(ctx, dev, steps, samples=8):
    """The paper's sample-based level 0 (axis samples per segment, Sec. 3.2-3.3) against the
    exact level 0 on the bench yarn: time, and occupancy / voxel / mass totals relative to the
    exact path (CUDA events; totals by tensor sums)."""
    import torch
    w = synth.config2()
    ctrl = torch.from_numpy(w.ctrl).to(dev)
    off = torch.from_numpy(w.fiber_offsets).to(dev)
    ms = []
    for i in range(steps + 2):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        Ls = ctx.voxelize_sampled(w.grid, ctrl=ctrl, fiber_offsets=off, samples=samples, num_prims=w.num_prims)
        b.record()
        torch.cuda.synchronize()
        if i >= 2:
            ms.append(a.elapsed_time(b))
        if i < steps + 1:
            del Ls
    Le = ctx.voxelize(w.grid, ctrl=ctrl, fiber_offsets=off, num_prims=w.num_prims)
    occ_s = int(Ls.occ.to(torch.int64).sum())
    occ_e = int(Le.occ.to(torch.int64).sum())
    out = {"workload": f"the bench yarn (768k capsules) at 512^3, {samples} axis samples per segment",
           "samples_per_segment": samples, "ms": statistics.mean(ms),
           "prims_per_s": w.num_prims / (statistics.mean(ms) * 1e-3),
           "voxels": int(Ls.num_voxels), "voxels_exact": int(Le.num_voxels),
           "occupied_subcells_ratio": occ_s / max(occ_e, 1),
           "mass_ratio": float(Ls.mass.double().sum() / Le.mass.double().sum())}
    del Ls, Le
    return out


def adjoint_vs_forward(ctx, dev, steps):
    """The differentiation workload: the yarn at 256^3 with 4 LoD levels (K = 1); forward
    (vx_voxelize + vx_build_lod) against the adjoint (vx_backward: level adjoints broadcast
    to level 0, candidate pairs recomputed, FP64 per-pair derivatives), CUDA events."""
    import torch
    w = synth.config5()
    ctrl = torch.from_numpy(w.ctrl).to(dev)
    off = torch.from_numpy(w.fiber_offsets).to(dev)
    L0 = ctx.voxelize(w.grid, ctrl=ctrl, fiber_offsets=off, num_prims=w.num_prims)
    pyr = ctx.build_lod(L0, K=1, num_levels=w.levels)
    gen = torch.Generator(device="cpu").manual_seed(5)
    gm = [torch.rand(lv.num_voxels, generator=gen).mul_(2).sub_(1).to(dev) for lv in [L0] + pyr]
    gM = [torch.rand(lv.num_voxels, 6, generator=gen).mul_(2).sub_(1).to(dev) for lv in [L0] + pyr]
    keys0 = L0.keys.clone()

    def fwd():
        a = ctx.voxelize(w.grid, ctrl=ctrl, fiber_offsets=off, num_prims=w.num_prims)
        return a, ctx.build_lod(a, K=1, num_levels=w.levels)

    def bwd():
        return ctx.backward(w.grid, ctrl=ctrl, fiber_offsets=off, keys0=keys0, grad_mass=gm, grad_moment=gM,
                            num_prims=w.num_prims)

    def timed(fn, n):
        # the median of three timed blocks of n calls (one disturbed block does not set it)
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        blocks = []
        for _ in range(3):
            a = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(n):
                fn()
            e.record()
            torch.cuda.synchronize()
            blocks.append(a.elapsed_time(e) / n)
        return sorted(blocks)[1], blocks

    tf, tf_blocks = timed(fwd, steps)
    tb, tb_blocks = timed(bwd, steps)
    return {"workload": ADJ_WORKLOAD, "prims": int(w.num_prims), "forward_ms": tf, "backward_ms": tb,
            "backward_over_forward": tb / tf, "forward_blocks_ms": tf_blocks, "backward_blocks_ms": tb_blocks,
            "timing": "median of three blocks of the step count, CUDA events"}


def _source_hash(name):
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_2604_13191_gb300", "csrc", name), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]


# FP32 operations the definition spends per unit of work:
#   reduce_fibers: per (pair, sub-cell) decision, the step-1/2 tests on precomputed per-axis
#     terms, each x^2 against r^2 - (y^2 + z^2): 3 x (2 adds + 1 compare) = 9, plus the
#     per-axis terms amortised (~1) -> 10
#   sggx_cluster: per sampled direction: mat-vec 9 (3 multiplies, 6 fused), squares and norm
#     5, thresholds 2, compares 6, reciprocal 1, scale 1, off-diagonal products 3, fused
#     product-roundings 6, integer sums 12 -> 45
ALU_OPS = {"reduce_fibers": 512 * 10, "sggx_cluster": N_SAMPLES * 45}
# algorithmic HBM bytes per unit of work
HBM_BYTES = {
    "sort_scatter": 16,          # per pair and pass: key + value read and written
    "sort_hist": 4,              # per pair and pass: key read
    "candidates_emit": 8 + 32,   # per pair written + the primitive record read (per pair upper)
    "finalize": 100 + 140,       # per candidate voxel read + written
}


def roofline(prof, w, level_sizes, steps):
    """Dominant stage by device time; achieved = algorithmic work per launch / average
    launch time (CUDA events on the launching stream, over the timed region)."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    clk_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = N_SMS * FP32_LANES_PER_SM * clk_mhz * 1e6 / 1e12    # Tops/s, FP32 lanes x clock
    stage, (nl, ms, units) = max(prof.items(), key=lambda kv: kv[1][1])
    avg_ms = ms / max(nl, 1)
    units_per_launch = units / max(nl, 1)
    traffic = None
    issue = None   # ncu's issue-slot figures of the same capture (ALU-bound kernels)
    tfile = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if os.path.exists(tfile):
        try:
            t = json.load(open(tfile))
            ent = t.get(stage)
            if ent and ent.get("source_hash") == _source_hash(ent["source"]):
                traffic = ent["bytes_per_launch"] * units_per_launch / ent["units_per_launch"]
                if "issue_active" in ent:
                    issue = {"issue_active": ent["issue_active"],
                             "lanes_active_per_inst": ent.get("lanes_active_per_inst"),
                             "alu_pipe_active": ent.get("alu_pipe_active"),
                             "source": "ncu capture of the same kernel source (profiles/ncu_traffic.json)"}
        except Exception:
            traffic = None
            issue = None
    if stage in ALU_OPS:
        ops = units_per_launch * ALU_OPS[stage]
        ach = ops / (avg_ms * 1e-3) / 1e12
        return {"kernel": stage, "bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "Tops/s",
                "frac": ach / alu_peak, "traffic": traffic, "avg_launch_ms": avg_ms,
                "launches_per_step": nl // steps, "units_per_launch": units_per_launch,
                "ops_per_unit": ALU_OPS[stage], "issue_slots": issue,
                "ops_note": "ops_per_unit counts the definition's FP32 operations (512 sub-cell tests of 10 "
                            "operations per pair); the kernel skips most of them with exact group tests, so "
                            "issue_slots says how busy the SM is",
                "peak_source": f"152 SMs x 128 FP32 lanes x {clk_mhz:.0f} MHz (max SM clock, MEASURED_PEAKS)"}
    per_unit = HBM_BYTES.get(stage)
    ach = None if per_unit is None else units_per_launch * per_unit / (avg_ms * 1e-3) / 1e9
    return {"kernel": stage, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
            "frac": None if ach is None else ach / hbm, "traffic": traffic, "avg_launch_ms": avg_ms,
            "launches_per_step": nl // steps, "units_per_launch": units_per_launch,
            "peak_source": "hbm_gbs of MEASURED_PEAKS (copy)"}


if __name__ == "__main__":
    main()
