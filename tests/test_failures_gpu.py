"""Failure paths of the C ABI driven from the host: an allocator that runs out of memory
after a byte budget (VX_ERR_OUT_OF_MEMORY), no block leaked, the context usable afterwards.

The failure is made on the host (the allocator callback returns NULL); nothing faults the GPU.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2604_13191_gb300 as vx  # noqa: E402
from paper_2604_13191_gb300 import api  # noqa: E402

DEV = torch.device("cuda", 0)


class BudgetAllocator(api._TorchAllocator):
    """torch's caching allocator behind a budget on the bytes ever allocated: the allocation
    that would pass the budget, and every later one, returns NULL, as an exhausted device
    would."""

    def __init__(self, device, budget):
        super().__init__(device)
        self.budget = budget
        self.total = 0
        self.refused = 0

    def _alloc(self, ctx, nbytes, stream):
        if self.total + int(nbytes) > self.budget:
            self.refused += 1
            return None
        self.total += int(nbytes)
        return super()._alloc(ctx, nbytes, stream)


def _context(budget):
    ctx = vx.Context.__new__(vx.Context)
    ctx.lib = vx.load()
    ctx.device = DEV
    ctx.alloc = BudgetAllocator(DEV, budget)
    h = C.c_void_p()
    assert ctx.lib.vx_context_create(C.byref(ctx.alloc.struct), C.byref(h)) == 0
    ctx.h = h
    return ctx


def _run(ctx, w, ctrl, off, dirs):
    L0 = ctx.voxelize(w.grid, ctrl=ctrl, fiber_offsets=off)
    pyr = ctx.build_lod(L0, K=4, dirs=dirs)
    torch.cuda.synchronize()
    return [L0] + pyr


@pytest.mark.parametrize("frac", [0.02, 0.3, 0.6, 0.9, 0.99])
def test_out_of_memory_is_reported_and_recoverable(frac, dirs5000):
    """The allocator fails part-way through voxelize + build_lod (at a point set by frac of
    the bytes the two calls allocate): VX_ERR_OUT_OF_MEMORY, nothing leaked, and the same
    context then gives the reference result bit for bit."""
    w = synth.config2(fibers_per_ply=4, segments=300, R=64, K=4)
    ctrl = torch.from_numpy(w.ctrl).to(DEV)
    off = torch.from_numpy(w.fiber_offsets).to(DEV)
    dirs = torch.from_numpy(dirs5000).to(DEV)
    probe = _context(1 << 50)
    ref = _run(probe, w, ctrl, off, dirs)
    need = probe.alloc.total

    ctx = _context(int(frac * need))
    with pytest.raises(vx.VxError) as e:
        _run(ctx, w, ctrl, off, dirs)
    assert e.value.status == 2 and ctx.alloc.refused > 0
    # the same context, given memory again, gives the reference result bit for bit
    ctx.alloc.budget = 1 << 50
    got = _run(ctx, w, ctrl, off, dirs)
    for a, b in zip(got, ref):
        ha, hb = a.host(), b.host()
        for k in ("keys", "mask", "mass", "moment", "occ", "proj", "lobe_count", "lobes"):
            assert np.array_equal(ha[k], hb[k]), k
    del got, ref
    ctx.close()
    probe.close()
    # vx_context_destroy returns the workspace; a level block lost by a failed call would remain
    assert not ctx.alloc.live, f"{len(ctx.alloc.live)} blocks still held after vx_context_destroy"
    assert not probe.alloc.live


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """The device waits of the sort's copy pipeline are bounded.  A wait on a barrier that no
    copy completes must give up (VX_ERR_TIMEOUT) rather than hang; afterwards the same
    context voxelizes as before."""
    ctx = vx.Context(DEV)
    w = synth.config2(fibers_per_ply=2, segments=200, R=64, K=1)
    ctrl = torch.from_numpy(w.ctrl).to(DEV)
    off = torch.from_numpy(w.fiber_offsets).to(DEV)
    ref = ctx.voxelize(w.grid, ctrl=ctrl, fiber_offsets=off).host()
    for polls in (1, 64, 4096):
        st = ctx.lib.vx_selftest_bounded_wait(ctx.h, polls, api._stream(None))
        assert st == 5, st                       # VX_ERR_TIMEOUT
    assert ctx.lib.vx_selftest_bounded_wait(ctx.h, 0, api._stream(None)) == 1
    got = ctx.voxelize(w.grid, ctrl=ctrl, fiber_offsets=off).host()
    for k in ("keys", "mask", "mass", "moment"):
        assert np.array_equal(got[k], ref[k])
    ctx.close()


def test_build_lod_events_rejects_bad_event_arguments():
    """vx_build_lod_events checks its event arguments before any work: a negative count, or
    no array for a positive count, is VX_ERR_INVALID_ARG with nothing allocated; an empty
    list of events gives the result of vx_build_lod."""
    ctx = vx.Context(DEV)
    w = synth.config2(fibers_per_ply=2, segments=200, R=64, K=1)
    L0 = ctx.voxelize(w.grid, ctrl=torch.from_numpy(w.ctrl).to(DEV),
                      fiber_offsets=torch.from_numpy(w.fiber_offsets).to(DEV))
    prm = api.VxLodParams()
    prm.num_levels, prm.K, prm.n_samples, prm.merge = 0, 1, 0, 0
    outs = (api.VxLevel * 8)()
    live = len(ctx.alloc.live)
    for arr, n in ((None, 2), (None, -1), ((C.c_void_p * 1)(), -3)):
        st = ctx.lib.vx_build_lod_events(ctx.h, C.byref(L0._c), C.byref(prm), api._stream(None), outs, arr, n)
        assert st == 1, (n, st)
    assert len(ctx.alloc.live) == live
    ref = [p.host() for p in ctx.build_lod(L0, K=1)]
    got = [p.host() for p in ctx.build_lod(L0, K=1, events=[])]
    assert len(ref) == len(got)
    for a, b in zip(ref, got):
        for k in ("keys", "mask", "mass", "moment", "occ", "proj", "lobe_count", "lobes"):
            assert np.array_equal(a[k], b[k]), k
    ctx.close()
