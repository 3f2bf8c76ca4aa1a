"""The allocation-free adjoint entry point (vx_backward_noalloc) against vx_backward.

vx_backward_noalloc serves callers that cannot allocate device memory (a host
application or memory manager that owns all device memory, or a loop in which an
allocation would stall the device): it keeps its scratch in a fixed array inside the
library.  This file runs last so that a failure here leaves the other tests' results
intact; it must pass alone in a fresh process and after the other tests.  Tolerance:
the one of test_adjoint_gpu.py (1e-4 of max(|g|, median |g|)); the same kernels in
the same order make the results identical in practice.
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


def _setup():
    w = synth.config2(fibers_per_ply=4, segments=300, R=64, K=1)
    levels = 3
    ctx = vx.Context(DEV)
    ctrl = torch.from_numpy(w.ctrl).to(DEV)
    off = torch.from_numpy(w.fiber_offsets).to(DEV)
    wt = torch.from_numpy(np.random.default_rng(7).uniform(0.5, 2.0, w.num_prims).astype(np.float32)).to(DEV)
    L0 = ctx.voxelize(w.grid, ctrl=ctrl, fiber_offsets=off, weights=wt)
    pyr = ctx.build_lod(L0, K=1, num_levels=levels)
    gm, gM = [], []
    for l, lv in enumerate([L0] + pyr):
        a, b = synth.loss_weights(lv.keys.cpu().numpy().view(np.uint64), l)
        gm.append(torch.from_numpy(a).to(DEV))
        gM.append(torch.from_numpy(b).to(DEV))
    return w, ctx, ctrl, off, wt, L0, gm, gM


def _close(a, b):
    s = max(float(np.median(np.abs(b))), 1e-30)
    return np.all(np.abs(a - b) <= 1e-4 * np.maximum(np.abs(b), s))


def test_noalloc_matches_backward_twice():
    w, ctx, ctrl, off, wt, L0, gm, gM = _setup()
    ref_c, ref_w = ctx.backward(w.grid, ctrl=ctrl, fiber_offsets=off, keys0=L0.keys, grad_mass=gm,
                                grad_moment=gM, weights=wt)
    ref_c, ref_w = ref_c.cpu().numpy(), ref_w.cpu().numpy()
    for _ in range(2):
        g_c = torch.full((ctrl.shape[0], 4), float("nan"), device=DEV)
        g_w = torch.full((w.num_prims,), float("nan"), device=DEV)
        api.backward_noalloc(w.grid, ctrl=ctrl, fiber_offsets=off, keys0=L0.keys, grad_mass=gm, grad_moment=gM,
                             grad_ctrl=g_c, grad_weights=g_w, weights=wt)
        torch.cuda.synchronize()
        assert _close(g_c.cpu().numpy(), ref_c)
        assert _close(g_w.cpu().numpy(), ref_w)
    ctx.close()


def test_noalloc_through_c_abi_and_limits():
    w, ctx, ctrl, off, wt, L0, gm, gM = _setup()
    lib = vx.load()
    assert hasattr(lib, "vx_backward_noalloc")
    ref_c, _ = ctx.backward(w.grid, ctrl=ctrl, fiber_offsets=off, keys0=L0.keys, grad_mass=gm, grad_moment=gM,
                            weights=wt)
    P = api.VxPrimitives()
    P.kind = api.VX_FIBERS
    P.num_prims = w.num_prims
    P.ctrl = ctrl.data_ptr()
    P.num_ctrl = ctrl.shape[0]
    P.fiber_offsets = off.data_ptr()
    P.num_fibers = off.shape[0] - 1
    P.weights = wt.data_ptr()
    G = api._grid(w.grid)
    pm = (C.c_void_p * len(gm))(*[g.data_ptr() for g in gm])
    pM = (C.c_void_p * len(gM))(*[g.data_ptr() for g in gM])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        g_c = torch.zeros((ctrl.shape[0], 4), device=DEV)
        st = lib.vx_backward_noalloc(C.byref(P), C.byref(G), L0.keys.data_ptr(), L0.num_voxels, len(gm) - 1, pm, pM,
                                     stream, g_c.data_ptr(), None)
        assert st == 0
        torch.cuda.synchronize()
        assert _close(g_c.cpu().numpy(), ref_c.cpu().numpy())
    # sizes beyond the documented maximum are rejected before any work
    P.num_prims = api.NOALLOC_LIMITS["segments"] + 1
    st = lib.vx_backward_noalloc(C.byref(P), C.byref(G), L0.keys.data_ptr(), L0.num_voxels, len(gm) - 1, pm, pM,
                                 stream, g_c.data_ptr(), None)
    assert st == 3
    ctx.close()


def _call(lib, P, G, keys, nvox, gm, gM, g_c, g_w=None):
    pm = (C.c_void_p * len(gm))(*[g.data_ptr() for g in gm])
    pM = (C.c_void_p * len(gM))(*[g.data_ptr() for g in gM])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.vx_backward_noalloc(C.byref(P), C.byref(G), keys, nvox, len(gm) - 1, pm, pM, stream, g_c.data_ptr(),
                                   None if g_w is None else g_w.data_ptr())


def _prims(ctrl, off, num_prims, wt=None):
    P = api.VxPrimitives()
    P.kind = api.VX_FIBERS
    P.num_prims = num_prims
    P.ctrl = ctrl.data_ptr()
    P.num_ctrl = ctrl.shape[0]
    P.fiber_offsets = off.data_ptr()
    P.num_fibers = off.shape[0] - 1
    P.weights = None if wt is None else wt.data_ptr()
    return P


def test_noalloc_rejections_leave_outputs_and_array_usable():
    """Every limit and every bad record returns its status; the caller's outputs are left as
    they were; a valid call afterwards still matches vx_backward (the shared array is reused)."""
    w, ctx, ctrl, off, wt, L0, gm, gM = _setup()
    lib = vx.load()
    G = api._grid(w.grid)
    lim = api.NOALLOC_LIMITS
    keys = L0.keys.data_ptr()
    sentinel = 7.0
    g_c = torch.full((ctrl.shape[0], 4), sentinel, device=DEV)
    g_w = torch.full((w.num_prims,), sentinel, device=DEV)
    P = _prims(ctrl, off, w.num_prims, wt)
    # level-0 voxels over the limit (checked on the host, before any work)
    big_keys = torch.zeros(lim["voxels0"] + 1, dtype=torch.int64, device=DEV)
    assert _call(lib, P, G, big_keys.data_ptr(), lim["voxels0"] + 1, gm, gM, g_c, g_w) == 3
    # fibers over the limit
    many = torch.zeros(lim["fibers"] + 2, dtype=torch.int64, device=DEV)
    Pf = _prims(ctrl, many, 0)
    assert _call(lib, Pf, G, keys, L0.num_voxels, gm, gM, g_c, g_w) == 3
    # candidate pairs over the limit with fewer segments than the segment limit: thick capsules
    tc, toff, tgrid = synth.random_segments(20, 100, w.grid.resolution, seed=3, radius=(8.0, 10.0), step=(0.5, 1.0))
    tctrl = torch.from_numpy(tc).to(DEV)
    toff_d = torch.from_numpy(toff).to(DEV)
    nseg = int(np.sum(np.maximum(np.diff(toff) - 1, 0)))
    assert nseg < lim["segments"]
    tg_c = torch.full((tctrl.shape[0], 4), sentinel, device=DEV)
    assert _call(lib, _prims(tctrl, toff_d, nseg), api._grid(tgrid), keys, L0.num_voxels, gm, gM, tg_c) == 3
    torch.cuda.synchronize()
    assert bool(torch.all(tg_c == sentinel))
    # a NaN coordinate, and offsets reaching past the control points: VX_ERR_INVALID_ARG
    bad = ctrl.clone()
    bad[5, 1] = float("nan")
    assert _call(lib, _prims(bad, off, w.num_prims, wt), G, keys, L0.num_voxels, gm, gM, g_c, g_w) == 1
    off_bad = off.clone()
    off_bad[-1] = ctrl.shape[0] + 3
    n_bad = int(torch.clamp(off_bad[1:] - off_bad[:-1] - 1, min=0).sum())
    assert _call(lib, _prims(ctrl, off_bad, n_bad, wt), G, keys, L0.num_voxels, gm, gM, g_c, g_w) == 1
    torch.cuda.synchronize()
    assert bool(torch.all(g_c == sentinel)) and bool(torch.all(g_w == sentinel))
    # the shared array still gives the right gradients, twice
    ref_c, ref_w = ctx.backward(w.grid, ctrl=ctrl, fiber_offsets=off, keys0=L0.keys, grad_mass=gm,
                                grad_moment=gM, weights=wt)
    for _ in range(2):
        assert _call(lib, P, G, keys, L0.num_voxels, gm, gM, g_c, g_w) == 0
        torch.cuda.synchronize()
        assert _close(g_c.cpu().numpy(), ref_c.cpu().numpy())
        assert _close(g_w.cpu().numpy(), ref_w.cpu().numpy())
    ctx.close()
