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
