"""The C-ABI library builds, loads without a GPU and exports every declared entry point;
the ctypes mirrors of the structs match the header's layout (checked with a C compiler)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vx.h")


def declared_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"VX_API\s+[\w\s\*]+?\b(vx_\w+)\s*\(", txt)))


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("vx_voxelize", "vx_build_lod", "vx_context_create", "vx_context_destroy",
              "vx_level_release", "vx_status_string", "vx_last_cuda_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2604_13191_gb300 import _build
    lib_path = _build.build()
    lib = C.CDLL(lib_path)
    for n in declared_functions():
        assert hasattr(lib, n), f"{n} declared in vx.h but not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (vx_\w+)", out))
    assert exported == set(declared_functions())


def test_status_strings_without_gpu():
    import paper_2604_13191_gb300 as vx
    lib = vx.load()
    for s in range(7):
        assert lib.vx_status_string(s)
    assert b"unknown" in lib.vx_status_string(99)


def test_ctypes_layout_matches_header():
    gcc = "gcc"
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "vx.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("vx_grid %zu\n", sizeof(vx_grid));
  printf("vx_primitives %zu\n", sizeof(vx_primitives));
  printf("vx_level %zu\n", sizeof(vx_level));
  printf("vx_lod_params %zu\n", sizeof(vx_lod_params));
  printf("vx_allocator %zu\n", sizeof(vx_allocator));
  printf("vx_window %zu\n", sizeof(vx_window));
  printf("vx_batch_info %zu\n", sizeof(vx_batch_info));
  P(vx_batch_info, cluster_ms) P(vx_batch_info, reduce_ms)
  P(vx_window, log2_size) P(vx_window, index)
  P(vx_primitives, weights) P(vx_primitives, fiber_offsets) P(vx_level, compact) P(vx_level, block)
  P(vx_level, num_voxels) P(vx_lod_params, dirs) P(vx_lod_params, merge) P(vx_grid, resolution)
  return 0;
}
"""
    from paper_2604_13191_gb300 import api
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(src, "w").write(prog)
        subprocess.check_call([gcc, "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        got = dict(line.split() for line in subprocess.check_output([exe], text=True).splitlines())
    assert int(got["vx_grid"]) == C.sizeof(api.VxGrid)
    assert int(got["vx_primitives"]) == C.sizeof(api.VxPrimitives)
    assert int(got["vx_level"]) == C.sizeof(api.VxLevel)
    assert int(got["vx_lod_params"]) == C.sizeof(api.VxLodParams)
    assert int(got["vx_allocator"]) == C.sizeof(api.VxAllocator)
    assert int(got["vx_window"]) == C.sizeof(api.VxWindow)
    assert int(got["vx_batch_info"]) == C.sizeof(api.VxBatchInfo)
    assert int(got["vx_batch_info.cluster_ms"]) == api.VxBatchInfo.cluster_ms.offset
    assert int(got["vx_batch_info.reduce_ms"]) == api.VxBatchInfo.reduce_ms.offset
    assert int(got["vx_window.log2_size"]) == api.VxWindow.log2_size.offset
    assert int(got["vx_window.index"]) == api.VxWindow.index.offset
    assert int(got["vx_primitives.weights"]) == api.VxPrimitives.weights.offset
    assert int(got["vx_primitives.fiber_offsets"]) == api.VxPrimitives.fiber_offsets.offset
    assert int(got["vx_level.compact"]) == api.VxLevel.compact.offset
    assert int(got["vx_level.block"]) == api.VxLevel.block.offset
    assert int(got["vx_level.num_voxels"]) == api.VxLevel.num_voxels.offset
    assert int(got["vx_lod_params.dirs"]) == api.VxLodParams.dirs.offset
    assert int(got["vx_lod_params.merge"]) == api.VxLodParams.merge.offset
    assert int(got["vx_grid.resolution"]) == api.VxGrid.resolution.offset


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2604_13191_gb300")
    for dp, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "vxoracle" not in txt


def test_merge_mode_names():
    from paper_2604_13191_gb300 import api
    assert api._merge_mode("pooled") == 0 and api._merge_mode("mass") == 1
    with pytest.raises(ValueError):
        api._merge_mode("median")


def test_new_entry_points_reject_bad_arguments_without_gpu():
    """Argument checks that return before any device work (NULL context or level)."""
    import paper_2604_13191_gb300 as vx
    lib = vx.load()
    assert lib.vx_export_compact8(None, None, None) == 1                 # VX_ERR_INVALID_ARG
    n = C.c_int64(5)
    assert lib.vx_export_leaves(None, None, None, None, None, C.byref(n), None) == 1
    assert lib.vx_tessellate_catmull_rom(None, None, None, 0, 0, 1, None, None, None) == 1
    assert lib.vx_voxelize_sampled(None, None, None, 4, None, None) == 1


def test_backward_noalloc_checks_output_shapes_before_any_call():
    """The allocation-free adjoint writes num_ctrl * 16 bytes into grad_ctrl and num_prims * 4
    into grad_weights: a buffer of the wrong shape, type or layout is refused on the host."""
    import torch

    from paper_2604_13191_gb300 import api
    import synth
    w = synth.config2(fibers_per_ply=2, segments=20, R=32, K=1)
    ctrl = torch.from_numpy(w.ctrl)
    off = torch.from_numpy(w.fiber_offsets)
    keys = torch.zeros(4, dtype=torch.int64)
    gm, gM = [torch.zeros(4)], [torch.zeros(4, 6)]
    good_w = torch.zeros(w.num_prims)
    kw = dict(ctrl=ctrl, fiber_offsets=off, keys0=keys, grad_mass=gm, grad_moment=gM)
    with pytest.raises(ValueError, match="grad_ctrl"):
        api.backward_noalloc(w.grid, grad_ctrl=torch.zeros(ctrl.shape[0] - 1, 4), **kw)
    with pytest.raises(ValueError, match="grad_ctrl"):
        api.backward_noalloc(w.grid, grad_ctrl=torch.zeros(4, ctrl.shape[0]).t(), **kw)
    with pytest.raises(TypeError, match="grad_ctrl"):
        api.backward_noalloc(w.grid, grad_ctrl=torch.zeros(ctrl.shape[0], 4, dtype=torch.float64), **kw)
    with pytest.raises(ValueError, match="grad_weights"):
        api.backward_noalloc(w.grid, grad_ctrl=torch.zeros(ctrl.shape[0], 4),
                             grad_weights=torch.zeros(w.num_prims + 1), **kw)
    with pytest.raises(ValueError, match="grad_weights"):
        api.backward_noalloc(w.grid, grad_ctrl=torch.zeros(ctrl.shape[0], 4),
                             grad_weights=torch.zeros(2 * w.num_prims)[::2], **kw)
    with pytest.raises(TypeError, match="grad"):
        api.backward_noalloc(w.grid, ctrl=ctrl, fiber_offsets=off, keys0=keys, grad_mass=[torch.zeros(4).double()],
                             grad_moment=gM, grad_ctrl=torch.zeros(ctrl.shape[0], 4), grad_weights=good_w)
    # well-formed buffers get as far as the device check (no GPU here)
    with pytest.raises(ValueError, match="CUDA"):
        api.backward_noalloc(w.grid, grad_ctrl=torch.zeros(ctrl.shape[0], 4), grad_weights=good_w, **kw)
