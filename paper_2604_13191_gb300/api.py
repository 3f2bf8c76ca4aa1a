"""Thin Python binding of the C ABI in include/vx.h (argument marshalling only).

Every step of the voxelization / LoD path runs in the CUDA library libvx.so; this
module passes device pointers of torch tensors, supplies torch's caching allocator as
the library's allocator, and wraps the returned level blocks as typed tensor views.
There is no CPU fallback: if the library cannot be loaded the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import torch

from . import _build

VX_TRIANGLES, VX_FIBERS = 0, 1
STATUS = {0: "VX_OK", 1: "VX_ERR_INVALID_ARG", 2: "VX_ERR_OUT_OF_MEMORY", 3: "VX_ERR_CAPACITY",
          4: "VX_ERR_CUDA", 5: "VX_ERR_TIMEOUT", 6: "VX_ERR_UNSUPPORTED"}


class VxError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class VxGrid(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("voxel_size", C.c_float), ("resolution", C.c_uint32),
                ("sub_res", C.c_uint32)]


class VxPrimitives(C.Structure):
    _fields_ = [("kind", C.c_int32), ("num_prims", C.c_int64), ("tri_verts", C.c_void_p),
                ("ctrl", C.c_void_p), ("num_ctrl", C.c_int64), ("fiber_offsets", C.c_void_p),
                ("num_fibers", C.c_int64), ("weights", C.c_void_p)]


class VxLevel(C.Structure):
    _fields_ = [("level", C.c_int32), ("resolution", C.c_int32), ("num_voxels", C.c_int64),
                ("K", C.c_int32), ("block", C.c_void_p), ("keys", C.c_void_p), ("mask", C.c_void_p),
                ("mass", C.c_void_p), ("moment", C.c_void_p), ("occ", C.c_void_p),
                ("occ_proj", C.c_void_p), ("lobe_count", C.c_void_p), ("lobes", C.c_void_p),
                ("compact", C.c_void_p)]


class VxLodParams(C.Structure):
    _fields_ = [("num_levels", C.c_int32), ("K", C.c_int32), ("n_samples", C.c_int32),
                ("merge", C.c_int32), ("dirs", C.c_void_p)]


class VxWindow(C.Structure):
    _fields_ = [("lo", C.c_int32 * 3), ("log2_size", C.c_int32), ("index", C.c_int64)]


WINDOW_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(VxWindow), C.POINTER(VxLevel), C.c_int, C.c_void_p)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class VxAllocator(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN)]


EXPORTS = ["vx_context_create", "vx_context_destroy", "vx_voxelize", "vx_build_lod",
           "vx_level_release", "vx_status_string", "vx_last_cuda_error", "vx_profile_enable",
           "vx_profile_read", "vx_backward", "vx_backward_noalloc", "vx_batch_create", "vx_batch_run",
           "vx_batch_level", "vx_batch_destroy", "vx_set_max_pairs_per_pass", "vx_batch_create_lod",
           "vx_export_compact8", "vx_tessellate_catmull_rom", "vx_voxelize_sampled", "vx_export_leaves",
           "vx_voxelize_lod_windowed", "vx_batch_query", "vx_selftest_bounded_wait", "vx_build_lod_events"]


class VxInstance(C.Structure):
    _fields_ = [("kind", C.c_int32), ("grid", VxGrid), ("prim_begin", C.c_int64), ("num_prims", C.c_int64),
                ("fiber_begin", C.c_int64), ("num_fibers", C.c_int64)]


class VxBatchInfo(C.Structure):
    _fields_ = [("num_groups", C.c_int32 * 2), ("max_group_pairs", C.c_int64 * 2),
                ("reduce_blocks_per_sm", C.c_int32 * 2), ("reduce_candidates", (C.c_int32 * 5) * 2),
                ("reduce_ms", (C.c_float * 5) * 2), ("cluster_tier", (C.c_int32 * 12) * 2),
                ("cluster_ms", ((C.c_float * 3) * 12) * 2)]


class VxStageTime(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("total_ms", C.c_double),
                ("units", C.c_int64)]

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> C.CDLL:
    """Loads libvx.so (building it in-tree first if needed and nvcc exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"CUDA library not built: {_build.LIB} (run __graft_entry__.build())")
        lib = C.CDLL(_build.LIB)
        P = C.c_void_p
        lib.vx_context_create.restype = C.c_int
        lib.vx_context_create.argtypes = [C.POINTER(VxAllocator), C.POINTER(C.c_void_p)]
        lib.vx_context_destroy.restype = None
        lib.vx_context_destroy.argtypes = [P]
        lib.vx_voxelize.restype = C.c_int
        lib.vx_voxelize.argtypes = [P, C.POINTER(VxPrimitives), C.POINTER(VxGrid), P, C.POINTER(VxLevel)]
        lib.vx_build_lod.restype = C.c_int
        lib.vx_build_lod.argtypes = [P, C.POINTER(VxLevel), C.POINTER(VxLodParams), P, C.POINTER(VxLevel)]
        lib.vx_build_lod_events.restype = C.c_int
        lib.vx_build_lod_events.argtypes = [P, C.POINTER(VxLevel), C.POINTER(VxLodParams), P, C.POINTER(VxLevel),
                                            C.POINTER(C.c_void_p), C.c_int]
        lib.vx_level_release.restype = None
        lib.vx_level_release.argtypes = [P, C.POINTER(VxLevel), P]
        lib.vx_status_string.restype = C.c_char_p
        lib.vx_status_string.argtypes = [C.c_int]
        lib.vx_last_cuda_error.restype = C.c_char_p
        lib.vx_last_cuda_error.argtypes = [P]
        lib.vx_profile_enable.restype = C.c_int
        lib.vx_profile_enable.argtypes = [P, C.c_int]
        lib.vx_set_max_pairs_per_pass.restype = C.c_int
        lib.vx_set_max_pairs_per_pass.argtypes = [P, C.c_int64]
        lib.vx_profile_read.restype = C.c_int
        lib.vx_profile_read.argtypes = [P, C.POINTER(VxStageTime), C.c_int, C.POINTER(C.c_int)]
        lib.vx_backward.restype = C.c_int
        lib.vx_backward.argtypes = [P, C.POINTER(VxPrimitives), C.POINTER(VxGrid), P, C.c_int64, C.c_int,
                                    C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), P, P, P]
        lib.vx_batch_create_lod.restype = C.c_int
        lib.vx_batch_create_lod.argtypes = [P, C.POINTER(VxPrimitives), C.POINTER(VxPrimitives),
                                            C.POINTER(VxInstance), C.c_int, C.POINTER(VxLodParams), C.c_float, P,
                                            C.POINTER(C.c_void_p)]
        lib.vx_batch_create.restype = C.c_int
        lib.vx_batch_create.argtypes = [P, C.POINTER(VxPrimitives), C.POINTER(VxPrimitives), C.POINTER(VxInstance),
                                        C.c_int, C.c_float, P, C.POINTER(C.c_void_p)]
        lib.vx_batch_run.restype = C.c_int
        lib.vx_batch_run.argtypes = [P, P]
        lib.vx_batch_level.restype = C.c_int
        lib.vx_batch_level.argtypes = [P, C.c_int, C.c_int, P, C.POINTER(VxLevel)]
        lib.vx_selftest_bounded_wait.restype = C.c_int
        lib.vx_selftest_bounded_wait.argtypes = [P, C.c_int, P]
        lib.vx_batch_query.restype = C.c_int
        lib.vx_batch_query.argtypes = [P, C.POINTER(VxBatchInfo)]
        lib.vx_batch_destroy.restype = None
        lib.vx_batch_destroy.argtypes = [P]
        lib.vx_export_leaves.restype = C.c_int
        lib.vx_export_leaves.argtypes = [P, C.POINTER(VxLevel), P, P, P, C.POINTER(C.c_int64), P]
        lib.vx_voxelize_sampled.restype = C.c_int
        lib.vx_voxelize_sampled.argtypes = [P, C.POINTER(VxPrimitives), C.POINTER(VxGrid), C.c_int, P,
                                            C.POINTER(VxLevel)]
        lib.vx_tessellate_catmull_rom.restype = C.c_int
        lib.vx_tessellate_catmull_rom.argtypes = [P, P, P, C.c_int64, C.c_int64, C.c_int, P, P, P]
        lib.vx_export_compact8.restype = C.c_int
        lib.vx_export_compact8.argtypes = [C.POINTER(VxLevel), P, P]
        lib.vx_voxelize_lod_windowed.restype = C.c_int
        lib.vx_voxelize_lod_windowed.argtypes = [P, C.POINTER(VxPrimitives), C.POINTER(VxGrid),
                                                 C.POINTER(VxLodParams), C.c_int, WINDOW_FN, P, P,
                                                 C.POINTER(VxLevel), C.POINTER(C.c_int)]
        lib.vx_backward_noalloc.restype = C.c_int
        lib.vx_backward_noalloc.argtypes = [C.POINTER(VxPrimitives), C.POINTER(VxGrid), P, C.c_int64, C.c_int,
                                            C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), P, P, P]
        _lib = lib
        return lib


class _TorchAllocator:
    """Device memory for the library from torch's caching allocator (current stream)."""

    def __init__(self, device):
        self.device = device
        self.live = {}
        self._a = ALLOC_FN(self._alloc)
        self._f = FREE_FN(self._free)
        self.struct = VxAllocator(None, self._a, self._f)

    def _alloc(self, ctx, nbytes, stream):
        try:
            t = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        except Exception:      # out of memory: the library reports VX_ERR_OUT_OF_MEMORY
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ctx, p, stream):
        self.live.pop(p, None)

    def take(self, p):
        return self.live.pop(p, None)


@dataclass
class Level:
    """One pyramid level: typed views of a block owned by this object."""
    level: int
    resolution: int
    num_voxels: int
    K: int
    keys: torch.Tensor        # int64 [n] (Morton keys, bit pattern of uint64)
    mask: torch.Tensor        # int64 [n, 8] (bit patterns of uint64 words)
    mass: torch.Tensor        # float32 [n]
    moment: torch.Tensor      # float32 [n, 6]
    occ: torch.Tensor         # int16 [n] (uint16 values <= 512)
    occ_proj: torch.Tensor    # uint8 [n, 3]
    lobe_count: torch.Tensor  # uint8 [n]
    lobes: torch.Tensor       # float32 [n, K, 7]
    compact: torch.Tensor     # float32 [n, K, 6]
    block: torch.Tensor
    _c: VxLevel

    def host(self) -> dict:
        """Copies every array to host numpy arrays (uint64 views restored)."""
        import numpy as np
        d = {}
        for k in ("keys", "mask", "mass", "moment", "occ", "occ_proj", "lobe_count", "lobes", "compact"):
            d[k] = getattr(self, k).cpu().numpy()
        d["keys"] = d["keys"].view(np.uint64)
        d["mask"] = d["mask"].view(np.uint64)
        d["occ"] = d["occ"].view(np.uint16)
        d["proj"] = d.pop("occ_proj")
        d["K"] = self.K
        return d


def _view(block: torch.Tensor, base: int, ptr: int, nbytes: int, dtype, shape):
    off = ptr - base
    return block[off: off + nbytes].view(dtype).view(*shape)


class Context:
    """A library context (allocator + reusable device workspace) on one CUDA device."""

    def __init__(self, device=None):
        self.lib = load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.alloc = _TorchAllocator(self.device)
        h = C.c_void_p()
        st = self.lib.vx_context_create(C.byref(self.alloc.struct), C.byref(h))
        if st != 0:
            raise VxError(st, "vx_context_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.vx_context_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_max_pairs_per_pass(self, max_pairs: int):
        """vx_set_max_pairs_per_pass: candidate pairs per voxelization pass (windows over
        the limit are split into octants; the outputs do not change)."""
        st = self.lib.vx_set_max_pairs_per_pass(self.h, int(max_pairs))
        if st != 0:
            raise self._err(st, "vx_set_max_pairs_per_pass")

    def profile(self, enable: bool = True):
        """vx_profile_enable: per-launch CUDA-event timing of every library kernel."""
        st = self.lib.vx_profile_enable(self.h, 1 if enable else 0)
        if st != 0:
            raise self._err(st, "vx_profile_enable")

    def profile_read(self) -> dict:
        """vx_profile_read: {stage: (launches, total device ms, work units)} (synchronises)."""
        n = C.c_int()
        buf = (VxStageTime * 64)()
        st = self.lib.vx_profile_read(self.h, buf, 64, C.byref(n))
        if st != 0:
            raise self._err(st, "vx_profile_read")
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms), int(buf[i].units))
                for i in range(n.value)}

    def _err(self, st, what):
        detail = self.lib.vx_last_cuda_error(self.h).decode() if st == 4 else ""
        return VxError(st, what, detail)

    def _wrap(self, L: VxLevel) -> Level:
        n, K = int(L.num_voxels), int(L.K)
        block = self.alloc.take(L.block)
        if block is None:
            raise RuntimeError("level block was not allocated through this context")
        base = block.data_ptr()
        return Level(
            level=int(L.level), resolution=int(L.resolution), num_voxels=n, K=K,
            keys=_view(block, base, L.keys, n * 8, torch.int64, (n,)),
            mask=_view(block, base, L.mask, n * 64, torch.int64, (n, 8)),
            mass=_view(block, base, L.mass, n * 4, torch.float32, (n,)),
            moment=_view(block, base, L.moment, n * 24, torch.float32, (n, 6)),
            occ=_view(block, base, L.occ, n * 2, torch.int16, (n,)),
            occ_proj=_view(block, base, L.occ_proj, n * 3, torch.uint8, (n, 3)),
            lobe_count=_view(block, base, L.lobe_count, n, torch.uint8, (n,)),
            lobes=_view(block, base, L.lobes, n * K * 28, torch.float32, (n, K, 7)),
            compact=_view(block, base, L.compact, n * K * 24, torch.float32, (n, K, 6)),
            block=block, _c=L)

    def voxelize(self, grid, *, tri_verts=None, ctrl=None, fiber_offsets=None, weights=None,
                 num_prims=None, stream=None) -> Level:
        """vx_voxelize: level 0 from triangles ([T,3,4] float32) or fibers (ctrl [P,4]
        float32, fiber_offsets [F+1] int64), all CUDA tensors on this context's device."""
        keep = []
        P = self._prims(tri_verts, ctrl, fiber_offsets, weights, num_prims, keep)
        G = _grid(grid)
        L = VxLevel()
        s = _stream(stream)
        st = self.lib.vx_voxelize(self.h, C.byref(P), C.byref(G), s, C.byref(L))
        if st != 0:
            raise self._err(st, "vx_voxelize")
        return self._wrap(L)

    def voxelize_sampled(self, grid, *, samples: int, tri_verts=None, ctrl=None, fiber_offsets=None, weights=None,
                         num_prims=None, stream=None) -> Level:
        """vx_voxelize_sampled: the sample-based level 0 of fibers (`samples` axis samples per
        segment) or triangles (up to `samples` per triangle, by area), for comparison with
        voxelize()."""
        keep = []
        P = self._prims(tri_verts, ctrl, fiber_offsets, weights, num_prims, keep)
        G = _grid(grid)
        L = VxLevel()
        st = self.lib.vx_voxelize_sampled(self.h, C.byref(P), C.byref(G), int(samples), _stream(stream), C.byref(L))
        if st != 0:
            raise self._err(st, "vx_voxelize_sampled")
        return self._wrap(L)

    def _prims(self, tri_verts, ctrl, fiber_offsets, weights, num_prims, keep):
        P = VxPrimitives()
        if tri_verts is not None:
            t = tri_verts.contiguous()
            _check(t, torch.float32, self.device, "tri_verts")
            keep.append(t)
            P.kind = VX_TRIANGLES
            P.num_prims = t.shape[0]
            P.tri_verts = t.data_ptr()
        else:
            c = ctrl.contiguous()
            o = fiber_offsets.contiguous()
            _check(c, torch.float32, self.device, "ctrl")
            _check(o, torch.int64, self.device, "fiber_offsets")
            keep += [c, o]
            P.kind = VX_FIBERS
            P.ctrl = c.data_ptr()
            P.num_ctrl = c.shape[0]
            P.fiber_offsets = o.data_ptr()
            P.num_fibers = o.shape[0] - 1
            if num_prims is None:
                oc = o.cpu()
                num_prims = int(torch.clamp(oc[1:] - oc[:-1] - 1, min=0).sum())
            P.num_prims = int(num_prims)
        if weights is not None:
            w = weights.contiguous()
            _check(w, torch.float32, self.device, "weights")
            keep.append(w)
            P.weights = w.data_ptr()
        return P

    def voxelize_lod_windowed(self, grid, *, window_log2: int, on_window, K: int = 1, dirs=None,
                              merge: str = "pooled", tri_verts=None, ctrl=None, fiber_offsets=None, weights=None,
                              num_prims=None, stream=None) -> list:
        """vx_voxelize_lod_windowed: the pyramid window by window.  on_window(window, levels)
        is called for every non-empty window of 2^window_log2 voxels per side (window: dict
        with lo, log2_size, index; levels: its levels 0 .. window_log2 - 1 as Level objects,
        which it may keep or drop).  Returns the levels window_log2 .. log2 R built from the
        windows' roots."""
        keep = []
        P = self._prims(tri_verts, ctrl, fiber_offsets, weights, num_prims, keep)
        G = _grid(grid)
        prm = VxLodParams()
        prm.num_levels = 0
        prm.K = int(K)
        prm.merge = _merge_mode(merge)
        if dirs is not None:
            d = dirs.contiguous()
            _check(d, torch.float32, self.device, "dirs")
            keep.append(d)
            prm.dirs = d.data_ptr()
            prm.n_samples = d.shape[0]
        failure = []

        def cb(user, win, levels, n, stream_):
            try:
                w = win.contents
                lv = [self._wrap(levels[i]) for i in range(n)]
                on_window({"lo": tuple(w.lo), "log2_size": int(w.log2_size), "index": int(w.index)}, lv)
                return 0
            except BaseException as e:       # stop the call; re-raised below
                failure.append(e)
                return 1
        fn = WINDOW_FN(cb)
        R = int(G.resolution)
        L = R.bit_length() - 1
        top = (VxLevel * (max(L - int(window_log2), 0) + 1))()
        ntop = C.c_int(0)
        st = self.lib.vx_voxelize_lod_windowed(self.h, C.byref(P), C.byref(G), C.byref(prm), int(window_log2), fn,
                                               None, _stream(stream), top, C.byref(ntop))
        if failure:
            raise failure[0]
        if st != 0:
            raise self._err(st, "vx_voxelize_lod_windowed")
        return [self._wrap(top[i]) for i in range(ntop.value)]

    def backward(self, grid, *, keys0, grad_mass, grad_moment, tri_verts=None, ctrl=None, fiber_offsets=None,
                 weights=None, num_prims=None, stream=None):
        """vx_backward: gradients of sum_l <grad_mass[l], m_l> + <grad_moment[l], M_l> w.r.t.
        the control points ([P,4]: xyz, radius) or the triangle vertices ([T,3,4]: xyz, 0),
        and the per-primitive weights."""
        keep = []
        P = self._prims(tri_verts, ctrl, fiber_offsets, weights, num_prims, keep)
        L = len(grad_mass) - 1
        gm = [g.contiguous() for g in grad_mass]
        gM = [g.contiguous() for g in grad_moment]
        for g in gm + gM:
            _check(g, torch.float32, self.device, "grad")
        k0 = keys0.contiguous()
        keep += gm + gM + [k0]
        pm = (C.c_void_p * (L + 1))(*[g.data_ptr() for g in gm])
        pM = (C.c_void_p * (L + 1))(*[g.data_ptr() for g in gM])
        shape = (P.num_prims, 3, 4) if tri_verts is not None else (P.num_ctrl, 4)
        g_ctrl = torch.empty(shape, dtype=torch.float32, device=self.device)
        g_w = torch.empty((P.num_prims,), dtype=torch.float32, device=self.device)
        G = _grid(grid)
        st = self.lib.vx_backward(self.h, C.byref(P), C.byref(G), k0.data_ptr(), k0.shape[0], L, pm, pM,
                                  _stream(stream), g_ctrl.data_ptr(), g_w.data_ptr())
        if st != 0:
            raise self._err(st, "vx_backward")
        return g_ctrl, g_w

    def batch(self, instances, *, K: int = 1, dirs=None, headroom: float = 0.125, merge: str = "pooled",
              stream=None) -> "Batch":
        """vx_batch_create_lod: instances = list of dicts with kind ("triangles" | "fibers"),
        grid, and tri_verts [T,3,4] or ctrl [P,4] + fiber_offsets [F+1] (+ optional weights),
        CUDA tensors; K lobes per voxel above level 0 (dirs [N,3] when K > 1).  Returns a
        Batch whose run() replays one captured graph."""
        return Batch(self, instances, headroom, stream, K=K, dirs=dirs, merge=merge)

    def _view_level(self, L: VxLevel, keep) -> Level:
        """Typed tensors over a level whose arrays live in blocks of this context's allocator."""
        n, K = int(L.num_voxels), int(L.K)

        def find(ptr, nbytes):
            for base, t in self.alloc.live.items():
                if base <= ptr and ptr + nbytes <= base + t.numel():
                    return t, base
            raise RuntimeError("level array outside the context's blocks")

        def v(ptr, nbytes, dtype, shape):
            if n == 0:
                return torch.empty(shape, dtype=dtype, device=self.device)
            t, base = find(ptr, nbytes)
            return t[ptr - base: ptr - base + nbytes].view(dtype).view(*shape)
        return Level(level=int(L.level), resolution=int(L.resolution), num_voxels=n, K=K,
                     keys=v(L.keys, n * 8, torch.int64, (n,)), mask=v(L.mask, n * 64, torch.int64, (n, 8)),
                     mass=v(L.mass, n * 4, torch.float32, (n,)), moment=v(L.moment, n * 24, torch.float32, (n, 6)),
                     occ=v(L.occ, n * 2, torch.int16, (n,)), occ_proj=v(L.occ_proj, n * 3, torch.uint8, (n, 3)),
                     lobe_count=v(L.lobe_count, n, torch.uint8, (n,)),
                     lobes=v(L.lobes, n * K * 28, torch.float32, (n, K, 7)),
                     compact=v(L.compact, n * K * 24, torch.float32, (n, K, 6)), block=None, _c=L)

    def tessellate_catmull_rom(self, nodes: torch.Tensor, offsets: torch.Tensor, subdiv: int, stream=None):
        """vx_tessellate_catmull_rom: spline nodes [P, 4] (xyz, radius) and offsets [F+1] ->
        fiber control points [(P - F) * subdiv + F, 4] and their offsets [F+1]."""
        nodes = nodes.contiguous()
        offsets = offsets.contiguous()
        _check(nodes, torch.float32, self.device, "nodes")
        _check(offsets, torch.int64, self.device, "offsets")
        F = offsets.shape[0] - 1
        P = nodes.shape[0]
        total = max((P - F) * int(subdiv) + F, 0)
        out = torch.empty((max(total, 1), 4), dtype=torch.float32, device=self.device)
        out_off = torch.empty((F + 1,), dtype=torch.int64, device=self.device)
        st = self.lib.vx_tessellate_catmull_rom(self.h, C.c_void_p(nodes.data_ptr() if P else 0),
                                                C.c_void_p(offsets.data_ptr()), F, P, int(subdiv),
                                                C.c_void_p(out.data_ptr()), C.c_void_p(out_off.data_ptr()),
                                                _stream(stream))
        if st != 0:
            raise self._err(st, "vx_tessellate_catmull_rom")
        return out[:total], out_off

    def export_leaves(self, level: Level, stream=None):
        """vx_export_leaves: the level's OpenVDB-style 8^3 leaf table: (leaf_keys int64 [L],
        value masks int64 [L, 8] (uint64 bit patterns, x-major bit order), first voxel of each
        leaf int32 [L + 1])."""
        n = max(level.num_voxels, 0)
        keys = torch.empty((max(n, 1),), dtype=torch.int64, device=self.device)
        masks = torch.empty((max(n, 1), 8), dtype=torch.int64, device=self.device)
        first = torch.empty((n + 1,), dtype=torch.int32, device=self.device)
        nl = C.c_int64(0)
        st = self.lib.vx_export_leaves(self.h, C.byref(level._c), C.c_void_p(keys.data_ptr()),
                                       C.c_void_p(masks.data_ptr()), C.c_void_p(first.data_ptr()), C.byref(nl),
                                       _stream(stream))
        if st != 0:
            raise self._err(st, "vx_export_leaves")
        L = int(nl.value)
        return keys[:L], masks[:L], first[: L + 1]

    def export_compact8(self, level: Level, stream=None) -> torch.Tensor:
        """vx_export_compact8: the level's lobes as 8-bit compact SGGX, uint8 [n, K, 6]."""
        out = torch.zeros((max(level.num_voxels, 0), level.K, 6), dtype=torch.uint8, device=self.device)
        st = self.lib.vx_export_compact8(C.byref(level._c), C.c_void_p(out.data_ptr() if out.numel() else 0),
                                         _stream(stream))
        if st != 0:
            raise self._err(st, "vx_export_compact8")
        return out

    def build_lod(self, level: Level, *, K: int = 1, dirs=None, num_levels: int = 0,
                  merge: str = "pooled", stream=None, events=None) -> list:
        """vx_build_lod: levels level+1 .. level+L (L = num_levels, 0 = down to 1^3).  merge:
        "pooled" (the two lobes' pooled samples) or "mass" (their moments weighted by mass).
        events: torch.cuda.Event objects; events[l] is recorded on the stream once level
        l of the result is complete (vx_build_lod_events)."""
        prm = VxLodParams()
        prm.num_levels = int(num_levels)
        prm.K = int(K)
        prm.merge = _merge_mode(merge)
        if dirs is not None:
            d = dirs.contiguous()
            _check(d, torch.float32, self.device, "dirs")
            prm.dirs = d.data_ptr()
            prm.n_samples = d.shape[0]
        R = level.resolution
        L = int(num_levels) if num_levels else int(R).bit_length() - 1
        outs = (VxLevel * max(L, 1))()
        if events is None:
            st = self.lib.vx_build_lod(self.h, C.byref(level._c), C.byref(prm), _stream(stream), outs)
        else:
            handles = []
            for ev in events:
                if ev.cuda_event == 0:   # a torch event is created by its first record
                    ev.record(torch.cuda.current_stream(self.device))
                handles.append(ev.cuda_event)
            arr = (C.c_void_p * max(len(handles), 1))(*handles)
            st = self.lib.vx_build_lod_events(self.h, C.byref(level._c), C.byref(prm), _stream(stream), outs,
                                              arr, len(handles))
        if st != 0:
            raise self._err(st, "vx_build_lod")
        return [self._wrap(outs[i]) for i in range(L)]


def _merge_mode(merge) -> int:
    modes = {"pooled": 0, "mass": 1}
    if merge not in modes:
        raise ValueError(f"merge: expected one of {sorted(modes)}, got {merge!r}")
    return modes[merge]


def _check(t, dtype, device, name):
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if t.device != device:
        raise ValueError(f"{name}: expected a tensor on {device}, got {t.device}")


def _grid(g) -> VxGrid:
    G = VxGrid()
    for i in range(3):
        G.origin[i] = float(g.origin[i])
    G.voxel_size = float(g.voxel_size)
    G.resolution = int(g.resolution)
    G.sub_res = int(getattr(g, "sub_res", 8))
    return G


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class VoxelizeLoD(torch.autograd.Function):
    """Differentiable voxelization + K = 1 pyramid.

    forward(geom, weights [N], fiber_offsets, grid, num_levels, context): geom is the
    control points ctrl [P,4] of fibers (fiber_offsets [F+1]) or, with fiber_offsets
    None, the triangle vertices [T,3,4].  Returns (mass_0, moment_0, ..., mass_L,
    moment_L).  backward runs vx_backward; it keeps only the level-0 keys (coarse levels
    are not stored, their parent structure is recomputed from the keys) and recomputes
    the candidate pairs.
    """

    @staticmethod
    def forward(fctx, geom, weights, fiber_offsets, grid, num_levels, context):
        if fiber_offsets is None:
            L0 = context.voxelize(grid, tri_verts=geom, weights=weights)
        else:
            L0 = context.voxelize(grid, ctrl=geom, fiber_offsets=fiber_offsets, weights=weights)
        pyr = context.build_lod(L0, K=1, num_levels=num_levels) if num_levels else []
        outs = []
        for lv in [L0] + pyr:
            outs += [lv.mass.clone(), lv.moment.clone()]
        fctx.save_for_backward(geom, weights, fiber_offsets, L0.keys.clone())
        fctx.grid = grid
        fctx.context = context
        fctx.num_levels = num_levels
        return tuple(outs)

    @staticmethod
    def backward(fctx, *grads):
        geom, weights, off, keys0 = fctx.saved_tensors
        gm = [torch.zeros_like(g) if g is None else g for g in grads[0::2]]
        gM = [torch.zeros_like(g) if g is None else g for g in grads[1::2]]
        kw = dict(tri_verts=geom) if off is None else dict(ctrl=geom, fiber_offsets=off)
        g_geom, g_w = fctx.context.backward(fctx.grid, keys0=keys0, grad_mass=[g.float() for g in gm],
                                            grad_moment=[g.float() for g in gM], weights=weights, **kw)
        return g_geom, g_w, None, None, None, None


NOALLOC_LIMITS = {"segments": 65536, "fibers": 8192, "voxels0": 262144, "pairs": 2097152}


def backward_noalloc(grid, *, ctrl, fiber_offsets, keys0, grad_mass, grad_moment, grad_ctrl, grad_weights=None,
                     weights=None, num_prims=None, stream=None):
    """vx_backward_noalloc: the gradients of Context.backward written into the caller's
    grad_ctrl [P,4] (and grad_weights [N]) with no device allocation (fixed library
    scratch; limits in NOALLOC_LIMITS).  Calls that overlap on the GPU race."""
    # the library writes num_ctrl * 16 bytes into grad_ctrl and num_prims * 4 into
    # grad_weights: their shapes, types, devices and layouts are checked before any call
    dev = ctrl.device
    _check(ctrl, torch.float32, dev, "ctrl")
    _check(fiber_offsets, torch.int64, dev, "fiber_offsets")
    if ctrl.dim() != 2 or ctrl.shape[1] != 4:
        raise ValueError(f"ctrl: expected shape (P, 4), got {tuple(ctrl.shape)}")
    if fiber_offsets.dim() != 1 or fiber_offsets.shape[0] < 2:
        raise ValueError("fiber_offsets: expected shape (F + 1,) with F >= 1")
    if not isinstance(grad_ctrl, torch.Tensor):
        raise TypeError("grad_ctrl: expected a tensor")
    _check(grad_ctrl, torch.float32, dev, "grad_ctrl")
    if tuple(grad_ctrl.shape) != (ctrl.shape[0], 4) or not grad_ctrl.is_contiguous():
        raise ValueError(f"grad_ctrl: expected a contiguous ({ctrl.shape[0]}, 4) tensor, got "
                         f"{tuple(grad_ctrl.shape)}{'' if grad_ctrl.is_contiguous() else ' (non-contiguous)'}")
    if len(grad_mass) != len(grad_moment) or len(grad_mass) < 1:
        raise ValueError("grad_mass / grad_moment: one tensor per level, the same number of each")
    for g in list(grad_mass) + list(grad_moment):
        _check(g, torch.float32, dev, "grad")
    _check(keys0, torch.int64, dev, "keys0")
    if num_prims is None:
        oc = fiber_offsets.cpu()
        num_prims = int(torch.clamp(oc[1:] - oc[:-1] - 1, min=0).sum())
    if grad_weights is not None:
        _check(grad_weights, torch.float32, dev, "grad_weights")
        if tuple(grad_weights.shape) != (int(num_prims),) or not grad_weights.is_contiguous():
            raise ValueError(f"grad_weights: expected a contiguous ({int(num_prims)},) tensor, got "
                             f"{tuple(grad_weights.shape)}")
    if weights is not None:
        _check(weights, torch.float32, dev, "weights")
        if tuple(weights.shape) != (int(num_prims),):
            raise ValueError(f"weights: expected shape ({int(num_prims)},), got {tuple(weights.shape)}")
    if dev.type != "cuda":
        raise ValueError(f"backward_noalloc: tensors must be on a CUDA device, got {dev}")
    lib = load()
    keep = []
    c = ctrl.contiguous()
    o = fiber_offsets.contiguous()
    P = VxPrimitives()
    P.kind = VX_FIBERS
    P.ctrl = c.data_ptr()
    P.num_ctrl = c.shape[0]
    P.fiber_offsets = o.data_ptr()
    P.num_fibers = o.shape[0] - 1
    P.num_prims = int(num_prims)
    if weights is not None:
        wt = weights.contiguous()
        keep.append(wt)
        P.weights = wt.data_ptr()
    L = len(grad_mass) - 1
    gm = [g.contiguous() for g in grad_mass]
    gM = [g.contiguous() for g in grad_moment]
    k0 = keys0.contiguous()
    keep += [c, o, k0] + gm + gM
    pm = (C.c_void_p * (L + 1))(*[g.data_ptr() for g in gm])
    pM = (C.c_void_p * (L + 1))(*[g.data_ptr() for g in gM])
    G = _grid(grid)
    st = lib.vx_backward_noalloc(C.byref(P), C.byref(G), k0.data_ptr(), k0.shape[0], L, pm, pM, _stream(stream),
                                 grad_ctrl.data_ptr(), None if grad_weights is None else grad_weights.data_ptr())
    if st != 0:
        detail = f"limits {NOALLOC_LIMITS}" if st == 3 else ""
        raise VxError(st, "vx_backward_noalloc", detail)


class Batch:
    """A planned batch (vx_batch_*): one captured CUDA graph runs every instance from its
    primitives to all of its pyramid levels (K lobes per voxel above level 0)."""

    def __init__(self, ctx: Context, instances, headroom=0.125, stream=None, K: int = 1, dirs=None,
                 merge: str = "pooled"):
        self.ctx = ctx
        lib = ctx.lib
        tris = [i for i in instances if i["kind"] == "triangles"]
        fibs = [i for i in instances if i["kind"] == "fibers"]
        self.keep = []
        tp = fp = None
        insts = (VxInstance * len(instances))()
        tb, fb, ffb, cb = 0, 0, 0, 0
        order = []
        # instances of a kind keep their relative order; the C side requires contiguous ranges
        for k, inst in enumerate(instances):
            I = insts[k]
            I.grid = _grid(inst["grid"])
            if inst["kind"] == "triangles":
                n = int(inst["tri_verts"].shape[0])
                I.kind, I.prim_begin, I.num_prims, I.fiber_begin, I.num_fibers = VX_TRIANGLES, tb, n, 0, 0
                tb += n
            else:
                o = inst["fiber_offsets"].cpu()
                n = int(torch.clamp(o[1:] - o[:-1] - 1, min=0).sum())
                F = int(o.shape[0] - 1)
                I.kind, I.prim_begin, I.num_prims, I.fiber_begin, I.num_fibers = VX_FIBERS, fb, n, ffb, F
                fb += n
                ffb += F
            order.append(k)
        if tris:
            tv = torch.cat([i["tri_verts"].reshape(-1, 3, 4) for i in tris]).contiguous()
            tw = None
            if any(i.get("weights") is not None for i in tris):
                tw = torch.cat([i["weights"] if i.get("weights") is not None else
                                torch.ones(i["tri_verts"].shape[0], device=ctx.device) for i in tris]).contiguous()
            self.keep += [tv, tw]
            tp = VxPrimitives()
            tp.kind, tp.num_prims, tp.tri_verts = VX_TRIANGLES, tv.shape[0], tv.data_ptr()
            tp.weights = None if tw is None else tw.data_ptr()
        if fibs:
            ctrls, offs, ws = [], [], []
            base = 0
            for i in fibs:
                o = i["fiber_offsets"].to(torch.int64)
                o0, o1 = int(o[0]), int(o[-1])
                c = i["ctrl"].reshape(-1, 4)[o0:o1]
                offs.append(o[:-1] - o0 + base)
                ctrls.append(c)
                base += c.shape[0]
            offs.append(torch.tensor([base], dtype=torch.int64, device=ctx.device))
            cc = torch.cat(ctrls).contiguous()
            oo = torch.cat(offs).contiguous()
            fw = None
            if any(i.get("weights") is not None for i in fibs):
                fw = torch.cat([i["weights"] if i.get("weights") is not None else
                                torch.ones(int(torch.clamp(i["fiber_offsets"][1:] - i["fiber_offsets"][:-1] - 1,
                                                           min=0).sum()), device=ctx.device)
                                for i in fibs]).contiguous()
            self.keep += [cc, oo, fw]
            fp = VxPrimitives()
            fp.kind, fp.num_prims = VX_FIBERS, fb
            fp.ctrl, fp.num_ctrl, fp.fiber_offsets, fp.num_fibers = cc.data_ptr(), cc.shape[0], oo.data_ptr(), oo.shape[0] - 1
            fp.weights = None if fw is None else fw.data_ptr()
        lod = VxLodParams()
        lod.num_levels, lod.K, lod.n_samples, lod.dirs = 0, int(K), 0, None
        lod.merge = _merge_mode(merge)
        if K > 1:
            if dirs is None:
                raise ValueError("K > 1 needs the direction set (dirs [N,3])")
            d = dirs.contiguous()
            _check(d, torch.float32, ctx.device, "dirs")
            self.keep.append(d)
            lod.n_samples, lod.dirs = int(d.shape[0]), d.data_ptr()
        h = C.c_void_p()
        st = lib.vx_batch_create_lod(ctx.h, None if tp is None else C.byref(tp), None if fp is None else C.byref(fp),
                                     insts, len(instances), C.byref(lod), float(headroom), _stream(stream),
                                     C.byref(h))
        if st != 0:
            raise ctx._err(st, "vx_batch_create_lod")
        self.h = h
        self.instances = instances

    def run(self, stream=None):
        st = self.ctx.lib.vx_batch_run(self.h, _stream(stream))
        if st != 0:
            raise self.ctx._err(st, "vx_batch_run")

    def level(self, instance: int, level: int, stream=None) -> Level:
        L = VxLevel()
        st = self.ctx.lib.vx_batch_level(self.h, int(instance), int(level), _stream(stream), C.byref(L))
        if st != 0:
            raise self.ctx._err(st, "vx_batch_level")
        return self.ctx._view_level(L, self.keep)

    def query(self) -> dict:
        """vx_batch_query: the plan's groups per kind and the launch shapes its autotuner
        picked (with the candidates' planning-run times)."""
        info = VxBatchInfo()
        st = self.ctx.lib.vx_batch_query(self.h, C.byref(info))
        if st != 0:
            raise self.ctx._err(st, "vx_batch_query")
        out = {}
        for k, name in enumerate(("triangles", "fibers")):
            out[name] = {
                "groups": int(info.num_groups[k]), "max_group_pairs": int(info.max_group_pairs[k]),
                "reduce_blocks_per_sm": int(info.reduce_blocks_per_sm[k]),
                "reduce_ms": {int(info.reduce_candidates[k][c]): float(info.reduce_ms[k][c]) for c in range(5)
                              if info.reduce_candidates[k][c]},
                "cluster_tier": {l: int(info.cluster_tier[k][l]) for l in range(12) if info.cluster_tier[k][l] >= 0},
                "cluster_ms": {l: [float(x) for x in info.cluster_ms[k][l]] for l in range(12)
                               if info.cluster_tier[k][l] >= 0}}
        return out

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.vx_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
