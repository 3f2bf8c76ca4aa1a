"""CPU oracle for the voxelization / LoD / SGGX-H path (test infrastructure).

Only the tests, `__graft_entry__.smoke()` and the bench's `cpu_baseline` leg may
import this package.  It wraps `vxoracle.c`, a plain single-threaded C program
written from the paper's definitions (see the header of that file), compiled
with `-ffp-contract=off` so that FP32 decisions are taken in the same precision
and operation order as the kernels.  It shares no code with the CUDA library.

The exact-EMD option of SGGX-H (the unsliced reading of Eq. similarity) lives in
`oracle/emd.py`, in Python with scipy's LP solver, for tiny cross-checks only.

Parity unpinned: none.  Every function is pinned by tests/test_oracle_pins.py,
tests/test_oracle_adjoint_pins.py and tests/test_oracle_emd.py; the lobe sampling,
its six-count histogram encoding and the integer distance are pinned against a
literal 125-bin FP64 histogram and its sliced Wasserstein distance, and the whole
SGGX-H loop against an FP64 restatement (oracle/emd.py, distance "sliced").
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vxoracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libvxoracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-fvisibility=hidden", "-Wall", "-Wno-unused-function"]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/libvxoracle.so (gcc, a second or two)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("voxel_size", C.c_float), ("resolution", C.c_int32)]


class _Level(C.Structure):
    _fields_ = [("n", C.c_int64), ("K", C.c_int32),
                ("keys", C.POINTER(C.c_uint64)), ("mask", C.POINTER(C.c_uint64)),
                ("mass", C.POINTER(C.c_float)), ("moment", C.POINTER(C.c_float)),
                ("mass64", C.POINTER(C.c_double)), ("moment64", C.POINTER(C.c_double)),
                ("occ", C.POINTER(C.c_uint16)), ("proj", C.POINTER(C.c_uint8)),
                ("lobe_count", C.POINTER(C.c_uint8)), ("lobes", C.POINTER(C.c_float)),
                ("compact", C.POINTER(C.c_float))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            P = C.c_void_p
            lib.vxo_morton.restype = C.c_uint64
            lib.vxo_morton.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32]
            lib.vxo_capsule_box.restype = C.c_int
            lib.vxo_capsule_box.argtypes = [P, P, C.c_float, P, P]
            lib.vxo_capsule_mask.restype = C.c_int
            lib.vxo_capsule_mask.argtypes = [P, P, C.c_float, C.c_int, C.c_int, C.c_int, P]
            lib.vxo_capsule_measure.restype = C.c_float
            lib.vxo_capsule_measure.argtypes = [P, P, C.c_float, C.c_int, C.c_int, C.c_int]
            lib.vxo_tri_mask.restype = C.c_int
            lib.vxo_tri_mask.argtypes = [P, C.c_int, C.c_int, C.c_int, P]
            lib.vxo_tri_measure.restype = C.c_float
            lib.vxo_tri_measure.argtypes = [P, C.c_int, C.c_int, C.c_int]
            lib.vxo_tri_measure64.restype = C.c_double
            lib.vxo_tri_measure64.argtypes = [P, C.c_int, C.c_int, C.c_int]
            lib.vxo_compact.restype = None
            lib.vxo_compact.argtypes = [P, P]
            lib.vxo_compact8.restype = None
            lib.vxo_compact8.argtypes = [P, C.c_int64, P]
            lib.vxo_catmull_rom.restype = None
            lib.vxo_catmull_rom.argtypes = [P, P, C.c_int64, C.c_int, P, P]
            lib.vxo_sqrtm3.restype = None
            lib.vxo_sqrtm3.argtypes = [P, P]
            lib.vxo_sample_lobe.restype = None
            lib.vxo_sample_lobe.argtypes = [P, P, C.c_int, P, P]
            lib.vxo_hist_dist.restype = C.c_int64
            lib.vxo_hist_dist.argtypes = [P, P]
            lib.vxo_sggx_h.restype = C.c_int
            lib.vxo_sggx_h.argtypes = [P, C.c_int, C.c_int, P, C.c_int, P, P, C.c_int]
            lib.vxo_voxelize_tris_sampled.restype = C.c_int
            lib.vxo_voxelize_tris_sampled.argtypes = [P, C.c_int64, P, C.POINTER(_Grid), C.c_int, C.POINTER(_Level)]
            lib.vxo_voxelize_fibers_sampled.restype = C.c_int
            lib.vxo_voxelize_fibers_sampled.argtypes = [P, P, C.c_int64, P, C.POINTER(_Grid), C.c_int,
                                                        C.POINTER(_Level)]
            lib.vxo_voxelize_fibers.restype = C.c_int
            lib.vxo_voxelize_fibers.argtypes = [P, P, C.c_int64, P, C.POINTER(_Grid), C.c_int,
                                                C.POINTER(_Level)]
            lib.vxo_voxelize_tris.restype = C.c_int
            lib.vxo_voxelize_tris.argtypes = [P, C.c_int64, P, C.POINTER(_Grid), C.c_int,
                                              C.POINTER(_Level)]
            lib.vxo_lod_step.restype = C.c_int
            lib.vxo_lod_step.argtypes = [C.POINTER(_Level), C.c_int, P, C.c_int, C.POINTER(_Level), C.c_int]
            lib.vxo_level_free.restype = None
            lib.vxo_level_free.argtypes = [C.POINTER(_Level)]
            lib.vxo_fiber_voxels.restype = C.c_int
            lib.vxo_fiber_voxels.argtypes = [P, P, C.c_int64, P, C.POINTER(_Grid), P, C.c_int64,
                                             P, P, P, P, P]
            lib.vxo_level_from_voxels.restype = C.c_int
            lib.vxo_level_from_voxels.argtypes = [P, P, P, P, P, P, C.c_int64, C.POINTER(_Level)]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _grid(g) -> _Grid:
    G = _Grid()
    for i in range(3):
        G.origin[i] = float(g.origin[i])
    G.voxel_size = float(g.voxel_size)
    G.resolution = int(g.resolution)
    return G


_FIELDS = {"keys": (np.uint64, 1), "mask": (np.uint64, 8), "mass": (np.float32, 1),
           "moment": (np.float32, 6), "mass64": (np.float64, 1), "moment64": (np.float64, 6),
           "occ": (np.uint16, 1), "proj": (np.uint8, 3), "lobe_count": (np.uint8, 1)}


def _level_to_dict(L: _Level) -> dict:
    n, K = int(L.n), int(L.K)
    out = {"K": K}
    for name, (dt, w) in _FIELDS.items():
        ptr = getattr(L, name)
        arr = np.ctypeslib.as_array(ptr, shape=(max(n, 1) * w,)).copy()[: n * w]
        out[name] = arr.reshape(n, w) if w > 1 else arr
        out[name] = out[name].astype(dt, copy=False)
    out["lobes"] = np.ctypeslib.as_array(L.lobes, shape=(max(n, 1) * K * 7,)).copy()[: n * K * 7].reshape(n, K, 7)
    out["compact"] = np.ctypeslib.as_array(L.compact, shape=(max(n, 1) * K * 6,)).copy()[: n * K * 6].reshape(n, K, 6)
    return out


def _dict_to_level(d: dict, keep: list) -> _Level:
    L = _Level()
    n = int(d["keys"].shape[0])
    K = int(d["K"])
    L.n, L.K = n, K
    conv = {"keys": (np.uint64, C.c_uint64), "mask": (np.uint64, C.c_uint64),
            "mass": (np.float32, C.c_float), "moment": (np.float32, C.c_float),
            "mass64": (np.float64, C.c_double), "moment64": (np.float64, C.c_double),
            "occ": (np.uint16, C.c_uint16), "proj": (np.uint8, C.c_uint8),
            "lobe_count": (np.uint8, C.c_uint8), "lobes": (np.float32, C.c_float),
            "compact": (np.float32, C.c_float)}
    for name, (dt, ct) in conv.items():
        a = np.ascontiguousarray(d[name], dtype=dt)
        keep.append(a)
        setattr(L, name, a.ctypes.data_as(C.POINTER(ct)))
    return L


# ----------------------------------------------------------------------------
# public wrappers
# ----------------------------------------------------------------------------
def demorton(k: int):
    """(x, y, z) of a Morton key (x in bit 0 of every triple)."""
    x = y = z = 0
    for i in range(21):
        x |= ((k >> (3 * i)) & 1) << i
        y |= ((k >> (3 * i + 1)) & 1) << i
        z |= ((k >> (3 * i + 2)) & 1) << i
    return x, y, z


def morton(x: int, y: int, z: int) -> int:
    return int(_load().vxo_morton(x, y, z))


def capsule_box(a, b, rr, lo, hi) -> int:
    a, b, lo, hi = _f32(a), _f32(b), _f32(lo), _f32(hi)
    return int(_load().vxo_capsule_box(_ptr(a), _ptr(b), float(np.float32(rr)), _ptr(lo), _ptr(hi)))


def capsule_mask(A, B, rg, vijk) -> np.ndarray:
    A, B = _f32(A), _f32(B)
    m = np.zeros(8, dtype=np.uint64)
    _load().vxo_capsule_mask(_ptr(A), _ptr(B), float(np.float32(rg)), int(vijk[0]), int(vijk[1]),
                             int(vijk[2]), _ptr(m))
    return m


def capsule_measure(A, B, rg, vijk) -> float:
    A, B = _f32(A), _f32(B)
    return float(_load().vxo_capsule_measure(_ptr(A), _ptr(B), float(np.float32(rg)), *map(int, vijk)))


def tri_mask(U, vijk) -> np.ndarray:
    U = _f32(U).reshape(9)
    m = np.zeros(8, dtype=np.uint64)
    _load().vxo_tri_mask(_ptr(U), int(vijk[0]), int(vijk[1]), int(vijk[2]), _ptr(m))
    return m


def tri_measure(U, vijk) -> float:
    U = _f32(U).reshape(9)
    return float(_load().vxo_tri_measure(_ptr(U), *map(int, vijk)))


def tri_measure64(U, vijk) -> float:
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(9)
    return float(_load().vxo_tri_measure64(_ptr(U), *map(int, vijk)))


def compact(S) -> np.ndarray:
    S = _f32(S).reshape(6)
    o = np.zeros(6, dtype=np.float32)
    _load().vxo_compact(_ptr(S), _ptr(o))
    return o


def catmull_rom(nodes, offsets, subdiv: int):
    """Tessellated Catmull-Rom spline fibers (Sec. 3.2): (ctrl [P', 4] float32, offsets [F+1])
    with (n_f - 1) * subdiv + 1 points per spline of n_f >= 1 nodes."""
    nodes = _f32(nodes).reshape(-1, 4)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    F = off.shape[0] - 1
    assert F >= 0 and np.all(np.diff(off) >= 1) and int(subdiv) >= 1
    total = int((off[-1] - F) * subdiv + F)
    out = np.zeros((max(total, 1), 4), dtype=np.float32)
    out_off = np.zeros(F + 1, dtype=np.int64)
    _load().vxo_catmull_rom(_ptr(nodes), _ptr(off), F, int(subdiv), _ptr(out), _ptr(out_off))
    return out[:total], out_off


def vdb_leaves(keys):
    """OpenVDB-style 8^3 leaf table of a level's sorted Morton keys: (leaf keys = key >> 9,
    value masks [L, 8] uint64 with bit (x & 7) * 64 + (y & 7) * 8 + (z & 7) per voxel, first
    voxel index of each leaf [L + 1])."""
    keys = np.asarray(keys, dtype=np.uint64)
    leaf = keys >> np.uint64(9)
    if keys.size == 0:
        return np.zeros(0, np.uint64), np.zeros((0, 8), np.uint64), np.zeros(1, np.int64)
    head = np.concatenate([[True], leaf[1:] != leaf[:-1]])
    first = np.concatenate([np.nonzero(head)[0], [keys.size]]).astype(np.int64)
    masks = np.zeros((first.size - 1, 8), dtype=np.uint64)
    for l in range(first.size - 1):
        for i in range(first[l], first[l + 1]):
            x, y, z = demorton(int(keys[i]) & 511)
            bit = x * 64 + y * 8 + z
            masks[l, bit >> 6] |= np.uint64(1) << np.uint64(bit & 63)
    return leaf[head], masks, first


def compact8(c) -> np.ndarray:
    """8-bit compact SGGX of parameter sextuples c [..., 6] (Sec. 4.3): bytes [..., 6]."""
    c = _f32(c)
    shape = c.shape
    flat = np.ascontiguousarray(c.reshape(-1, 6))
    o = np.zeros(flat.shape, dtype=np.uint8)
    if flat.shape[0]:
        _load().vxo_compact8(_ptr(flat), flat.shape[0], _ptr(o))
    return o.reshape(shape)


def sqrtm3(S) -> np.ndarray:
    S = _f32(S).reshape(6)
    R = np.zeros(9, dtype=np.float32)
    _load().vxo_sqrtm3(_ptr(S), _ptr(R))
    return R.reshape(3, 3)


def sample_lobe(S, dirs):
    S = _f32(S).reshape(6)
    dirs = _f32(dirs).reshape(-1, 3)
    h = np.zeros(6, dtype=np.int32)
    M = np.zeros(6, dtype=np.float32)
    _load().vxo_sample_lobe(_ptr(S), _ptr(dirs), int(dirs.shape[0]), _ptr(h), _ptr(M))
    return h, M


def hist_dist(a, b) -> int:
    a = np.ascontiguousarray(a, dtype=np.int32)
    b = np.ascontiguousarray(b, dtype=np.int32)
    return int(_load().vxo_hist_dist(_ptr(a), _ptr(b)))


def sggx_h(cand, K, dirs, merge: int = 0):
    """cand [n,7] (S6 + weight) -> (lobes [m,7] sorted by weight desc, merges [(i,j)])."""
    cand = _f32(cand).reshape(-1, 7)
    n = int(cand.shape[0])
    dirs = _f32(dirs).reshape(-1, 3)
    out = np.zeros((max(n, 1), 7), dtype=np.float32)
    merges = np.zeros((max(n, 1), 2), dtype=np.int32)
    m = _load().vxo_sggx_h(_ptr(cand), n, int(K), _ptr(dirs), int(dirs.shape[0]), _ptr(out),
                           _ptr(merges), int(merge))
    return out[:m].copy(), [tuple(x) for x in merges[: max(0, n - m)]]


def voxelize_fibers(ctrl, offsets, grid, weights=None, K=1) -> dict:
    ctrl = _f32(ctrl).reshape(-1, 4)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    w = None if weights is None else _f32(weights)
    L = _Level()
    G = _grid(grid)
    _load().vxo_voxelize_fibers(_ptr(ctrl), _ptr(offsets), int(offsets.shape[0] - 1), _ptr(w),
                                C.byref(G), int(K), C.byref(L))
    d = _level_to_dict(L)
    _load().vxo_level_free(C.byref(L))
    return d


def voxelize_fibers_sampled(ctrl, offsets, grid, samples: int, weights=None) -> dict:
    """Sample-based level 0 of fiber segments: `samples` axis samples per segment, each
    marking one sub-cell and carrying 1/samples of the segment's measure (Sec. 3.2-3.3)."""
    ctrl = _f32(ctrl).reshape(-1, 4)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    w = None if weights is None else _f32(weights)
    L = _Level()
    G = _grid(grid)
    _load().vxo_voxelize_fibers_sampled(_ptr(ctrl), _ptr(offsets), int(offsets.shape[0] - 1), _ptr(w),
                                        C.byref(G), int(samples), C.byref(L))
    d = _level_to_dict(L)
    _load().vxo_level_free(C.byref(L))
    return d


def voxelize_tris_sampled(tris, grid, samples: int, weights=None) -> dict:
    """Sample-based level 0 of triangles: up to `samples` per triangle by area relative to the
    largest, placed by Heitz's square-to-triangle map (Sec. 3.2-3.3)."""
    tris = _f32(tris).reshape(-1, 3, 4)
    w = None if weights is None else _f32(weights)
    L = _Level()
    G = _grid(grid)
    _load().vxo_voxelize_tris_sampled(_ptr(tris), int(tris.shape[0]), _ptr(w), C.byref(G), int(samples), C.byref(L))
    d = _level_to_dict(L)
    _load().vxo_level_free(C.byref(L))
    return d


def voxelize_tris(tris, grid, weights=None, K=1) -> dict:
    tris = _f32(tris).reshape(-1, 3, 4)
    w = None if weights is None else _f32(weights)
    L = _Level()
    G = _grid(grid)
    _load().vxo_voxelize_tris(_ptr(tris), int(tris.shape[0]), _ptr(w), C.byref(G), int(K), C.byref(L))
    d = _level_to_dict(L)
    _load().vxo_level_free(C.byref(L))
    return d


def voxelize(workload, K=None) -> dict:
    K = workload.K if K is None else K
    if workload.kind == "triangles":
        return voxelize_tris(workload.tri_verts, workload.grid, workload.weights, K)
    return voxelize_fibers(workload.ctrl, workload.fiber_offsets, workload.grid, workload.weights, K)


def lod_step(level: dict, K: int, dirs, merge: int = 0) -> dict:
    """One LoD level (Sec. 4.2-4.4); merge 0 = pooled-sample merge, 1 = mass-weighted."""
    keep = []
    Lin = _dict_to_level(level, keep)
    dirs = _f32(dirs).reshape(-1, 3)
    Lout = _Level()
    _load().vxo_lod_step(C.byref(Lin), int(K), _ptr(dirs), int(dirs.shape[0]), C.byref(Lout), int(merge))
    d = _level_to_dict(Lout)
    _load().vxo_level_free(C.byref(Lout))
    return d


def build_pyramid(level0: dict, resolution: int, K: int, dirs, num_levels: int = 0, merge: int = 0) -> list:
    """Levels 1..L (L = log2(resolution) when num_levels == 0)."""
    L = int(round(np.log2(resolution))) if num_levels == 0 else num_levels
    out, cur = [], level0
    for _ in range(L):
        cur = lod_step(cur, K, dirs, merge)
        out.append(cur)
    return out


def fiber_voxels(ctrl, offsets, grid, keys, weights=None) -> dict:
    ctrl = _f32(ctrl).reshape(-1, 4)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    nk = int(keys.shape[0])
    w = None if weights is None else _f32(weights)
    mask = np.zeros((nk, 8), dtype=np.uint64)
    mass = np.zeros(nk, dtype=np.float32)
    mom = np.zeros((nk, 6), dtype=np.float32)
    mass64 = np.zeros(nk, dtype=np.float64)
    mom64 = np.zeros((nk, 6), dtype=np.float64)
    G = _grid(grid)
    _load().vxo_fiber_voxels(_ptr(ctrl), _ptr(offsets), int(offsets.shape[0] - 1), _ptr(w),
                             C.byref(G), _ptr(keys), nk, _ptr(mask), _ptr(mass), _ptr(mom),
                             _ptr(mass64), _ptr(mom64))
    return {"mask": mask, "mass": mass, "moment": mom, "mass64": mass64, "moment64": mom64}


def level_from_voxels(keys, vox: dict) -> dict:
    """Level-0 dict (oracle layout) from brute-force voxel attributes (fiber_voxels);
    keys must be sorted; voxels with an empty mask are dropped."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    order = np.argsort(keys, kind="stable")
    keys = keys[order]
    arrs = [np.ascontiguousarray(vox[k][order]) for k in ("mask", "mass", "moment", "mass64", "moment64")]
    L = _Level()
    _load().vxo_level_from_voxels(_ptr(keys), *[_ptr(a) for a in arrs], int(keys.shape[0]), C.byref(L))
    d = _level_to_dict(L)
    _load().vxo_level_free(C.byref(L))
    return d


def fiber_adjoint(ctrl, offsets, grid, keys0, gm0, gM0, weights=None, prims=None, with_abs=False):
    """FP64 loss sum gm*m + gM.M over level-0 voxels and its gradient w.r.t. ctrl
    ([P,4]: xyz and radius, world units) and the per-segment weights.  With with_abs,
    also the summed magnitudes of each control-point gradient's per-pair terms."""
    lib = _load()
    if not hasattr(lib, "_adj_ready"):
        lib.vxo_fiber_adjoint.restype = C.c_double
        lib.vxo_fiber_adjoint.argtypes = [C.c_void_p] * 4 + [C.c_void_p, C.c_double, C.c_int] + \
            [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
             C.c_void_p]
        lib.vxo_fiber_adjoint.argtypes[2] = C.c_int64
        lib._adj_ready = True
    ctrl = np.ascontiguousarray(ctrl, dtype=np.float64).reshape(-1, 4)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    keys0 = np.ascontiguousarray(keys0, dtype=np.uint64)
    gm0 = np.ascontiguousarray(gm0, dtype=np.float64)
    gM0 = np.ascontiguousarray(gM0, dtype=np.float64).reshape(-1, 6)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    pr = None if prims is None else np.ascontiguousarray(np.sort(prims), dtype=np.int64)
    origin = np.ascontiguousarray(grid.origin, dtype=np.float64)
    nseg = int(np.sum(np.maximum(offsets[1:] - offsets[:-1] - 1, 0)))
    d_ctrl = np.zeros_like(ctrl)
    d_w = np.zeros(nseg, dtype=np.float64)
    d_abs = np.zeros_like(ctrl) if with_abs else None
    loss = lib.vxo_fiber_adjoint(_ptr(ctrl), _ptr(offsets), int(offsets.shape[0] - 1), _ptr(w), _ptr(origin),
                                 float(grid.voxel_size), int(grid.resolution), _ptr(keys0), int(keys0.shape[0]),
                                 _ptr(gm0), _ptr(gM0), _ptr(pr), 0 if pr is None else int(pr.shape[0]),
                                 _ptr(d_ctrl), _ptr(d_w), _ptr(d_abs))
    if with_abs:
        return float(loss), d_ctrl, d_w, d_abs
    return float(loss), d_ctrl, d_w


def broadcast_adjoints(keys0, level_keys, alphas, betas):
    """FP64 level-0 adjoints g0 = sum_l alpha_l[parent_l], gM0 = sum_l beta_l[parent_l]
    (m and M of a parent are sums over its children, Sec. 4.3)."""
    keys0 = np.asarray(keys0, np.uint64)
    gm = np.zeros(keys0.shape[0], np.float64)
    gM = np.zeros((keys0.shape[0], 6), np.float64)
    for l, (k, a, b) in enumerate(zip(level_keys, alphas, betas)):
        idx = np.searchsorted(np.asarray(k, np.uint64), keys0 >> np.uint64(3 * l))
        assert np.array_equal(np.asarray(k, np.uint64)[idx], keys0 >> np.uint64(3 * l))
        gm += np.asarray(a, np.float64)[idx]
        gM += np.asarray(b, np.float64)[idx]
    return gm, gM


def clip_signature(ctrl, offsets, grid, prims) -> int:
    """Hash of the clipped-piece active sets of the listed segments (FP64)."""
    lib = _load()
    if not hasattr(lib, "_sig_ready"):
        lib.vxo_clip_signature.restype = C.c_uint64
        lib.vxo_clip_signature.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_double, C.c_int,
                                           C.c_void_p, C.c_int64]
        lib._sig_ready = True
    ctrl = np.ascontiguousarray(ctrl, dtype=np.float64).reshape(-1, 4)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    pr = np.ascontiguousarray(np.sort(prims), dtype=np.int64)
    origin = np.ascontiguousarray(grid.origin, dtype=np.float64)
    return int(lib.vxo_clip_signature(_ptr(ctrl), _ptr(offsets), int(offsets.shape[0] - 1), _ptr(origin),
                                      float(grid.voxel_size), int(grid.resolution), _ptr(pr), int(pr.shape[0])))


def tri_adjoint(tris, grid, keys0, gm0, gM0, weights=None, prims=None, with_abs=False):
    """FP64 loss sum gm*m + gM.M over level-0 voxels and its gradient w.r.t. the triangle
    vertices ([T,3,3] world units) and the per-triangle weights, by complex-step
    differentiation of the clipped area and the face normal.  With with_abs, also the
    summed magnitudes of each vertex coordinate's per-pair terms."""
    lib = _load()
    if not hasattr(lib, "_tadj_ready"):
        lib.vxo_tri_adjoint.restype = C.c_double
        lib.vxo_tri_adjoint.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                                        C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                        C.c_void_p, C.c_void_p, C.c_void_p]
        lib._tadj_ready = True
    t = np.asarray(tris, dtype=np.float64)
    T = t.shape[0]
    t4 = np.zeros((T, 3, 4), np.float64)
    t4[:, :, :3] = t.reshape(T, 3, -1)[:, :, :3]
    keys0 = np.ascontiguousarray(keys0, dtype=np.uint64)
    gm0 = np.ascontiguousarray(gm0, dtype=np.float64)
    gM0 = np.ascontiguousarray(gM0, dtype=np.float64).reshape(-1, 6)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    pr = None if prims is None else np.ascontiguousarray(np.sort(prims), dtype=np.int64)
    origin = np.ascontiguousarray(grid.origin, dtype=np.float64)
    d_t = np.zeros((T, 3, 3), np.float64)
    d_w = np.zeros(T, np.float64)
    d_abs = np.zeros((T, 3, 3), np.float64) if with_abs else None
    loss = lib.vxo_tri_adjoint(_ptr(t4), T, _ptr(w), _ptr(origin), float(grid.voxel_size), int(grid.resolution),
                               _ptr(keys0), int(keys0.shape[0]), _ptr(gm0), _ptr(gM0), _ptr(pr),
                               0 if pr is None else int(pr.shape[0]), _ptr(d_t), _ptr(d_w), _ptr(d_abs))
    if with_abs:
        return float(loss), d_t, d_w, d_abs
    return float(loss), d_t, d_w


def tri_clip_signature(tris, grid, prims) -> int:
    """Hash of the clip structure of the listed triangles' clipped polygons (FP64)."""
    lib = _load()
    if not hasattr(lib, "_tsig_ready"):
        lib.vxo_tri_clip_signature.restype = C.c_uint64
        lib.vxo_tri_clip_signature.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_double, C.c_int,
                                               C.c_void_p, C.c_int64]
        lib._tsig_ready = True
    t = np.asarray(tris, dtype=np.float64)
    T = t.shape[0]
    t4 = np.zeros((T, 3, 4), np.float64)
    t4[:, :, :3] = t.reshape(T, 3, -1)[:, :, :3]
    pr = np.ascontiguousarray(np.sort(prims), dtype=np.int64)
    origin = np.ascontiguousarray(grid.origin, dtype=np.float64)
    return int(lib.vxo_tri_clip_signature(_ptr(t4), T, _ptr(origin), float(grid.voxel_size),
                                          int(grid.resolution), _ptr(pr), int(pr.shape[0])))
