"""Seeded synthetic inputs shared by the tests, the bench and the oracle wrappers.

This module holds input generators only: primitive geometry with the shapes,
sizes and structure of the paper's workloads (fiber-level yarns and fabrics,
brushed-metal heightfields; paper Sec. 5.1 and Table "insertion times"), grid
placements, and the fixed set of unit directions that the SGGX-H histogram
step draws its N samples from (Sec. 4.4, "Implementation details").  None of
the method's arithmetic lives here: the voxelizer, the LoD build and the
clustering are implemented independently by `oracle/` and by the CUDA library.

Every generator is deterministic given its seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Grid", "Workload", "heightfield", "yarn", "woven_patch", "sample_directions",
    "random_segments", "random_triangles", "config1", "config2", "config3",
    "config4", "config5", "fiber_segment_count", "loss_weights",
]


@dataclass(frozen=True)
class Grid:
    """Cubic voxel grid: voxel (i,j,k) covers origin + h*[i,i+1]x[j,j+1]x[k,k+1]."""
    origin: tuple
    voxel_size: float
    resolution: int
    sub_res: int = 8


@dataclass
class Workload:
    name: str
    kind: str                      # "triangles" | "fibers"
    grid: Grid
    tri_verts: np.ndarray | None = None    # [T,3,4] float32 (xyz, w unused)
    ctrl: np.ndarray | None = None         # [P,4] float32 (xyz, radius)
    fiber_offsets: np.ndarray | None = None  # [F+1] int64 into ctrl
    weights: np.ndarray | None = None      # [num_prims] float32 or None (= 1)
    K: int = 1
    levels: int = 0                # 0 = down to 1^3
    extra: dict = field(default_factory=dict)

    @property
    def num_prims(self) -> int:
        if self.kind == "triangles":
            return int(self.tri_verts.shape[0])
        return fiber_segment_count(self.fiber_offsets)


def fiber_segment_count(offsets: np.ndarray) -> int:
    off = np.asarray(offsets, dtype=np.int64)
    return int(np.sum(np.maximum(off[1:] - off[:-1] - 1, 0)))


# ----------------------------------------------------------------------------
# Heightfield (brushed metal): 64x64 vertices on the unit square, heights
# sigma*N(0,1) box-filtered along x (anisotropic ridges), two triangles per cell
# with unshared vertices (triangles do not share vertex records, Sec. 3.2).
# ----------------------------------------------------------------------------
def heightfield(n: int = 64, seed: int = 1, sigma: float = 0.02, taps: int = 16,
                extent: float = 1.0, z0: float = 0.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    h = sigma * rng.standard_normal((n, n))          # [y, x]
    if taps > 1:
        acc = np.zeros_like(h)
        for k in range(-(taps // 2), taps - taps // 2):
            acc += np.roll(h, k, axis=1)
        h = acc / taps
    xs = np.linspace(0.0, extent, n)
    X, Y = np.meshgrid(xs, xs)                        # [y, x]
    P = np.stack([X, Y, h + z0], axis=-1)             # [n, n, 3]
    v00 = P[:-1, :-1].reshape(-1, 3)
    v10 = P[:-1, 1:].reshape(-1, 3)
    v11 = P[1:, 1:].reshape(-1, 3)
    v01 = P[1:, :-1].reshape(-1, 3)
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    tris = np.stack([t1, t2], axis=1).reshape(-1, 3, 3)
    out = np.zeros((tris.shape[0], 3, 4), dtype=np.float32)
    out[..., :3] = tris.astype(np.float32)
    return out


# ----------------------------------------------------------------------------
# Yarn: plies twisted around the yarn axis (x), fibers twisted around each ply
# centre, each fiber a polyline of `segments` segments with constant radius.
# ----------------------------------------------------------------------------
GOLDEN_ANGLE = math.pi * (3.0 - math.sqrt(5.0))


def yarn(plies: int = 3, fibers_per_ply: int = 64, segments: int = 4000,
         ply_radius: float = 0.15, fiber_radius: float = 0.004,
         twist: float = 2.0, jitter: float = 0.05, seed: int = 2,
         x0: float = 0.0, x1: float = 1.0, center=(0.5, 0.5),
         scale: float = 1.0, crimp=None):
    """Returns (ctrl [P,4] float32, fiber_offsets [F+1] int64).

    Ply p centre: angle 2*pi*p/plies + 2*pi*twist*x at distance ply_radius.
    Fiber f of a ply: local radius 0.1*sqrt((f+0.5)/n)*scale/1 + U(0, jitter),
    golden-angle phase, counter-twisted by -2*pi*twist*x.  `crimp(x)` optionally
    returns a (dy, dz) offset of the whole yarn axis (woven patches).
    """
    rng = np.random.default_rng(seed)
    F = plies * fibers_per_ply
    t = np.linspace(0.0, 1.0, segments + 1)
    x = x0 + (x1 - x0) * t
    xn = (x - x0) / max(x1 - x0, 1e-30)              # twist is per unit of yarn length
    pts = np.zeros((F, segments + 1, 4), dtype=np.float64)
    fi = 0
    for p in range(plies):
        th = 2.0 * math.pi * p / plies + 2.0 * math.pi * twist * xn
        cy = center[0] + scale * ply_radius * np.cos(th)
        cz = center[1] + scale * ply_radius * np.sin(th)
        for f in range(fibers_per_ply):
            rho = scale * (0.1 * math.sqrt((f + 0.5) / fibers_per_ply) + rng.uniform(0.0, jitter))
            ph = f * GOLDEN_ANGLE - 2.0 * math.pi * twist * xn
            y = cy + rho * np.cos(ph)
            z = cz + rho * np.sin(ph)
            if crimp is not None:
                dy, dz = crimp(x)
                y = y + dy
                z = z + dz
            pts[fi, :, 0] = x
            pts[fi, :, 1] = y
            pts[fi, :, 2] = z
            pts[fi, :, 3] = fiber_radius
            fi += 1
    ctrl = pts.reshape(-1, 4).astype(np.float32)
    offsets = np.arange(F + 1, dtype=np.int64) * (segments + 1)
    return ctrl, offsets


def woven_patch(n_warp: int = 16, n_weft: int = 16, plies: int = 3, fibers_per_ply: int = 80,
                segments_per_span: int = 2000, fiber_radius: float = 0.002, seed: int = 3):
    """Plain weave on the unit square: warp yarns along x, weft yarns along y.

    Each yarn is the twisted-ply yarn scaled by 0.1 (yarn radius about 0.03)
    with a sinusoidal over/under crimp of amplitude equal to the yarn radius.
    """
    pitch = 1.0 / n_warp
    yarn_r = 0.1 * 0.3
    ctrls, offs = [], [np.zeros(1, dtype=np.int64)]
    base = 0
    for w in range(n_warp):
        yc = (w + 0.5) * pitch
        ph = 0.0 if (w % 2 == 0) else math.pi

        def crimp(x, ph=ph):
            return 0.0 * x, yarn_r * np.sin(math.pi * n_weft * x + ph)
        c, o = yarn(plies, fibers_per_ply, segments_per_span, 0.15, fiber_radius, 2.0, 0.05,
                    seed * 1000 + w, 0.0, 1.0, (yc, 0.5), 0.1, crimp)
        ctrls.append(c)
        offs.append(o[1:] + base)
        base += c.shape[0]
    for w in range(n_weft):
        xc = (w + 0.5) * pitch
        ph = math.pi if (w % 2 == 0) else 0.0

        def crimp(x, ph=ph):
            return 0.0 * x, yarn_r * np.sin(math.pi * n_warp * x + ph)
        c, o = yarn(plies, fibers_per_ply, segments_per_span, 0.15, fiber_radius, 2.0, 0.05,
                    seed * 1000 + 500 + w, 0.0, 1.0, (xc, 0.5), 0.1, crimp)
        # swap x and y: weft runs along y
        c = c.copy()
        c[:, [0, 1]] = c[:, [1, 0]]
        ctrls.append(c)
        offs.append(o[1:] + base)
        base += c.shape[0]
    return np.concatenate(ctrls, axis=0), np.concatenate(offs).astype(np.int64)


# ----------------------------------------------------------------------------
# The fixed direction set of the SGGX-H histograms: a spherical Fibonacci set
# of n unit vectors (uniform on the whole sphere, deterministic).
# ----------------------------------------------------------------------------
def sample_directions(n: int = 5000) -> np.ndarray:
    k = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * k + 1.0) / n
    rxy = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    ph = k * GOLDEN_ANGLE
    d = np.stack([rxy * np.cos(ph), rxy * np.sin(ph), z], axis=1)
    return d.astype(np.float32)


# ----------------------------------------------------------------------------
# Small random cases for the tests.
# ----------------------------------------------------------------------------
def random_segments(n_fibers: int, pts_per_fiber: int, R: int, seed: int,
                    radius=(0.05, 0.6), step=(0.1, 1.5)):
    """Random-walk polylines in grid units of an R^3 grid with origin 0, h = 1/R.

    Returns (ctrl [P,4] float32 in world units, offsets [F+1] int64, grid).
    Radii and steps are in voxel units.
    """
    rng = np.random.default_rng(seed)
    h = 1.0 / R
    ctrl = []
    for _ in range(n_fibers):
        p = rng.uniform(0.2 * R, 0.8 * R, size=3)
        r = rng.uniform(*radius)
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        for _ in range(pts_per_fiber):
            ctrl.append([p[0] * h, p[1] * h, p[2] * h, r * h])
            d = d + 0.6 * rng.standard_normal(3)
            d /= np.linalg.norm(d)
            p = p + d * rng.uniform(*step)
            p = np.clip(p, -1.0, R + 1.0)
    ctrl = np.asarray(ctrl, dtype=np.float32)
    offsets = np.arange(n_fibers + 1, dtype=np.int64) * pts_per_fiber
    return ctrl, offsets, Grid((0.0, 0.0, 0.0), h, R)


def random_triangles(n: int, R: int, seed: int, size=(0.2, 3.0)):
    """Random triangles (grid units of an R^3 grid with origin 0, h = 1/R)."""
    rng = np.random.default_rng(seed)
    h = 1.0 / R
    c = rng.uniform(0.1 * R, 0.9 * R, size=(n, 1, 3))
    e = rng.standard_normal((n, 3, 3))
    s = rng.uniform(*size, size=(n, 1, 1))
    v = (c + e * s) * h
    out = np.zeros((n, 3, 4), dtype=np.float32)
    out[..., :3] = v.astype(np.float32)
    return out, Grid((0.0, 0.0, 0.0), h, R)


# ----------------------------------------------------------------------------
# Workload configurations (the shapes and sizes of the paper's regime).
# ----------------------------------------------------------------------------
def config1(seed: int = 1) -> Workload:
    """Brushed-metal heightfield, 64x64 vertices (7,938 triangles) at 128^3, K=1."""
    tris = heightfield(64, seed)
    return Workload("heightfield-7938tri-128^3-K1", "triangles",
                    Grid((0.0, 0.0, -0.5), 1.0 / 128.0, 128), tri_verts=tris, K=1)


def config2(seed: int = 2, plies: int = 3, fibers_per_ply: int = 64, segments: int = 4000,
            R: int = 512, K: int = 4) -> Workload:
    """Fiber yarn: 3 plies x 64 fibers x 4,000 segments (768k segments) at 512^3, K=4."""
    ctrl, off = yarn(plies, fibers_per_ply, segments, seed=seed)
    nseg = plies * fibers_per_ply * segments
    return Workload(f"yarn-{nseg}seg-{R}^3-K{K}", "fibers",
                    Grid((0.0, 0.0, 0.0), 1.0 / R, R), ctrl=ctrl, fiber_offsets=off, K=K)


def config3(seed: int = 3, n_yarns: int = 16, fibers_per_ply: int = 80,
            segments_per_span: int = 2000, R: int = 2048, K: int = 4) -> Workload:
    """Woven patch: 16 warp x 16 weft yarns, 3x80 fibers, 2,000 segments, 2048^3, K=4."""
    ctrl, off = woven_patch(n_yarns, n_yarns, 3, fibers_per_ply, segments_per_span, 0.002, seed)
    return Workload(f"woven-{n_yarns}x{n_yarns}-{R}^3-K{K}", "fibers",
                    Grid((0.0, 0.0, 0.0), 1.0 / R, R), ctrl=ctrl, fiber_offsets=off, K=K)


def config4(seed: int = 4, n_instances: int = 64, min_tris: int = 2000, max_tris: int = 2_000_000,
            min_segs: int = 10_000, max_segs: int = 4_000_000, fiber_radius_voxels: float = 1.5):
    """Instances of uneven size for the batched path: half heightfields (min_tris..max_tris
    triangles), half yarn patches (min_segs..max_segs segments), log-uniform sizes, grids
    64^3..1024^3 drawn independently of the size.  A patch's fibers are fiber_radius_voxels
    voxels thick at its own resolution (the resolution is chosen to resolve the fibers)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_instances):
        R = int(2 ** rng.integers(6, 11))
        if i % 2 == 0:
            nt = int(math.exp(rng.uniform(math.log(min_tris), math.log(max_tris))))
            n = max(2, int(round(math.sqrt(nt / 2.0))) + 1)
            tris = heightfield(n, seed * 1000 + i)
            out.append(Workload(f"inst{i}-hf{tris.shape[0]}", "triangles",
                                Grid((0.0, 0.0, -0.5), 1.0 / R, R), tri_verts=tris, K=1))
        else:
            ns = int(math.exp(rng.uniform(math.log(min_segs), math.log(max_segs))))
            fibers = max(3, min(192, ns // 200))
            fpp = max(1, fibers // 3)
            segs = max(4, ns // (3 * fpp))
            ctrl, off = yarn(3, fpp, segs, fiber_radius=fiber_radius_voxels / R, seed=seed * 1000 + i)
            out.append(Workload(f"inst{i}-yarn{3 * fpp * segs}", "fibers",
                                Grid((0.0, 0.0, 0.0), 1.0 / R, R), ctrl=ctrl,
                                fiber_offsets=off, K=1))
    return out


def config5(seed: int = 5, R: int = 256, levels: int = 4, n_params: int = 64,
            segments: int = 4000, fibers_per_ply: int = 64):
    """Differentiation workload: the yarn re-gridded to 256^3 with 4 LoD levels,
    FP32 loss weights U(-1,1) drawn per output, 64 random parameter indices."""
    w = config2(seed=2, fibers_per_ply=fibers_per_ply, segments=segments, R=R, K=1)
    w.levels = levels
    w.name = f"yarn-adjoint-{w.num_prims}seg-{R}^3-L{levels}"
    w.extra["seed"] = seed
    w.extra["n_params"] = n_params
    return w


# ----------------------------------------------------------------------------
# Loss weights of the differentiation workload: U(-1,1) per (level, key, component),
# from SplitMix64 (Steele, Lea, Flood 2014) of a counter built from the key, the level,
# the component and the seed, so that any set of voxels gets the same weights
# regardless of how it is ordered or who enumerated it.
# ----------------------------------------------------------------------------
def _splitmix64(x: np.ndarray) -> np.ndarray:
    x = (x + np.uint64(0x9E3779B97F4A7C15)) & np.uint64(0xFFFFFFFFFFFFFFFF)
    z = x
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def loss_weights(keys, level: int, seed: int = 5):
    """(alpha [n] float32, beta [n,6] float32) in U(-1,1) for the voxels `keys` of `level`."""
    k = np.asarray(keys, dtype=np.uint64)
    with np.errstate(over="ignore"):
        base = (k << np.uint64(8)) ^ (np.uint64(level) << np.uint64(4)) ^ (np.uint64(seed) << np.uint64(56))
        cols = []
        for c in range(7):
            h = _splitmix64(base + np.uint64(c))
            u = (h >> np.uint64(40)).astype(np.float64) / float(1 << 24)
            cols.append((2.0 * u - 1.0).astype(np.float32))
    return cols[0], np.stack(cols[1:], axis=1)
