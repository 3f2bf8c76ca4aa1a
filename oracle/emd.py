"""Exact-EMD option of SGGX-H (oracle only; test infrastructure like the rest of oracle/).

Sec. 4.4 merges, at each step, the two lobes whose direction histograms (5 bins per axis,
Eq. similarity) are closest in a Wasserstein distance.  The library and the C oracle use the
sliced reading: the Wasserstein-1 distance of the three axis marginals, summed.  This module
evaluates the unsliced reading on tiny cases, so that the merge orders of the two can be
compared:

  hist125(S, dirs)  the literal 5 x 5 x 5 histogram (counts) of a lobe: directions
                    omega_k = normalize(S'^(1/2) u_k) in FP64 (numpy eigh),
                    S' = S + 1e-6 tr(S) I, both omega_k and -omega_k counted (2N entries),
                    bin = min(4, floor((c + 1) * 2.5)) per axis.
  emd(Ha, Hb)       the exact Wasserstein-1 distance between two histograms
                    (normalised to 1) with the L1 ground distance between bin centres
                    (spacing 0.4).  With an L1 ground distance on a grid the cost of moving
                    mass between two bins is 0.4 x the length of a shortest grid path, so the
                    transport problem is the uncapacitated min-cost flow on the 5^3 grid
                    graph with unit arcs; it is solved as a linear program (scipy HiGHS).
  sggx_h_emd(...)   the agglomerative procedure of Sec. 4.4 with that distance: pairwise
                    distances, argmin (ties: smaller distance, then smaller i, then smaller
                    j over creation ids with i > j), merged lobe = the second moment of the
                    two lobes' pooled samples (M^_i + M^_j) / 2, its histogram re-sampled,
                    repeated until K lobes remain.  FP64 sampling; the distances are
                    compared as exact integers (emd_units, sliced_units: counts moved x
                    bins), so equal distances tie exactly.

Pinned by tests/test_oracle_emd.py: the flow program against the 125 x 125 coupling
program, closed forms for point masses, and the sliced distance as a lower bound.
"""
from __future__ import annotations

import numpy as np

_AB = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def lobe_directions(s6, dirs) -> np.ndarray:
    s6 = np.asarray(s6, np.float32)
    tr = np.float32(np.float32(s6[0] + s6[1]) + s6[2])
    eps = np.float32(1e-6) * tr
    S = np.array([[s6[0] + eps, s6[3], s6[4]], [s6[3], s6[1] + eps, s6[5]], [s6[4], s6[5], s6[2] + eps]],
                 np.float32).astype(np.float64)
    w, U = np.linalg.eigh(S)
    R = U @ np.diag(np.sqrt(np.maximum(w, 0.0))) @ U.T
    v = np.asarray(dirs, np.float64) @ R.T
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def hist125(s6, dirs):
    """(histogram counts [5,5,5] of the 2N entries, sample second moment M^ [6]) of a lobe.
    The normalised histogram is counts / 2N."""
    om = lobe_directions(s6, dirs)
    pts = np.concatenate([om, -om])
    b = np.minimum(4, np.floor((pts + 1.0) * 2.5).astype(np.int64))
    H = np.zeros((5, 5, 5), np.int64)
    np.add.at(H, (b[:, 0], b[:, 1], b[:, 2]), 1)
    M = np.array([np.mean(om[:, a] * om[:, c]) for a, c in _AB])
    return H, M


def _grid_arcs():
    idx = np.arange(125).reshape(5, 5, 5)
    arcs = []
    for ax in range(3):
        sl_a = [slice(None)] * 3
        sl_b = [slice(None)] * 3
        sl_a[ax] = slice(0, 4)
        sl_b[ax] = slice(1, 5)
        a = idx[tuple(sl_a)].ravel()
        b = idx[tuple(sl_b)].ravel()
        arcs += list(zip(a, b)) + list(zip(b, a))
    return np.asarray(arcs, np.int64)


_ARCS = _grid_arcs()


def emd_units(Ca, Cb) -> int:
    """Exact transport cost between two count histograms of equal total, in units of one
    count moved by one bin: the min-cost flow on the grid graph with unit arcs.  Supplies
    and costs are integers, so the optimum is an integer (the flow program is totally
    unimodular); the program's value is rounded to it."""
    return int(round(emd(np.asarray(Ca, np.float64), np.asarray(Cb, np.float64)) / 0.4))


def sliced_units(Ca, Cb) -> int:
    """Sliced transport cost of two count histograms in the same units, computed exactly in
    integers: sum over the axes of sum_k |CDF_a(k) - CDF_b(k)|."""
    d = 0
    for ax in range(3):
        other = tuple(i for i in range(3) if i != ax)
        ca = np.cumsum(np.asarray(Ca, np.int64).sum(axis=other))
        cb = np.cumsum(np.asarray(Cb, np.int64).sum(axis=other))
        d += int(np.abs(ca - cb)[:4].sum())
    return d


def emd(Ha, Hb) -> float:
    """Exact Wasserstein-1 (L1 ground distance, bin spacing 0.4) between two histograms of
    equal total mass, as a min-cost flow on the grid graph."""
    from scipy.optimize import linprog
    from scipy.sparse import coo_matrix
    supply = (np.asarray(Ha, np.float64) - np.asarray(Hb, np.float64)).ravel()
    if not np.any(supply):
        return 0.0
    m = _ARCS.shape[0]
    rows = np.concatenate([_ARCS[:, 0], _ARCS[:, 1]])
    cols = np.concatenate([np.arange(m), np.arange(m)])
    vals = np.concatenate([np.ones(m), -np.ones(m)])
    A = coo_matrix((vals, (rows, cols)), shape=(125, m)).tocsr()
    res = linprog(np.full(m, 0.4), A_eq=A, b_eq=supply, bounds=(0, None), method="highs")
    if res.status != 0:
        raise RuntimeError(f"min-cost flow failed: {res.message}")
    return float(res.fun)


def emd_coupling(Ha, Hb) -> float:
    """The same distance from the 125 x 125 coupling program (a second formulation, used to
    pin emd())."""
    from scipy.optimize import linprog
    from scipy.sparse import coo_matrix, vstack
    a = np.asarray(Ha, np.float64).ravel()
    b = np.asarray(Hb, np.float64).ravel()
    c = np.stack(np.unravel_index(np.arange(125), (5, 5, 5)), axis=1).astype(np.float64)
    cost = 0.4 * np.abs(c[:, None, :] - c[None, :, :]).sum(axis=2)
    i = np.repeat(np.arange(125), 125)
    j = np.tile(np.arange(125), 125)
    k = np.arange(125 * 125)
    Arow = coo_matrix((np.ones(k.size), (i, k)), shape=(125, k.size))
    Acol = coo_matrix((np.ones(k.size), (j, k)), shape=(125, k.size))
    res = linprog(cost.ravel(), A_eq=vstack([Arow, Acol]).tocsr(), b_eq=np.concatenate([a, b]), bounds=(0, None),
                  method="highs")
    if res.status != 0:
        raise RuntimeError(f"coupling program failed: {res.message}")
    return float(res.fun)


def sliced(Ha, Hb) -> float:
    """Sum over the axes of the Wasserstein-1 distance between the axis marginals."""
    d = 0.0
    for ax in range(3):
        other = tuple(i for i in range(3) if i != ax)
        ca = np.cumsum(np.asarray(Ha).sum(axis=other))
        cb = np.cumsum(np.asarray(Hb).sum(axis=other))
        d += 0.4 * float(np.abs(ca - cb)[:4].sum())
    return d


def sggx_h_emd(cand, K: int, dirs, distance: str = "emd"):
    """cand [n,7] (S6 + weight, candidate order) -> (lobes [m,7] sorted by weight, then
    creation id; merges [(i, j)] as creation ids).  distance: "emd" or "sliced" (the same
    loop with the sliced distance, for comparison within one formulation)."""
    dist = emd_units if distance == "emd" else sliced_units   # exact integers: ties are ties
    cand = np.asarray(cand, np.float64).reshape(-1, 7)
    S = [c[:6].copy() for c in cand]
    w = [float(c[6]) for c in cand]
    alive = list(range(len(S)))
    merges = []
    if len(S) > K:
        stats = [hist125(s, dirs) for s in S]
        D = {}
        for a in range(len(S)):
            for b in range(a):
                D[(a, b)] = dist(stats[a][0], stats[b][0])
        while len(alive) > K:
            best = None
            for a in alive:
                for b in alive:
                    if b < a:
                        key = (D[(a, b)], a, b)
                        if best is None or key < best:
                            best = key
            _, i, j = best
            Sn = 0.5 * (stats[i][1] + stats[j][1])
            n = len(S)
            S.append(Sn)
            w.append(w[i] + w[j])
            stats.append(hist125(Sn, dirs))
            alive = [x for x in alive if x not in (i, j)]
            for b in alive:
                D[(n, b)] = dist(stats[n][0], stats[b][0])
            alive.append(n)
            merges.append((i, j))
    order = sorted(alive, key=lambda x: (-w[x], x))
    out = np.array([list(S[x]) + [w[x]] for x in order]) if order else np.zeros((0, 7))
    return out, merges
