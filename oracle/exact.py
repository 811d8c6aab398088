"""Exact marginal gain, route 1 (test infrastructure only).

Eq. 2: E(n) = | I(n, psi_n) minus the union over ancestors a of I(a, psi_a) |, with the
yaws fixed to the depth-buffer method's choices (the paper validates with fixed yaws,
Sec. V-A). The paper's exact reference keeps each node's visible unknown voxels in a hash
map and merges the ancestors' maps per candidate (Sec. I, Sec. IV-E); exact_hash_merge does
exactly that with Python sets. exact_sorted_merge is the same set algebra on sorted numpy
arrays for large trees. Route 2 (depth-first reference counts) is oracle_exact_dfs in C.
"""
from __future__ import annotations

import numpy as np


def _ancestors(parent, n):
    out = []
    p = int(parent[n])
    while p >= 0:
        out.append(p)
        p = int(parent[p])
    return out


def exact_hash_merge(parent, offsets, ids, node_mask=None):
    parent = np.asarray(parent)
    n = parent.shape[0]
    sets = [set(ids[offsets[i]:offsets[i + 1]].tolist()) for i in range(n)]
    E = np.full(n, -1, np.int32)
    for i in range(n):
        if node_mask is not None and not node_mask[i]:
            continue
        merged = set()
        for a in _ancestors(parent, i):  # merge the ancestors' hash sets, rebuilt per candidate
            merged |= sets[a]
        E[i] = len(sets[i] - merged)
    return E


def exact_sorted_merge(parent, offsets, ids, node_mask=None):
    parent = np.asarray(parent)
    n = parent.shape[0]
    E = np.full(n, -1, np.int32)
    for i in range(n):
        if node_mask is not None and not node_mask[i]:
            continue
        anc = _ancestors(parent, i)
        mine = ids[offsets[i]:offsets[i + 1]]
        if not anc:
            E[i] = mine.size
            continue
        merged = np.unique(np.concatenate([ids[offsets[a]:offsets[a + 1]] for a in anc]))
        E[i] = int(np.count_nonzero(~np.isin(mine, merged, assume_unique=True)))
    return E


def gap_report(depth, marg_db, exact, abs_gain=None):
    """Relative gap of the depth-buffer marginal gain to the exact one (Fig. 4 style):
    overall sum ratio, per-depth mean ratio, least-squares slope through the origin and R^2."""
    depth = np.asarray(depth)
    db = np.asarray(marg_db, np.float64)
    ex = np.asarray(exact, np.float64)
    out = {"sum_db": float(db.sum()), "sum_exact": float(ex.sum())}
    out["sum_ratio"] = out["sum_db"] / out["sum_exact"] if out["sum_exact"] > 0 else float("nan")
    per = {}
    for d in np.unique(depth):
        m = (depth == d) & (ex > 0)
        if m.any():
            per[int(d)] = float(np.mean(db[m] / ex[m]))
    out["per_depth_mean_ratio"] = per
    if ex.size > 1 and np.var(ex) > 0:
        slope = float(np.dot(ex, db) / np.dot(ex, ex))
        A = np.vstack([ex, np.ones_like(ex)]).T
        coef, *_ = np.linalg.lstsq(A, db, rcond=None)
        pred = A @ coef
        ss_res = float(np.sum((db - pred) ** 2))
        ss_tot = float(np.sum((db - db.mean()) ** 2))
        out["slope_through_origin"] = slope
        out["slope"] = float(coef[0])
        out["r2"] = 1.0 - ss_res / ss_tot if ss_tot > 0 else float("nan")
    if abs_gain is not None:
        a = np.asarray(abs_gain, np.float64)
        out["abs_sum_ratio"] = float(a.sum() / ex.sum()) if ex.sum() > 0 else float("nan")
    return out
