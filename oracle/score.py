"""Path scoring of the planner (test infrastructure only), fp64, in depth order.

Eq. 3: c(n) = c(Pa(n)) + ||p_n - p_Pa(n)||, c(root) = 0 (travelled distance along the path).
Eq. 4: o(n) = o(Pa(n)) + g(n) exp(-lambda c(n)), o(root) = g(root) (c = 0), with the gain g(n) in
cubic metres: the voxel count times v_size^3 (Eq. 1 / Eq. 2). The best node is the one with the
largest objective (lowest index on ties); the planner executes the first segment towards it.
"""
from __future__ import annotations

import numpy as np


def score_tree(parent, pos, gain_counts, voxel_size, lam=0.5):
    parent = np.asarray(parent)
    pos = np.asarray(pos, np.float64).reshape(-1, 3)
    g = np.asarray(gain_counts, np.float64) * float(voxel_size) ** 3
    n = parent.shape[0]
    depth = np.zeros(n, np.int64)
    order = []
    for i in range(n):  # depth of each node by walking to the root
        d, q = 0, int(parent[i])
        while q >= 0:
            d += 1
            q = int(parent[q])
        depth[i] = d
    order = np.argsort(depth, kind="stable")
    cost = np.zeros(n)
    obj = np.zeros(n)
    for i in order:  # parents before children
        p = int(parent[i])
        if p < 0:
            cost[i] = 0.0
            obj[i] = g[i]
        else:
            cost[i] = cost[p] + float(np.sqrt(np.sum((pos[i] - pos[p]) ** 2)))
            obj[i] = obj[p] + g[i] * np.exp(-lam * cost[i])
    best = int(np.argmax(obj)) if n else -1
    return cost, obj, best
