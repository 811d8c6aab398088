"""Pins of the oracle's exact-yaw variant (Eq. 2 with each node's yaw chosen by the exact marginal
gain itself): a Python hash-set walk over the tree, built on the visible sets of every (node, yaw)
(oracle.visible_sets, pinned separately by the voxel-centric brute force), must choose the same
yaws and gains; with one yaw it reduces to the exact gain of route 2; the root's choice is the
depth-buffer method's (its marginal gain is its absolute gain)."""
import numpy as np
import pytest

import synth
from synth import Sensor


def _children(parent):
    ch = {i: [] for i in range(len(parent))}
    for i, p in enumerate(parent):
        if p >= 0:
            ch[int(p)].append(i)
    return ch


@pytest.mark.parametrize("seed", [3, 7])
def test_exact_yaw_matches_hash_set_walk(oracle_lib, seed):
    s = Sensor(90, 60, 14, 9, 2.0, 6, 0.0)
    p = synth.random_small(seed, n_nodes=12, max_depth=4, sensor=s)
    args = (p.map.grid, p.map.voxel_size, p.map.origin)
    n, K = p.tree.n, s.yaw_bins
    sets = []
    for k in range(K):
        off, ids = oracle_lib.visible_sets(*args, p.tree.pos, np.full(n, k, np.int32), s)
        sets.append([set(ids[off[i]:off[i + 1]].tolist()) for i in range(n)])
    parent = p.tree.parent
    root = int(np.nonzero(parent < 0)[0][0])
    ch = _children(parent)
    yaw = np.full(n, -1)
    E = np.full(n, -1)

    def walk(nd, seen):
        gains = [len(sets[k][nd] - seen) for k in range(K)]
        kb = int(np.argmax(gains))  # lowest index on ties
        yaw[nd], E[nd] = kb, gains[kb]
        for c in ch[nd]:
            walk(c, seen | sets[kb][nd])

    walk(root, set())
    y2, E2 = oracle_lib.exact_yaw(*args, parent, p.tree.pos, s)
    assert np.array_equal(y2, yaw) and np.array_equal(E2, E)
    assert E.sum() > 0


def test_exact_yaw_special_cases(oracle_lib):
    # one yaw: the exact-yaw variant is the exact gain of route 2 at that yaw
    s1 = Sensor(90, 60, 14, 9, 2.0, 1, 0.0)
    p = synth.random_small(5, n_nodes=12, max_depth=4, sensor=s1)
    args = (p.map.grid, p.map.voxel_size, p.map.origin)
    y, E = oracle_lib.exact_yaw(*args, p.tree.parent, p.tree.pos, s1)
    off, ids = oracle_lib.visible_sets(*args, p.tree.pos, np.zeros(p.tree.n, np.int32), s1)
    assert np.array_equal(E, oracle_lib.exact_dfs(p.tree.parent, off, ids, p.map.grid.size)) and np.all(y == 0)
    # the root: both methods take the yaw with the largest visible set
    s = Sensor(90, 60, 14, 9, 2.0, 6, 0.0)
    p = synth.random_small(6, n_nodes=8, max_depth=3, sensor=s)
    args = (p.map.grid, p.map.voxel_size, p.map.origin)
    y, E = oracle_lib.exact_yaw(*args, p.tree.parent, p.tree.pos, s)
    db = oracle_lib.eval_tree(*args, p.tree.parent, p.tree.pos, s)
    root = int(np.nonzero(p.tree.parent < 0)[0][0])
    assert y[root] == db["yaw"][root] and E[root] == db["abs"][root]
