"""Writes tests/golden/batched_oracle.npz: the CPU oracle's depth-buffer result on every tree of
the 64-tree batched workload (64 seeded 400x400x100 rooms maps at 0.1 m, trees of U[50, 2000]
nodes and depth limits U[3, 15], ray grids drawn from 64x48 ... 320x240, 16 yaws, 6 m).

Test infrastructure only: the stored gains and yaws come from oracle.eval_tree alone (Sec. IV-A..C);
the inputs from the seeded generator `synth.batched()`. Per tree the file also records the SHA-256 of
its inputs, so that a test can tell a different input from a parity failure.

    python oracle/make_batched_golden.py [--threads N] [--trees 64]

About 1.5 hours on 8 x86 cores.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, _ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(_ROOT, "tests", "golden", "batched_oracle.npz")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0, help="oracle threads (0 = every core)")
    ap.add_argument("--trees", type=int, default=64)
    ap.add_argument("--out", default=OUT)
    a = ap.parse_args()
    t0 = time.time()
    probs = synth.batched(seed_base=404, n_trees=a.trees)
    print(f"{len(probs)} problems generated in {time.time() - t0:.0f} s", flush=True)
    n = np.array([p.tree.n for p in probs], np.int64)
    off = np.concatenate([[0], np.cumsum(n)])
    absv, marg, yaw = (np.zeros(off[-1], np.int32) for _ in range(3))
    shas = []
    secs = 0.0
    for i, p in enumerate(probs):
        t1 = time.time()
        r = oracle.eval_tree(p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor,
                             n_threads=a.threads)
        dt = time.time() - t1
        secs += dt
        absv[off[i]:off[i + 1]], marg[off[i]:off[i + 1]], yaw[off[i]:off[i + 1]] = r["abs"], r["marg"], r["yaw"]
        shas.append(synth.sha256(p.map.grid, p.tree.parent, p.tree.pos))
        print(f"tree {i}: {p.tree.n} nodes, {p.sensor.width}x{p.sensor.height}, {dt:.0f} s", flush=True)
    np.savez_compressed(a.out, offsets=off, abs=absv, marg=marg, yaw=yaw, inputs_sha256=np.array(shas),
                        oracle_seconds=np.array(secs), oracle_threads=np.array(a.threads))
    print(f"wrote {a.out}", flush=True)


if __name__ == "__main__":
    main()
