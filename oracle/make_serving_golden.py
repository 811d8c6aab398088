"""Writes tests/golden/serving_oracle.npz: the CPU oracle's depth-buffer result for the first
requests of the serving workload (16 robots on 4 seeded 400x400x100 rooms maps at 0.1 m, Poisson
arrivals at 20 Hz per robot, trees of U[100, 1500] nodes, 160x120 rays, 16 yaws, 6 m, and before
each request a map update re-labelling 10 % of its map's voxels).

Test infrastructure only: each stored result comes from oracle.eval_tree (Sec. IV-A..C) on the map
exactly as it stands when the request is submitted (every earlier update of that map applied, in
arrival order); the inputs come from the seeded generator `synth.serving_requests()`. Per request
the file records the SHA-256 of the map as evaluated and of the tree.

    python oracle/make_serving_golden.py [--threads N] [--requests 24]

About 20 minutes on 8 x86 cores.
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

OUT = os.path.join(_ROOT, "tests", "golden", "serving_oracle.npz")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0, help="oracle threads (0 = every core)")
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--out", default=OUT)
    a = ap.parse_args()
    maps, pools, events, sensor, updates = synth.serving_requests(n_first=a.requests)
    grids = [m.grid for m in maps]
    n = []
    absv, marg, yaw, shas = [], [], [], []
    secs = 0.0
    for i, (t, rid, mi, ti) in enumerate(events):
        grids[mi] = synth.apply_update(grids[mi], updates[i])
        tr = pools[rid][1][ti]
        t1 = time.time()
        r = oracle.eval_tree(grids[mi], maps[mi].voxel_size, maps[mi].origin, tr.parent, tr.pos, sensor,
                             n_threads=a.threads)
        secs += time.time() - t1
        n.append(tr.n)
        absv.append(r["abs"])
        marg.append(r["marg"])
        yaw.append(r["yaw"])
        shas.append(synth.sha256(grids[mi], tr.parent, tr.pos))
        print(f"request {i}: map {mi}, robot {rid}, {tr.n} nodes, {time.time() - t1:.0f} s", flush=True)
    off = np.concatenate([[0], np.cumsum(n)])
    np.savez_compressed(a.out, offsets=off, abs=np.concatenate(absv), marg=np.concatenate(marg),
                        yaw=np.concatenate(yaw), inputs_sha256=np.array(shas), oracle_seconds=np.array(secs),
                        oracle_threads=np.array(a.threads))
    print(f"wrote {a.out}", flush=True)


if __name__ == "__main__":
    main()
