"""Writes tests/golden/large_oracle.npz: the CPU oracle's depth-buffer result on the whole
800x800x200 workload (0.05 m voxels, 2000-node RRT of depth <= 15, 320x240 rays, 8 m, 36 yaws).

Test infrastructure only. The stored values come from oracle.eval_tree alone (Sec. IV-A..C,
the depth-buffer method: per node and yaw the absolute and marginal counts, the selected yaw);
the inputs come from the seeded generator `synth.large()`. The file also records the SHA-256 of
the inputs and of the oracle's camera tables, so that a test on another machine can tell a
different input or a different host libm from a parity failure.

    python oracle/make_large_golden.py [--threads N]

About 35 minutes on 8 x86 cores.
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

OUT = os.path.join(_ROOT, "tests", "golden", "large_oracle.npz")


def camera_sha(sensor) -> str:
    t = oracle.camera_tables(sensor)
    return synth.sha256(t["body"], t["dzc"], t["ck"], t["sk"], t["M"])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0, help="oracle threads (0 = every core)")
    ap.add_argument("--out", default=OUT)
    a = ap.parse_args()
    t0 = time.time()
    p = synth.large()
    inputs_sha = synth.sha256(p.map.grid, p.tree.parent, p.tree.pos)
    print(f"inputs {inputs_sha[:16]} generated in {time.time() - t0:.1f} s", flush=True)
    t1 = time.time()
    r = oracle.eval_tree(p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor,
                         want_counts=True, n_threads=a.threads)
    secs = time.time() - t1
    print(f"oracle: {p.tree.n} nodes in {secs:.0f} s", flush=True)
    np.savez_compressed(a.out, abs=r["abs"], marg=r["marg"], yaw=r["yaw"], cnt_abs=r["cnt_abs"],
                        cnt_marg=r["cnt_marg"], inputs_sha256=np.array(inputs_sha),
                        camera_sha256=np.array(camera_sha(p.sensor)),
                        oracle_seconds=np.array(secs), oracle_threads=np.array(a.threads))
    print(f"wrote {a.out}", flush=True)


if __name__ == "__main__":
    main()
