"""The bounds-checked build (MIG_DEBUG_BOUNDS=1): every voxel load and depth-buffer write checks its
index and a violation makes the call fail instead of touching memory outside the buffer. This stands
in for a memory sanitizer (not available here): the checked library, run in a child process on the
tiny, random and paper-scale workloads in every mode, reports no violation and returns the oracle's
results bit for bit."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, ROOT_DIR)
from paper_2609_40297_gb300 import _build
import paper_2609_40297_gb300 as mig
mig.LIB_PATH = _build.LIB_CHECKED
import oracle, synth
from synth import Sensor
assert mig.lib().mig_build_flags() == mig.BUILD_CHECKED
cases = [(synth.tiny(), (0, 1, 2, 3, 4))]
for seed in (1, 2):
    cases.append((synth.random_small(seed, n_nodes=20, max_depth=6, sensor=Sensor(90, 60, 16, 10, 2.0, 8, 0.0)),
                  (0, 3, 4)))
cases.append((synth.random_small(3, n_nodes=16, max_depth=5, sensor=Sensor(87, 58, 48, 28, 2.0, 12, 10.0)), (0, 3)))
cases.append((synth.paper_scale(), (0,)))
with mig.Context(0) as ctx:
    for p, modes in cases:
        m = mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin)
        try:
            for md in modes:
                got = mig.tree_eval(m, p.tree.parent, p.tree.pos, p.sensor, mode=md, want_counts=True)
                ref = oracle.eval_tree(p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos,
                                       p.sensor, mode=md, want_counts=True)
                for k in ("abs", "marg", "yaw", "cnt_abs", "cnt_marg"):
                    assert np.array_equal(got[k], ref[k]), (p.name, md, k)
        finally:
            m.close()
print("checked build ok")
"""


def test_checked_build_reports_no_violation_and_matches_oracle():
    from paper_2609_40297_gb300 import _build
    _build.build(checked=True)
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT_DIR", repr(ROOT))], capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked build ok" in r.stdout
