"""CPU tests of the owned-voxel count's helpers (csrc/voxcount.cuh), compiled for the host: the
brick and super-brick cast against a plain DDA (Sec. IV-B), the visit test against the voxels a
plain DDA visits, the float sufficient visit test and the float pixel/depth decisions against the
exact integer tests they stand in for (Eq. 5). The GPU parity tests check the kernels built from
them against the oracle; these check each helper against its definition on many random cases."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    out = str(tmp_path_factory.mktemp("helpers") / "kernel_helpers_check")
    cmd = [nvcc, "-x", "cu", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2609_40297_gb300", "csrc"),
           "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "kernel_helpers_check.cu"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return out


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_helpers_agree_with_their_definitions(checker, seed):
    r = subprocess.run([checker, str(seed), "1"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:]
    c = {k: int(v) for k, v in re.findall(r"(\w+) (\d+)", r.stdout)}
    assert c["cast_rays"] > 50_000 and c["cast_bad"] == 0
    assert c["visit_checks"] > 1_000_000 and c["visit_bad"] == 0
    # the sufficient visit test decides a good share of the visits and never a non-visit
    assert c["surely_bad"] == 0 and c["surely_yes"] > 0.5 * c["surely_visits"]
    # the float pixel decisions: no disagreement, and almost every case decided
    assert c["pixel_bad"] == 0
    assert c["decided"] > 500_000 and c["undecided"] < 0.002 * c["pixel"]
