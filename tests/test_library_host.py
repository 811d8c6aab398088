"""CPU tests of the C-ABI library: it loads without a GPU, exports every symbol the public
header declares, and its host-only entry points (tree check, the Sec. IV-A resolution rule)
behave as specified. No compute call is made here."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mig():
    from paper_2609_40297_gb300 import _build
    _build.build()
    import paper_2609_40297_gb300 as m
    m.lib()
    return m


def header_functions():
    txt = open(os.path.join(ROOT, "include", "mig.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mig_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(mig):
    names = header_functions()
    assert len(names) >= 20
    L = mig.lib()
    missing = [n for n in names if getattr(L, n, None) is None]
    assert not missing, missing
    assert sorted(mig.EXPORTS) == names


def test_libraries_resolve_every_symbol_at_load(mig):
    """Both builds (the library and the bounds-checked one) load with immediate binding: no symbol
    of the library's own code is left undefined."""
    import ctypes
    from paper_2609_40297_gb300 import _build
    for path in (_build.build(), _build.build(checked=True)):
        ctypes.CDLL(path, mode=os.RTLD_NOW)


def test_resolution_rule_golden(mig):
    """Sec. IV-A: W_D = ceil(2 d_max tan(theta_h/2) / v), H_D likewise (tests/golden)."""
    rows = [ln.split() for ln in open(os.path.join(ROOT, "tests", "golden", "resolution_rule.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert rows
    for r in rows:
        rng, hf, vf, v, W, H = float(r[0]), float(r[1]), float(r[2]), float(r[3]), int(r[4]), int(r[5])
        s = mig.Sensor(hf, vf, 1, 1, rng, 1, 0.0)
        assert mig.default_resolution(s, v) == (W, H)


def test_tree_check(mig):
    depth, md = mig.tree_check(np.array([-1, 0, 0, 1, 3, 4], np.int32))
    assert depth.tolist() == [0, 1, 1, 2, 3, 4] and md == 4
    for bad in ([1, 0], [-1, -1], [-1, 5], [-1, 1], [-1, 2, 1], [0]):
        with pytest.raises(mig.MigError) as e:
            mig.tree_check(np.array(bad, np.int32))
        assert e.value.status == mig.MIG_EINVAL
    chain = np.arange(-1, 64, dtype=np.int32)       # depth 64: allowed
    assert mig.tree_check(chain)[1] == 64
    with pytest.raises(mig.MigError):               # depth 65: rejected
        mig.tree_check(np.arange(-1, 65, dtype=np.int32))
    depth, md = mig.tree_check(np.zeros(0, np.int32))
    assert depth.size == 0 and md == -1
