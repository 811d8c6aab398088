"""GPU parity of the panoramic mode: the CUDA path through the C ABI against the oracle's
panoramic mode, bit for bit (gains, yaws, per-(node, yaw) window counts, depth buffers). Every
decision is integer: wedge cross products (Q30), strip projections (Q16), the DDA and the
ancestors' depth test."""
import numpy as np
import pytest

import synth
from synth import Sensor

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2609_40297_gb300 as mig  # noqa: E402
from test_gpu_parity import assert_same, run_both  # noqa: E402

MODE = mig.MODE_PANORAMIC


@pytest.fixture(scope="module")
def ctx():
    c = mig.Context(0)
    yield c
    c.close()


def test_pano_tiny_config_bit_exact(ctx):
    p = synth.tiny()
    got, ref = run_both(ctx, p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor,
                        mode=MODE)
    assert_same(got, ref)
    assert np.any(got["marg"] < got["abs"])


@pytest.mark.parametrize("seed,sensor", [(1, Sensor(90, 60, 16, 10, 2.0, 8, 0.0)),
                                         (2, Sensor(87, 58, 48, 28, 2.0, 12, 0.0)),
                                         (3, Sensor(60, 40, 20, 9, 3.0, 6, 0.0)),
                                         (4, Sensor(120, 90, 7, 5, 2.5, 3, 0.0))])
def test_pano_random_small_bit_exact(ctx, seed, sensor):
    p = synth.random_small(seed, n_nodes=20, max_depth=6, sensor=sensor)
    got, ref = run_both(ctx, p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor,
                        mode=MODE)
    assert_same(got, ref)


def test_pano_paper_scale_full_tree_bit_exact(ctx):
    """The 500-node paper-scale workload in the panoramic mode, every node and yaw window."""
    p = synth.paper_scale()
    got, ref = run_both(ctx, p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor,
                        mode=MODE, depth=False)
    assert_same(got, ref, ("abs", "marg", "yaw", "cnt_abs", "cnt_marg"))


def test_pano_mode_rejections(ctx):
    p = synth.tiny()
    m = mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin)
    try:
        pitched = Sensor(90, 60, 36, 24, 4.0, 8, 10.0)
        with pytest.raises(mig.MigError) as e:
            mig.tree_eval(m, p.tree.parent, p.tree.pos, pitched, mode=MODE)
        assert e.value.status == mig.MIG_EINVAL
        got = mig.tree_eval(m, p.tree.parent, p.tree.pos, p.sensor, mode=MODE)  # the context still works
        assert got["abs"].sum() > 0
    finally:
        m.close()
