"""GPU parity of the interval mode (Sec. IV-B, Eq. 5-7): the CUDA path through the C ABI against
the oracle's interval mode, bit for bit. Every decision of the mode is either integer or a fixed
sequence of correctly rounded single-precision operations, on both sides, so the bar is exact
equality of gains, yaws, per-(node, yaw) counts and depth buffers."""
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

MODE = mig.MODE_INTERVAL


@pytest.fixture(scope="module")
def ctx():
    c = mig.Context(0)
    yield c
    c.close()


def test_interval_tiny_config_bit_exact(ctx):
    p = synth.tiny()
    got, ref = run_both(ctx, p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor,
                        mode=MODE)
    assert_same(got, ref)
    assert np.any(got["marg"] < got["abs"])


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_interval_random_small_bit_exact(ctx, seed):
    p = synth.random_small(seed, n_nodes=24, max_depth=7)
    got, ref = run_both(ctx, p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor,
                        mode=MODE)
    assert_same(got, ref)


@pytest.mark.parametrize("sensor", [Sensor(87, 58, 48, 28, 2.0, 12, 10.0), Sensor(60, 45, 33, 17, 3.0, 5, -20.0),
                                    Sensor(120, 90, 7, 5, 2.5, 3, 0.0)])
def test_interval_sensors_bit_exact(ctx, sensor):
    p = synth.random_small(21, n_nodes=15, max_depth=5, sensor=sensor)
    got, ref = run_both(ctx, p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor,
                        mode=MODE)
    assert_same(got, ref)


def test_interval_deep_chain_and_unknown_map(ctx):
    # 65-node chain (64 ancestors for the last node), and an all-unknown map where long rays hold
    # more samples than one pending buffer
    v = 0.2
    grid = np.zeros((20, 20, 90), np.uint8)
    grid[:, :, 85:] = 2
    parent = np.arange(-1, 64, dtype=np.int32)
    pos = np.stack([np.linspace(1.0, 16.0, 65), np.full(65, 2.0), np.full(65, 2.0)], 1).astype(np.float32)
    s = Sensor(90, 60, 12, 8, 1.5, 4, 0.0)
    got, ref = run_both(ctx, grid, v, (0, 0, 0), parent, pos, s, mode=MODE, depth=False)
    assert_same(got, ref)
    g = np.zeros((24, 30, 32), np.uint8)
    parent = np.array([-1, 0, 1, 1, 0], np.int32)
    pos = (np.array([[16, 15, 12], [17.5, 15.2, 12.1], [19, 16, 11.5], [17, 13.5, 12.5], [14.2, 15.5, 12.3]]) * v
           ).astype(np.float32)
    s = Sensor(70, 50, 5, 4, 4.0, 6, 0.0)
    got, ref = run_both(ctx, g, v, (0, 0, 0), parent, pos, s, mode=MODE)
    assert_same(got, ref)


def test_interval_paper_scale_full_tree_bit_exact(ctx):
    """The 500-node paper-scale workload in the interval mode, every node and yaw, against the
    oracle's literal interval walk."""
    p = synth.paper_scale()
    got, ref = run_both(ctx, p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor,
                        mode=MODE, depth=False)
    assert_same(got, ref, ("abs", "marg", "yaw", "cnt_abs", "cnt_marg"))


def test_unknown_mode_rejected(ctx):
    p = synth.tiny()
    m = mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin)
    try:
        with pytest.raises(mig.MigError) as e:
            mig.tree_eval(m, p.tree.parent, p.tree.pos, p.sensor, mode=5)
        assert e.value.status == mig.MIG_EINVAL
        with pytest.raises(mig.MigError):
            mig.tree_eval_batch(ctx, [(p.tree.parent, p.tree.pos, p.sensor)], [m], mode=5)
    finally:
        m.close()
