"""GPU parity at the API's maximum sizes: the widest and tallest images (2048 pixels), the most yaw
bins (1024), the longest grid axis (4096 voxels) with the longest range (1024 voxels), each as a
thin case the oracle finishes quickly, in every gain mode, bit for bit."""
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

MODES = (mig.MODE_MARGINAL, mig.MODE_SINGLE_PARENT, mig.MODE_ABSOLUTE, mig.MODE_INTERVAL, mig.MODE_PANORAMIC)


@pytest.fixture(scope="module")
def ctx():
    c = mig.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("sensor", [Sensor(90, 10, 2048, 2, 2.5, 3, 0.0), Sensor(40, 120, 1, 2048, 2.5, 2, 0.0),
                                    Sensor(90, 60, 2, 2, 2.5, 1024, 0.0)],
                         ids=["width_2048", "height_2048", "yaw_bins_1024"])
def test_maximum_image_and_yaw_bins(ctx, sensor):
    p = synth.random_small(91, n_nodes=6, max_depth=3, sensor=sensor)
    for mode in MODES:
        got, ref = run_both(ctx, p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor,
                            mode=mode, depth=(mode == mig.MODE_MARGINAL))
        assert_same(got, ref)
        assert got["abs"].sum() > 0, mode


def test_longest_axis_and_range(ctx):
    """A 4096 x 6 x 6 grid at 0.05 m and a 51.2 m range (1024 voxels, the limit): rays along the
    long axis cross up to the whole range; the nodes sit along it."""
    rng = np.random.default_rng(92)
    v = 0.05
    grid = np.where(rng.random((6, 6, 4096)) < 0.5, 0, 1).astype(np.uint8)
    grid[:, :, 4000:] = 2
    grid[:, :, 2500:2503] = 2
    xs = np.array([100.3, 600.7, 1500.1, 2100.9, 2495.2])
    pos = (np.stack([xs, np.full(5, 3.1), np.full(5, 2.9)], 1) * v).astype(np.float32)
    parent = np.array([-1, 0, 1, 2, 3], np.int32)
    s = Sensor(30, 30, 8, 8, 1024 * v, 2, 0.0)
    for mode in MODES:
        got, ref = run_both(ctx, grid, v, (0, 0, 0), parent, pos, s, mode=mode, depth=(mode == mig.MODE_MARGINAL))
        assert_same(got, ref)
    assert got["abs"].sum() > 0
