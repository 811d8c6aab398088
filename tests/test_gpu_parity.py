"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit for bit.

Gains, yaws, per-(node, yaw) counts and depth buffers are integers under the fixed-point
reading of Sec. IV, so the bar is exact equality everywhere.
"""
import numpy as np
import pytest

import oracle
import synth
from synth import Sensor

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2609_40297_gb300 as mig  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = mig.Context(0)
    yield c
    c.close()


def run_both(ctx, grid, voxel, origin, parent, pos, sensor, mode=0, depth=True, tiles=None):
    m = mig.Map(ctx, grid, voxel, origin)
    try:
        if tiles:
            ctx.set_tiles(*tiles)
        got = mig.tree_eval(m, parent, pos, sensor, mode=mode, want_counts=True, want_depth=depth)
    finally:
        m.close()
        if tiles:
            ctx.set_tiles(4, 16, 4)
    ref = oracle.eval_tree(grid, voxel, origin, parent, pos, sensor, mode=mode, want_counts=True, want_depth=depth)
    return got, ref


def assert_same(got, ref, keys=("abs", "marg", "yaw", "cnt_abs", "cnt_marg", "depth")):
    for k in keys:
        if k in ref:
            a, b = got[k], ref[k]
            if not np.array_equal(a, b):
                bad = np.argwhere(a != b)
                raise AssertionError(f"{k}: {len(bad)} mismatches, first at {bad[:5].tolist()}: "
                                     f"gpu {a[tuple(bad[0])]} oracle {b[tuple(bad[0])]}")


def test_tiny_config_bit_exact(ctx):
    p = synth.tiny()
    got, ref = run_both(ctx, p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor)
    assert_same(got, ref)
    assert got["abs"].sum() > 0 and np.any(got["marg"] < got["abs"])


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6])
def test_random_small_bit_exact(ctx, seed):
    p = synth.random_small(seed, n_nodes=24, max_depth=7)
    got, ref = run_both(ctx, p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor)
    assert_same(got, ref)


@pytest.mark.parametrize("mode", [mig.MODE_SINGLE_PARENT, mig.MODE_ABSOLUTE])
def test_modes_bit_exact(ctx, mode):
    p = synth.random_small(11, n_nodes=20, max_depth=6)
    got, ref = run_both(ctx, p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor,
                        mode=mode)
    assert_same(got, ref)


@pytest.mark.parametrize("sensor", [Sensor(87, 58, 48, 28, 2.0, 12, 10.0), Sensor(60, 45, 33, 17, 3.0, 5, -20.0),
                                    Sensor(120, 90, 7, 5, 2.5, 3, 0.0), Sensor(90, 60, 1, 1, 2.0, 1, 0.0)])
def test_sensors_bit_exact(ctx, sensor):
    p = synth.random_small(21, n_nodes=15, max_depth=5, sensor=sensor)
    got, ref = run_both(ctx, p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor)
    assert_same(got, ref)


@pytest.mark.parametrize("tiles", [(32, 8, 4), (8, 4, 8), (16, 2, 4), (32, 1, 8), (8, 8, 4), (16, 64, 4)])
def test_tile_shapes_bit_exact(ctx, tiles):
    p = synth.random_small(31, n_nodes=18, max_depth=6)
    got, ref = run_both(ctx, p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor,
                        tiles=tiles)
    assert_same(got, ref)


def test_edge_cases(ctx):
    v = 0.25
    rng = np.random.default_rng(9)
    grid = np.where(rng.random((10, 12, 14)) < 0.1, 2, 0).astype(np.uint8)
    s = Sensor(90, 60, 9, 7, 1.5, 4, 0.0)
    # a node inside an occupied voxel, one exactly on a voxel corner, one at the grid's far edge
    occ = np.argwhere(grid == 2)[0]
    pos = np.array([[7.3, 6.1, 5.2], [(occ[2] + 0.5), (occ[1] + 0.5), (occ[0] + 0.5)], [4.0, 4.0, 4.0],
                    [13.99, 11.99, 9.99], [0.0, 0.0, 0.0]], np.float32) * v
    grid[5, 6, 7] = 1
    parent = np.array([-1, 0, 1, 0, 3], np.int32)
    got, ref = run_both(ctx, grid, v, (0, 0, 0), parent, pos, s)
    assert_same(got, ref)
    assert got["abs"][1] == 0  # inside an occupied voxel: the ray stops at t = 0
    # single node; all-free and all-unknown maps
    for fill in (1, 0):
        g = np.full((8, 9, 10), fill, np.uint8)
        got, ref = run_both(ctx, g, v, (0.1, -0.2, 0.3), np.array([-1], np.int32),
                            np.array([[1.3, 1.0, 1.1]], np.float32), s)
        assert_same(got, ref)
        assert (got["abs"][0] == 0) == (fill == 1)


def test_deep_chain(ctx):
    # a 65-node chain: depth 64, the maximum; every node excluded against up to 64 ancestors
    n = mig_max_depth = 64
    v = 0.2
    grid = np.zeros((20, 20, 90), np.uint8)
    grid[:, :, 85:] = 2
    parent = np.arange(-1, n, dtype=np.int32)
    pos = np.stack([np.linspace(1.0, 16.0, n + 1), np.full(n + 1, 2.0), np.full(n + 1, 2.0)], 1).astype(np.float32)
    s = Sensor(90, 60, 12, 8, 1.5, 4, 0.0)
    got, ref = run_both(ctx, grid, v, (0, 0, 0), parent, pos, s, depth=False)
    assert_same(got, ref)
    assert mig_max_depth == 64


def test_empty_tree(ctx):
    p = synth.tiny()
    m = mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin)
    got = mig.tree_eval(m, np.zeros(0, np.int32), np.zeros((0, 3), np.float32), p.sensor)
    m.close()
    assert got["abs"].size == 0


def test_invalid_inputs_rejected(ctx):
    p = synth.tiny()
    m = mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin)
    try:
        bad = p.tree.parent.copy()
        bad[5] = 5
        with pytest.raises(mig.MigError) as e:
            mig.tree_eval(m, bad, p.tree.pos, p.sensor)
        assert e.value.status == mig.MIG_EINVAL
        pos = p.tree.pos.copy()
        pos[3] = [-5.0, 0, 0]
        with pytest.raises(mig.MigError):
            mig.tree_eval(m, p.tree.parent, pos, p.sensor)
        for s in (Sensor(0, 60, 8, 8, 4.0, 8, 0), Sensor(90, 60, 0, 8, 4.0, 8, 0), Sensor(90, 60, 8, 8, 400.0, 8, 0),
                  Sensor(90, 60, 8, 8, 4.0, 0, 0), Sensor(0.5, 60, 2048, 8, 4.0, 8, 0)):  # last: focal length too long
            with pytest.raises(mig.MigError):
                mig.tree_eval(m, p.tree.parent, p.tree.pos, s)
        # the context still works afterwards
        got = mig.tree_eval(m, p.tree.parent, p.tree.pos, p.sensor)
        assert got["abs"].sum() > 0
    finally:
        m.close()
    g = p.map.grid.copy()
    g[0, 0, 0] = 3
    with pytest.raises(mig.MigError):
        mig.Map(ctx, g, p.map.voxel_size)


def test_map_update_and_read(ctx):
    p = synth.tiny()
    m = mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin)
    try:
        assert np.array_equal(m.read(), p.map.grid)
        g2 = p.map.grid.copy()
        rng = np.random.default_rng(4)
        box = rng.integers(0, 3, size=(7, 11, 13)).astype(np.uint8)
        g2[3:10, 20:31, 9:22] = box
        m.update(9, 20, 3, box)
        assert np.array_equal(m.read(), g2)
        got = mig.tree_eval(m, p.tree.parent, p.tree.pos, p.sensor)
    finally:
        m.close()
    ref = oracle.eval_tree(g2, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor)
    assert_same(got, ref, ("abs", "marg", "yaw"))


def test_device_path_matches_host_path(ctx):
    p = synth.random_small(7, n_nodes=30, max_depth=6)
    m = mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin)
    try:
        host = mig.tree_eval(m, p.tree.parent, p.tree.pos, p.sensor)
        dev = torch.device("cuda:0")
        par = torch.from_numpy(p.tree.parent).to(dev)
        pos = torch.from_numpy(p.tree.pos).to(dev)
        outs = [torch.empty(p.tree.n, dtype=torch.int32, device=dev) for _ in range(3)]
        for md in (6, 9):  # exact depth bound and a looser one (empty trailing levels)
            mig.tree_eval_device(m, par, pos, p.sensor, md, *outs)
            ctx.sync()
            for k, o in zip(("abs", "marg", "yaw"), outs):
                assert np.array_equal(o.cpu().numpy(), host[k]), k
        # a too-small depth bound is flagged on the device and reported at sync
        mig.tree_eval_device(m, par, pos, p.sensor, 2, *outs)
        with pytest.raises(mig.MigError):
            ctx.sync()
        assert (outs[0].cpu().numpy() == -1).all()
        ctx.sync()  # the flag was cleared
    finally:
        m.close()


def test_paper_scale_full_tree_bit_exact(ctx):
    """The 500-node, 400x400x100 workload the benchmark times, every node and yaw, in the
    benchmark's launch configuration (default tiles)."""
    p = synth.paper_scale()
    got, ref = run_both(ctx, p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor,
                        depth=False)
    assert_same(got, ref, ("abs", "marg", "yaw", "cnt_abs", "cnt_marg"))


def test_large_sampled_paths_bit_exact(ctx):
    """The 2000-node, 800x800x200, 320x240-ray, K=36 workload: the whole tree on the device path
    (the benchmark's launch configuration), checked against the oracle on every node of three
    seeded root-to-leaf paths (an ancestor-closed subset the oracle evaluates exactly)."""
    p = synth.large()
    dev = torch.device("cuda:0")
    m = mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin)
    try:
        par = torch.from_numpy(p.tree.parent).to(dev)
        pos = torch.from_numpy(p.tree.pos).to(dev)
        outs = [torch.empty(p.tree.n, dtype=torch.int32, device=dev) for _ in range(3)]
        mig.tree_eval_device(m, par, pos, p.sensor, int(p.tree.depth().max()), *outs)
        ctx.sync()
        got = [o.cpu().numpy() for o in outs]
    finally:
        m.close()
    parent = p.tree.parent
    is_leaf = np.ones(p.tree.n, bool)
    is_leaf[parent[parent >= 0]] = False
    depth = p.tree.depth()
    rng = np.random.default_rng(3030)
    deep = np.nonzero(is_leaf & (depth >= depth.max() - 2))[0]
    mask = np.zeros(p.tree.n, np.uint8)
    for leaf in rng.choice(deep, size=3, replace=False):
        q = int(leaf)
        while q >= 0:
            mask[q] = 1
            q = int(parent[q])
    ref = oracle.eval_tree(p.map.grid, p.map.voxel_size, p.map.origin, parent, p.tree.pos, p.sensor, node_mask=mask)
    sel = mask.astype(bool)
    assert sel.sum() >= 16
    for k, g in zip(("abs", "marg", "yaw"), got):
        assert np.array_equal(g[sel], ref[k][sel]), k


def test_path_scoring_matches_oracle(ctx):
    """Eq. 3 / Eq. 4 on the device against the fp64 oracle (libm exp vs CUDA exp: relative 1e-12);
    the best node is an argmax of the oracle's objective up to that tolerance."""
    from oracle.score import score_tree
    for p in (synth.tiny(), synth.paper_scale()):
        m = mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin)
        try:
            g = mig.tree_eval(m, p.tree.parent, p.tree.pos, p.sensor)
        finally:
            m.close()
        cost, obj, best = mig.tree_score(ctx, p.tree.parent, p.tree.pos, g["marg"], p.map.voxel_size, 0.5)
        c_ref, o_ref, b_ref = score_tree(p.tree.parent, p.tree.pos.astype(np.float64), g["marg"], p.map.voxel_size, 0.5)
        assert np.allclose(cost, c_ref, rtol=1e-12, atol=1e-12)
        assert np.allclose(obj, o_ref, rtol=1e-12, atol=0)
        assert obj[best] >= o_ref.max() * (1 - 1e-12) and (best == b_ref or abs(o_ref[best] - o_ref[b_ref]) <= 1e-12 * o_ref.max())
