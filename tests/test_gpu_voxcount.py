"""The owned-voxel count (each pixel ray cast once to its stopping point, then every unknown voxel of
the frustum tested against the ray of the pixel that owns it) against the CPU oracle, bit for bit:
gains, yaws, per-(node, yaw) counts and depth buffers, in the three sample modes, with the step-count
buffer split into many chunks, after map updates that add and remove occupied voxels (the brick
occupancy summary), and against the ray-by-ray count kernel on the same inputs."""
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

KEYS = ("abs", "marg", "yaw", "cnt_abs", "cnt_marg", "depth")


@pytest.fixture(scope="module")
def ctx():
    c = mig.Context(0)
    yield c
    c.set_count_kernel(mig.COUNT_AUTO, 0)
    c.close()


def _same(got, ref, keys=KEYS, what=""):
    for k in keys:
        if k in ref:
            a, b = got[k], ref[k]
            if not np.array_equal(a, b):
                bad = np.argwhere(a != b)
                raise AssertionError(f"{what} {k}: {len(bad)} mismatches, first at {bad[:5].tolist()}: "
                                     f"gpu {a[tuple(bad[0])]} oracle {b[tuple(bad[0])]}")


def _eval(ctx, p, grid=None, mode=0, depth=True):
    g = p.map.grid if grid is None else grid
    m = mig.Map(ctx, g, p.map.voxel_size, p.map.origin)
    try:
        return mig.tree_eval(m, p.tree.parent, p.tree.pos, p.sensor, mode=mode, want_counts=True, want_depth=depth)
    finally:
        m.close()


def _oracle(p, grid=None, mode=0, depth=True):
    g = p.map.grid if grid is None else grid
    return oracle.eval_tree(g, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor, mode=mode,
                            want_counts=True, want_depth=depth)


# includes frusta that hold the vertical (looking steeply down, and nearly straight up: every yaw
# may hold a voxel), steep pitch, a 1x1 image, a wide and flat image, and more yaws than the
# per-node pass caches in shared memory (130)
SENSORS = [None, Sensor(87, 58, 48, 28, 2.0, 12, 10.0), Sensor(60, 45, 33, 17, 3.0, 5, -20.0),
           Sensor(120, 90, 7, 5, 2.5, 3, 0.0), Sensor(90, 60, 1, 1, 2.0, 4, 0.0), Sensor(170, 20, 61, 9, 2.2, 7, 35.0),
           Sensor(100, 150, 21, 17, 2.5, 9, 50.0), Sensor(60, 40, 15, 11, 2.0, 24, -80.0),
           Sensor(30, 20, 16, 12, 3.0, 130, 0.0)]


@pytest.mark.parametrize("voxel_pass", [mig.COUNT_PAIRS, mig.COUNT_NODES])
@pytest.mark.parametrize("si", range(len(SENSORS)))
@pytest.mark.parametrize("mode", [mig.MODE_MARGINAL, mig.MODE_SINGLE_PARENT, mig.MODE_ABSOLUTE])
def test_owned_voxel_count_bit_exact(ctx, si, mode, voxel_pass):
    """Both owned-voxel passes (per (node, yaw) frustum and per node over all yaws; the per-node
    pass takes at most 64 yaws and falls back to the per-pair one above that)."""
    ctx.set_count_kernel(voxel_pass, 0)
    try:
        p = synth.random_small(300 + si, n_nodes=14, max_depth=5, sensor=SENSORS[si])
        _same(_eval(ctx, p, mode=mode), _oracle(p, mode=mode), what=f"sensor {si} mode {mode} pass {voxel_pass}")
    finally:
        ctx.set_count_kernel(mig.COUNT_AUTO, 0)


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_many_chunks_per_level(ctx, seed):
    """A step-count buffer of 3 (node, yaw) pairs: every level is counted in many chunks, the last
    one partial."""
    p = synth.random_small(seed, n_nodes=24, max_depth=4)
    s = p.sensor
    try:
        ctx.set_count_kernel(mig.COUNT_PAIRS, 3 * s.width * s.height * 2)
        got = _eval(ctx, p)
    finally:
        ctx.set_count_kernel(mig.COUNT_AUTO, 0)
    _same(got, _oracle(p), what="3-pair chunks")


@pytest.mark.parametrize("seed", [14, 15])
def test_node_chunks(ctx, seed):
    """A step-count buffer of two nodes' pairs (all their yaws): the per-node voxel pass runs over
    many chunks of whole nodes per level."""
    p = synth.random_small(seed, n_nodes=24, max_depth=4)
    s = p.sensor
    try:
        ctx.set_count_kernel(mig.COUNT_NODES, 2 * s.yaw_bins * s.width * s.height * 2)
        got = _eval(ctx, p)
    finally:
        ctx.set_count_kernel(mig.COUNT_AUTO, 0)
    _same(got, _oracle(p), what="two-node chunks")


def test_tiny_and_sampled_paper_scale_against_ray_by_ray(ctx):
    """The two owned-voxel passes and the ray-by-ray count kernel agree on the tiny workload and on the
    nodes of depth <= 3 of the paper-scale tree (host-array path), and the tiny workload equals the
    oracle."""
    for p in (synth.tiny(), synth.paper_scale()):
        d = p.tree.depth()
        keep = np.nonzero(d <= (10 if p.name == "tiny" else 3))[0]
        remap = -np.ones(p.tree.n, np.int64)
        remap[keep] = np.arange(keep.size)
        par = np.where(p.tree.parent[keep] >= 0, remap[p.tree.parent[keep]], -1).astype(np.int32)
        sub = synth.Problem(p.name, p.map, synth.Tree(par, p.tree.pos[keep]), p.sensor)
        outs = []
        for kern in (mig.COUNT_PAIRS, mig.COUNT_NODES, mig.COUNT_RAYS):
            ctx.set_count_kernel(kern, 0)
            outs.append(_eval(ctx, sub, depth=False))
        ctx.set_count_kernel(mig.COUNT_AUTO, 0)
        a = outs[0]
        for b in outs[1:]:
            _same(a, b, keys=("abs", "marg", "yaw", "cnt_abs", "cnt_marg"), what=p.name)
        if p.name == "tiny":
            _same(a, _oracle(sub, depth=False), keys=("abs", "marg", "yaw", "cnt_abs", "cnt_marg"), what="tiny")


def test_map_updates_refresh_brick_occupancy(ctx):
    """Updates that fill a free region with occupied voxels and clear occupied ones: the brick summary
    follows, so results equal the oracle on the updated grid after every update."""
    ctx.set_count_kernel(mig.COUNT_AUTO, 0)
    rng = np.random.default_rng(5)
    p = synth.random_small(21, nx=40, ny=36, nz=20, n_nodes=16, max_depth=4, sensor=Sensor(90, 60, 24, 16, 3.0, 6, 0.0))
    g = p.map.grid.copy()
    m = mig.Map(ctx, g, p.map.voxel_size, p.map.origin)
    try:
        for it in range(4):
            nz, ny, nx = g.shape
            dz, dy, dx = int(rng.integers(2, nz)), int(rng.integers(3, ny)), int(rng.integers(3, nx))
            z0, y0, x0 = (int(rng.integers(0, s - w + 1)) for s, w in ((nz, dz), (ny, dy), (nx, dx)))
            box = rng.choice(np.array([0, 1, 2], np.uint8), size=(dz, dy, dx), p=[0.3, 0.5 if it % 2 else 0.7, 0.2 if it % 2 else 0.0])
            m.update(x0, y0, z0, box)
            g[z0:z0 + dz, y0:y0 + dy, x0:x0 + dx] = box
            got = mig.tree_eval(m, p.tree.parent, p.tree.pos, p.sensor, want_counts=True, want_depth=True)
            _same(got, _oracle(p, grid=g), what=f"update {it}")
    finally:
        m.close()


def test_super_brick_walk_and_updates(ctx):
    """A sparse map spanning several 32-voxel super-bricks (long rays cross free super-bricks in one
    step each): single occupied voxels written into free super-bricks and cleared again by updates
    change the results exactly as the oracle says."""
    ctx.set_count_kernel(mig.COUNT_AUTO, 0)
    rng = np.random.default_rng(17)
    p = synth.random_small(23, nx=136, ny=100, nz=70, v=0.1, p_occ=0.00002, p_free=0.5, n_nodes=14, max_depth=4,
                           sensor=Sensor(100, 70, 26, 18, 5.5, 6, 5.0))
    g = p.map.grid.copy()
    m = mig.Map(ctx, g, p.map.voxel_size, p.map.origin)
    try:
        _same(mig.tree_eval(m, p.tree.parent, p.tree.pos, p.sensor, want_counts=True, want_depth=True), _oracle(p, grid=g),
              what="initial")
        c = (np.asarray(p.tree.pos[0]) / p.map.voxel_size).astype(int)
        spots = []
        for it in range(4):
            # an occupied voxel 20-50 voxels from the root, where the rays are sparse
            off = rng.integers(20, 50, 3) * rng.choice([-1, 1], 3)
            x, y, z = (int(np.clip(c[a] + off[a], 0, g.shape[2 - a] - 1)) for a in range(3))
            box = np.full((1, 1, 1), 2, np.uint8)
            if it == 3:  # clear the first one again
                (x, y, z), box = spots[0], np.full((1, 1, 1), 1, np.uint8)
            spots.append((x, y, z))
            m.update(x, y, z, box)
            g[z, y, x] = box[0, 0, 0]
            got = mig.tree_eval(m, p.tree.parent, p.tree.pos, p.sensor, want_counts=True, want_depth=True)
            _same(got, _oracle(p, grid=g), what=f"update {it} at {(x, y, z)}")
    finally:
        m.close()


def test_stats_agree_between_kernels(ctx):
    """The instrumented pass re-runs the ray-by-ray kernel beside the owned-voxel one: both count the
    same samples, and the cast covers every ray."""
    ctx.set_count_kernel(mig.COUNT_AUTO, 0)
    p = synth.tiny()
    m = mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin)
    try:
        out, st = mig.tree_eval_stats(m, p.tree.parent, p.tree.pos, p.sensor)
    finally:
        m.close()
    s = p.sensor
    assert st["rays"] == st["cast_rays"] == p.tree.n * s.yaw_bins * s.width * s.height
    assert st["owned_samples"] == st["samples"] > 0
    assert st["voxel_candidates"] >= st["voxel_unknown"] >= st["visit_tests"] >= st["owned_samples"]
    assert st["cast_steps"] + st["cast_jumps"] <= st["dda_steps"]
    ref = _oracle(p, depth=False)
    for k in ("abs", "marg", "yaw"):
        assert np.array_equal(out[k], ref[k])
