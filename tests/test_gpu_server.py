"""Serving loop: requests submitted together run in one continuous batch, and each result equals a
lone mig_tree_eval on the map as it was when the request was submitted, also when map updates
are interleaved with the requests (copy-on-write snapshots) and under a tight memory budget."""
import threading

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
    c = mig.Context(0, stream=torch.cuda.Stream())
    yield c
    c.close()


def _problems(k=8):
    sensors = [None, Sensor(87, 58, 48, 28, 2.0, 12, 10.0), Sensor(60, 45, 33, 17, 3.0, 5, -20.0)]
    return [synth.random_small(60 + i, n_nodes=8 + 5 * i, max_depth=2 + i % 5, sensor=sensors[i % 3])
            for i in range(k)]


def _alone(ctx, p, grid):
    m = mig.Map(ctx, grid, p.map.voxel_size, p.map.origin)
    try:
        return mig.tree_eval(m, p.tree.parent, p.tree.pos, p.sensor)
    finally:
        m.close()


def test_mix_equals_alone(ctx):
    probs = _problems(10)
    maps = [mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin) for p in probs]
    srv = mig.Server(ctx, arena_budget_bytes=1 << 30, max_inflight=16)
    try:
        subs = [srv.submit(m, p.tree.parent, p.tree.pos, p.sensor) for p, m in zip(probs, maps)]
        for t, _ in subs:
            assert srv.poll(t, timeout_us=30_000_000)
        for (t, out), p in zip(subs, probs):
            ref = _alone(ctx, p, p.map.grid)
            for k in ("abs", "marg", "yaw"):
                assert np.array_equal(out[k], ref[k]), (p.name, k)
            tm = srv.timing(t)
            assert 0 <= tm["admit_us"] <= tm["start_us"] <= tm["done_us"]
    finally:
        srv.close()
        for m in maps:
            m.close()


def test_map_updates_keep_snapshots(ctx):
    rng = np.random.default_rng(3)
    base = synth.random_small(70, n_nodes=30, max_depth=6)
    m = mig.Map(ctx, base.map.grid, base.map.voxel_size, base.map.origin)
    srv = mig.Server(ctx, arena_budget_bytes=1 << 30, max_inflight=8)
    grids = [base.map.grid.copy()]
    subs = []
    try:
        g = base.map.grid.copy()
        nz, ny, nx = g.shape
        for i in range(6):
            subs.append((srv.submit(m, base.tree.parent, base.tree.pos, base.sensor), len(grids) - 1))
            box = rng.integers(0, 3, size=(nz, ny // 2, nx // 2)).astype(np.uint8)
            x0, y0 = int(rng.integers(0, nx - nx // 2)), int(rng.integers(0, ny - ny // 2))
            srv.map_update(m, x0, y0, 0, box)
            g = g.copy()
            g[:, y0:y0 + ny // 2, x0:x0 + nx // 2] = box
            grids.append(g)
        subs.append((srv.submit(m, base.tree.parent, base.tree.pos, base.sensor), len(grids) - 1))
        for (t, out), gi in subs:
            assert srv.poll(t, timeout_us=30_000_000)
            ref = _alone(ctx, base, grids[gi])
            for k in ("abs", "marg", "yaw"):
                assert np.array_equal(out[k], ref[k]), (gi, k)
    finally:
        srv.close()
    assert np.array_equal(m.read(), grids[-1])  # the map ends with every update applied
    m.close()


def test_map_snapshots_count_against_the_budget(ctx):
    """Requests and map updates interleaved on one map. An update that arrives while requests read
    the map's grid copies it (the requests keep the old one); that copy counts against the budget
    like the requests' own bytes. With a budget below one request plus a grid copy, the update waits
    for the request to finish instead of copying: the server's peak holding stays exactly one
    request's bytes. With a large budget the server may copy. Every result equals the oracle on the
    map as submitted, and nothing is held at the end."""
    rng = np.random.default_rng(9)
    base = synth.random_small(71, nx=48, ny=40, nz=16, n_nodes=12, max_depth=4)
    g0 = base.map.grid.copy()
    nz, ny, nx = g0.shape
    updates, grids, g = [], [g0], g0
    for i in range(4):
        box = rng.integers(0, 3, size=(nz, ny // 2, nx // 2)).astype(np.uint8)
        x0, y0 = int(rng.integers(0, nx - nx // 2)), int(rng.integers(0, ny - ny // 2))
        updates.append((x0, y0, box))
        g = g.copy()
        g[:, y0:y0 + ny // 2, x0:x0 + nx // 2] = box
        grids.append(g)
    refs = [oracle.eval_tree(gi, base.map.voxel_size, base.map.origin, base.tree.parent, base.tree.pos, base.sensor)
            for gi in grids]

    def serve(budget, n_grids):
        m = mig.Map(ctx, g0, base.map.voxel_size, base.map.origin)
        srv = mig.Server(ctx, arena_budget_bytes=budget, max_inflight=8)
        subs = []
        try:
            for i in range(n_grids):
                subs.append((srv.submit(m, base.tree.parent, base.tree.pos, base.sensor), i))
                subs.append((srv.submit(m, base.tree.parent, base.tree.pos, base.sensor), i))
                if i < n_grids - 1:
                    x0, y0, box = updates[i]
                    srv.map_update(m, x0, y0, 0, box)
            for (t, out), gi in subs:
                assert srv.poll(t, timeout_us=60_000_000)
                for k in ("abs", "marg", "yaw"):
                    assert np.array_equal(out[k], refs[gi][k]), (budget, gi, k)
            mem = srv.memory()
        finally:
            srv.close()
            m.close()
        return mem

    alone = serve(1, 1)  # budget 1: one request at a time; this run has no update
    one_request = alone["peak"]
    assert one_request > 0
    tight = serve(1, len(grids))
    assert tight["peak"] == one_request and tight["snapshots"] == 0 and tight["in_use"] == 0
    big = serve(1 << 30, len(grids))
    assert big["snapshots"] == 0 and big["in_use"] == 0 and big["peak"] >= one_request


def test_tight_budget_and_threads(ctx):
    probs = _problems(6)
    maps = [mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin) for p in probs]
    srv = mig.Server(ctx, arena_budget_bytes=1, max_inflight=3)  # one request at a time
    results = {}
    try:
        def client(i):
            p, m = probs[i], maps[i]
            t, out = srv.submit(m, p.tree.parent, p.tree.pos, p.sensor)
            assert srv.poll(t, timeout_us=60_000_000)
            results[i] = out
        th = [threading.Thread(target=client, args=(i,)) for i in range(len(probs))]
        for x in th:
            x.start()
        for x in th:
            x.join()
        for i, p in enumerate(probs):
            ref = _alone(ctx, p, p.map.grid)
            for k in ("abs", "marg", "yaw"):
                assert np.array_equal(results[i][k], ref[k])
        with pytest.raises(mig.MigError) as e:
            srv.poll(10 ** 9)
        assert e.value.status == mig.MIG_ENOTFOUND
    finally:
        srv.close()
        for m in maps:
            m.close()


def test_destroy_drains_pending_requests(ctx):
    probs = _problems(4)
    maps = [mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin) for p in probs]
    srv = mig.Server(ctx, arena_budget_bytes=1 << 30, max_inflight=2)
    subs = [srv.submit(m, p.tree.parent, p.tree.pos, p.sensor) for p, m in zip(probs, maps)]
    srv.close()  # waits for the queue and the requests in flight
    for (t, out), p in zip(subs, probs):
        ref = _alone(ctx, p, p.map.grid)
        assert np.array_equal(out["marg"], ref["marg"])
    for m in maps:
        m.close()


def test_interval_and_panoramic_requests_in_the_mix(ctx):
    """Requests of the interval and panoramic modes served beside marginal ones: each result equals
    a lone evaluation in its mode."""
    probs = [synth.random_small(80 + i, n_nodes=9 + 4 * i, max_depth=2 + i % 4, sensor=Sensor(90, 60, 16, 10, 2.0, 8, 0.0))
             for i in range(6)]
    modes = [mig.MODE_MARGINAL, mig.MODE_INTERVAL, mig.MODE_PANORAMIC] * 2
    maps = [mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin) for p in probs]
    srv = mig.Server(ctx, arena_budget_bytes=1 << 30, max_inflight=16)
    try:
        subs = [srv.submit(m, p.tree.parent, p.tree.pos, p.sensor, mode=md) for p, m, md in zip(probs, maps, modes)]
        for t, _ in subs:
            assert srv.poll(t, timeout_us=30_000_000)
        for (t, out), p, m, md in zip(subs, probs, maps, modes):
            ref = mig.tree_eval(m, p.tree.parent, p.tree.pos, p.sensor, mode=md)
            for k in ("abs", "marg", "yaw"):
                assert np.array_equal(out[k], ref[k]), (p.name, md, k)
        with pytest.raises(mig.MigError):  # panoramic needs a level camera
            srv.submit(maps[0], probs[0].tree.parent, probs[0].tree.pos, Sensor(90, 60, 16, 10, 2.0, 8, 10.0),
                       mode=mig.MODE_PANORAMIC)
    finally:
        srv.close()
        for m in maps:
            m.close()
