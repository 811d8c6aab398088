"""Batched engine: many trees on different maps and sensors in one persistent launch give the
same results as separate evaluations (and as the oracle); the captured CUDA graph is replayed;
a device-side wait that runs out returns MIG_ETIMEOUT and leaves the context usable."""
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


def _problems():
    ps = [synth.tiny()]
    sensors = [None, Sensor(87, 58, 48, 28, 2.0, 12, 10.0), Sensor(60, 45, 33, 17, 3.0, 5, -20.0),
               Sensor(120, 90, 7, 5, 2.5, 3, 0.0)]
    for i, s in enumerate(sensors):
        ps.append(synth.random_small(40 + i, n_nodes=10 + 7 * i, max_depth=3 + i, sensor=s))
    ps.append(synth.random_small(50, n_nodes=1, max_depth=1))  # a lone root
    return ps


@pytest.fixture(scope="module")
def ctx():
    stream = torch.cuda.Stream()  # a capturable stream: batches replay a CUDA graph
    c = mig.Context(0, stream=stream)
    yield c
    c.close()


@pytest.mark.parametrize("engine", [0, 1])
def test_batch_equals_single_evaluations(ctx, engine):
    probs = _problems()
    maps = [mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin) for p in probs]
    tw, th, cps, eng0 = ctx.get_tiles()
    ctx.set_tiles(tw, th, cps, engine)
    try:
        for mode in (mig.MODE_MARGINAL, mig.MODE_SINGLE_PARENT, mig.MODE_ABSOLUTE):
            outs = mig.tree_eval_batch(ctx, [(p.tree.parent, p.tree.pos, p.sensor) for p in probs], maps, mode=mode)
            for p, m, o in zip(probs, maps, outs):
                single = mig.tree_eval(m, p.tree.parent, p.tree.pos, p.sensor, mode=mode)
                for k in ("abs", "marg", "yaw"):
                    assert np.array_equal(o[k], single[k]), (p.name, mode, k)
        ref = oracle.eval_tree(probs[1].map.grid, probs[1].map.voxel_size, probs[1].map.origin, probs[1].tree.parent,
                               probs[1].tree.pos, probs[1].sensor)
        outs = mig.tree_eval_batch(ctx, [(p.tree.parent, p.tree.pos, p.sensor) for p in probs], maps)
        for k in ("abs", "marg", "yaw"):
            assert np.array_equal(outs[1][k], ref[k])
    finally:
        ctx.set_tiles(tw, th, cps, eng0)
        for m in maps:
            m.close()


@pytest.mark.parametrize("engine", [0, 1])
def test_batch_graph_replay_same_results(ctx, engine):
    probs = _problems()[:4]
    maps = [mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin) for p in probs]
    tw, th, cps, eng0 = ctx.get_tiles()
    ctx.set_tiles(tw, th, cps, engine)
    try:
        args = [(p.tree.parent, p.tree.pos, p.sensor) for p in probs]
        a = mig.tree_eval_batch(ctx, args, maps)
        cap0, rep0 = ctx.graph_stats()
        b = mig.tree_eval_batch(ctx, args, maps)
        c = mig.tree_eval_batch(ctx, args, maps)
        cap1, rep1 = ctx.graph_stats()
        assert rep1 - rep0 == 2 and cap1 == cap0
        for x, y, z in zip(a, b, c):
            for k in ("abs", "marg", "yaw"):
                assert np.array_equal(x[k], y[k]) and np.array_equal(x[k], z[k])
    finally:
        ctx.set_tiles(tw, th, cps, eng0)
        for m in maps:
            m.close()


def test_batch_wait_timeout_is_reported_and_recoverable(ctx):
    """The persistent engine's device-side waits are bounded (engine 0)."""
    probs = _problems()[:3]
    maps = [mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin) for p in probs]
    args = [(p.tree.parent, p.tree.pos, p.sensor) for p in probs]
    tw, th, cps, eng0 = ctx.get_tiles()
    ctx.set_tiles(tw, th, cps, 0)
    try:
        good = mig.tree_eval_batch(ctx, args, maps)
        ctx.set_batch_timeout(200_000, debug_stall=True)  # 0.2 s; one level never completes
        with pytest.raises(mig.MigError) as e:
            mig.tree_eval_batch(ctx, args, maps)
        assert e.value.status == mig.MIG_ETIMEOUT
        ctx.set_batch_timeout(5_000_000, debug_stall=False)
        again = mig.tree_eval_batch(ctx, args, maps)
        for x, y in zip(good, again):
            for k in ("abs", "marg", "yaw"):
                assert np.array_equal(x[k], y[k])
    finally:
        ctx.set_batch_timeout(5_000_000, debug_stall=False)
        ctx.set_tiles(tw, th, cps, eng0)
        for m in maps:
            m.close()


def test_batch_larger_than_one_launch(ctx):
    """More trees than one persistent launch takes (they split into several launches) and more than
    the trees it keeps in flight: every result equals its single evaluation."""
    probs = [synth.random_small(900 + i, n_nodes=3 + i % 9, max_depth=1 + i % 4, sensor=Sensor(80, 55, 12, 9, 2.0, 4 + i % 5, 0.0))
             for i in range(110)]
    maps = [mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin) for p in probs[:10]]
    tw, th, cps, eng0 = ctx.get_tiles()
    ctx.set_tiles(tw, th, cps, 0)
    try:
        trees = [(p.tree.parent, p.tree.pos, p.sensor) for p in probs]
        tmaps = [maps[i % 10] for i in range(len(probs))]
        outs = mig.tree_eval_batch(ctx, trees, tmaps)
        for i, (t, m, o) in enumerate(zip(trees, tmaps, outs)):
            single = mig.tree_eval(m, *t)
            for k in ("abs", "marg", "yaw"):
                assert np.array_equal(o[k], single[k]), (i, k)
    finally:
        ctx.set_tiles(tw, th, cps, eng0)
        for m in maps:
            m.close()


def test_batch_empty_and_invalid(ctx):
    assert mig.tree_eval_batch(ctx, [], []) == []
    p = synth.tiny()
    m = mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin)
    try:
        bad = p.tree.parent.copy()
        bad[3] = 3
        with pytest.raises(mig.MigError) as e:
            mig.tree_eval_batch(ctx, [(p.tree.parent, p.tree.pos, p.sensor), (bad, p.tree.pos, p.sensor)], [m, m])
        assert e.value.status == mig.MIG_EINVAL
    finally:
        m.close()


def test_autotune_picks_a_candidate_and_keeps_results(ctx, tmp_path):
    probs = _problems()[:4]
    maps = [mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin) for p in probs]
    keep = ctx.get_tiles()
    try:
        args = [(p.tree.parent, p.tree.pos, p.sensor) for p in probs]
        before = mig.tree_eval_batch(ctx, args, maps)
        cands = [(4, 16, 4, 1), (8, 8, 4, 1), (4, 16, 4, 0), (32, 8, 2, 0)]
        cache = str(tmp_path / "tiles.json")
        best, times = mig.autotune(ctx, args, maps, candidates=cands, reps=1, cache_path=cache)
        assert best in cands and set(times) == set(cands) and ctx.get_tiles() == best
        after = mig.tree_eval_batch(ctx, args, maps)
        for x, y in zip(before, after):
            for k in ("abs", "marg", "yaw"):
                assert np.array_equal(x[k], y[k])
        ctx.set_tiles(*keep)
        best2, _ = mig.autotune(ctx, args, maps, candidates=cands, reps=1, cache_path=cache)  # cache hit
        assert best2 == best and ctx.get_tiles() == best
    finally:
        ctx.set_tiles(*keep)
        for m in maps:
            m.close()


@pytest.mark.parametrize("engine", [0, 1])
def test_batch_graph_survives_buffer_regrowth(ctx, engine):
    """A captured batch graph copies through the context's pinned staging buffer and device
    workspace. When a larger call regrows them, the old graph is dropped, never replayed into freed
    memory: the small batch recaptures and returns the same results."""
    small = _problems()[:3]
    big = [synth.random_small(60 + i, n_nodes=2000, max_depth=12) for i in range(20)]  # > 1 MiB of plan data
    maps = [mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin) for p in small + big]
    tw, th, cps, eng0 = ctx.get_tiles()
    ctx.set_tiles(tw, th, cps, engine)
    try:
        args = [(p.tree.parent, p.tree.pos, p.sensor) for p in small]
        a = mig.tree_eval_batch(ctx, args, maps[:3])
        a2 = mig.tree_eval_batch(ctx, args, maps[:3])  # a replay of the captured graph
        cap0, _ = ctx.graph_stats()
        mig.tree_eval_batch(ctx, [(p.tree.parent, p.tree.pos, p.sensor) for p in big], maps[3:])
        b = mig.tree_eval_batch(ctx, args, maps[:3])
        cap1, _ = ctx.graph_stats()
        assert cap1 >= cap0 + 1  # the big batch and the small one were captured anew
        for x, y, z in zip(a, a2, b):
            for k in ("abs", "marg", "yaw"):
                assert np.array_equal(x[k], y[k]) and np.array_equal(x[k], z[k])
    finally:
        ctx.set_tiles(tw, th, cps, eng0)
        for m in maps:
            m.close()


@pytest.mark.parametrize("mode", [mig.MODE_INTERVAL, mig.MODE_PANORAMIC])
def test_batch_interval_and_panoramic_modes(ctx, mode):
    """The interval and panoramic modes in a batch (on the stream-chain engine, whichever engine is
    set) equal separate evaluations; the panoramic batch uses level cameras only."""
    probs = [p for p in _problems() if p.sensor.pitch_deg == 0 or mode == mig.MODE_INTERVAL]
    maps = [mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin) for p in probs]
    tw, th, cps, eng0 = ctx.get_tiles()
    try:
        for engine in (0, 1):
            ctx.set_tiles(tw, th, cps, engine)
            outs = mig.tree_eval_batch(ctx, [(p.tree.parent, p.tree.pos, p.sensor) for p in probs], maps, mode=mode)
            for p, m, o in zip(probs, maps, outs):
                single = mig.tree_eval(m, p.tree.parent, p.tree.pos, p.sensor, mode=mode)
                for k in ("abs", "marg", "yaw"):
                    assert np.array_equal(o[k], single[k]), (p.name, mode, engine, k)
        if mode == mig.MODE_PANORAMIC:
            pitched = synth.random_small(44, n_nodes=6, sensor=Sensor(87, 58, 48, 28, 2.0, 12, 10.0))
            mp = mig.Map(ctx, pitched.map.grid, pitched.map.voxel_size, pitched.map.origin)
            try:
                with pytest.raises(mig.MigError):
                    mig.tree_eval_batch(ctx, [(pitched.tree.parent, pitched.tree.pos, pitched.sensor)], [mp], mode=mode)
            finally:
                mp.close()
    finally:
        ctx.set_tiles(tw, th, cps, eng0)
        for m in maps:
            m.close()
