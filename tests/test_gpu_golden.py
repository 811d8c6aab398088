"""Whole-workload parity against stored oracle results (tests/golden/*.npz, written by the
oracle/make_*_golden.py scripts, which call only the oracle and the seeded generators):

- the 800x800x200 workload: all 2000 nodes, per-(node, yaw) counts and yaws, through the
  device-resident call that the benchmark times;
- the 64-tree batch (64 maps, trees of 50-2000 nodes, ray grids 64x48 ... 320x240), every tree,
  through the batched call on both engines;
- the serving workload's first requests with their interleaved map updates, served together by the
  continuous-batching server, each against the oracle on its map as submitted.

Each file records the SHA-256 of the inputs the oracle saw; a different generator output on this
machine is reported as such, not as a parity failure.
"""
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2609_40297_gb300 as mig  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    path = os.path.join(GOLDEN, name)
    assert os.path.exists(path), f"{path} missing: run oracle/make_*_golden.py"
    return np.load(path)


def _first_diff(a, b):
    bad = np.argwhere(np.asarray(a) != np.asarray(b))
    return f"{len(bad)} mismatches, first at {bad[:5].tolist()}"


def test_large_workload_all_nodes_match_oracle():
    g = _load("large_oracle.npz")
    p = synth.large()
    sha = synth.sha256(p.map.grid, p.tree.parent, p.tree.pos)
    assert sha == str(g["inputs_sha256"]), "the generator produced different inputs on this machine"
    t = oracle.camera_tables(p.sensor)
    cam_sha = synth.sha256(t["body"], t["dzc"], t["ck"], t["sk"], t["M"])
    assert cam_sha == str(g["camera_sha256"]), "this host's libm gives different camera tables"
    s = p.sensor
    n = p.tree.n
    dev = torch.device("cuda", 0)
    with mig.Context(0) as ctx:
        m = mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin)
        try:
            # the benchmark's timed call: tree and outputs resident on the device
            par = torch.from_numpy(p.tree.parent).to(dev)
            pos = torch.from_numpy(p.tree.pos).to(dev)
            outs = [torch.empty(n, dtype=torch.int32, device=dev) for _ in range(3)]
            mig.tree_eval_device(m, par, pos, s, int(p.tree.depth().max()), *outs)
            ctx.sync()
            got = dict(zip(("abs", "marg", "yaw"), (o.cpu().numpy() for o in outs)))
            # the host-array call with per-(node, yaw) counts
            full = mig.tree_eval(m, p.tree.parent, p.tree.pos, s, want_counts=True)
        finally:
            m.close()
    for k in ("abs", "marg", "yaw"):
        assert np.array_equal(got[k], g[k]), f"device call {k}: {_first_diff(got[k], g[k])}"
        assert np.array_equal(full[k], g[k]), f"host call {k}: {_first_diff(full[k], g[k])}"
    for k in ("cnt_abs", "cnt_marg"):
        assert np.array_equal(full[k], g[k]), f"{k}: {_first_diff(full[k], g[k])}"


@pytest.mark.parametrize("engine", [0, 1])
def test_batched_workload_every_tree_matches_oracle(engine):
    g = _load("batched_oracle.npz")
    off = g["offsets"]
    probs = synth.batched(seed_base=404, n_trees=len(off) - 1)
    for i, p in enumerate(probs):
        assert synth.sha256(p.map.grid, p.tree.parent, p.tree.pos) == str(g["inputs_sha256"][i]), f"tree {i} inputs"
    with mig.Context(0, stream=torch.cuda.Stream()) as ctx:
        maps = [mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin) for p in probs]
        try:
            tw, th, cps, _ = ctx.get_tiles()
            ctx.set_tiles(tw, th, cps, engine)
            outs = mig.tree_eval_batch(ctx, [(p.tree.parent, p.tree.pos, p.sensor) for p in probs], maps)
        finally:
            for m in maps:
                m.close()
    for i, o in enumerate(outs):
        for k in ("abs", "marg", "yaw"):
            ref = g[k][off[i]:off[i + 1]]
            assert np.array_equal(o[k], ref), f"engine {engine} tree {i} {k}: {_first_diff(o[k], ref)}"


def test_serving_requests_match_oracle():
    g = _load("serving_oracle.npz")
    off = g["offsets"]
    maps_spec, pools, events, sensor, updates = synth.serving_requests(n_first=len(off) - 1)
    grids = [m.grid for m in maps_spec]
    for i, (_, rid, mi, ti) in enumerate(events):  # the map each request sees, in arrival order
        grids[mi] = synth.apply_update(grids[mi], updates[i])
        tr = pools[rid][1][ti]
        assert synth.sha256(grids[mi], tr.parent, tr.pos) == str(g["inputs_sha256"][i]), f"request {i} inputs"
    with mig.Context(0, stream=torch.cuda.Stream()) as ctx:
        maps = [mig.Map(ctx, m.grid, m.voxel_size, m.origin) for m in maps_spec]
        srv = mig.Server(ctx, arena_budget_bytes=8 << 30, max_inflight=4)
        try:
            tickets = []
            for i, (_, rid, mi, ti) in enumerate(events):
                (x0, y0, z0, dx, dy, dz), vox = updates[i]
                srv.map_update(maps[mi], x0, y0, z0, vox)
                tr = pools[rid][1][ti]
                tickets.append(srv.submit(maps[mi], tr.parent, tr.pos, sensor))
            for t, _ in tickets:
                assert srv.poll(t, timeout_us=120_000_000)
        finally:
            srv.close()
            for m in maps:
                m.close()
    for i, (_, out) in enumerate(tickets):
        for k in ("abs", "marg", "yaw"):
            ref = g[k][off[i]:off[i + 1]]
            assert np.array_equal(out[k], ref), f"request {i} {k}: {_first_diff(out[k], ref)}"
