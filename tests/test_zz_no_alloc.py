"""The allocation-free entry point (mig_tree_eval_device_noalloc), called through the C ABI,
gives the same results as the regular device entry point (mig_tree_eval_device), on two
different trees in a row: the second call must not see the first call's leftover scratch.
Collected last (file name) so that a stop-at-first-failure run has run every other test."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2609_40297_gb300 as mig  # noqa: E402


def _dev_tree(p, dev):
    par = torch.from_numpy(p.tree.parent).to(dev)
    pos = torch.from_numpy(p.tree.pos).to(dev)
    return par, pos


def test_noalloc_matches_regular_entry_point_twice():
    dev = torch.device("cuda:0")
    problems = [synth.paper_scale(), synth.tiny()]  # the larger tree first, then a smaller one
    with mig.Context(0) as ctx:
        for p in problems:
            m = mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin)
            try:
                par, pos = _dev_tree(p, dev)
                md = int(p.tree.depth().max())
                ref = [torch.full((p.tree.n,), -7, dtype=torch.int32, device=dev) for _ in range(3)]
                got = [torch.full((p.tree.n,), -7, dtype=torch.int32, device=dev) for _ in range(3)]
                mig.tree_eval_device(m, par, pos, p.sensor, md, *ref)
                ctx.sync()
                mig.tree_eval_device_noalloc(m, par, pos, p.sensor, md, *got)
                ctx.sync()
                for name, a, b in zip(("abs", "marg", "yaw"), got, ref):
                    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy()), (p.name, name)
                assert ref[0].sum().item() > 0
            finally:
                m.close()


def test_noalloc_pitched_odd_sensor_and_many_yaws():
    """A pitched camera (20 deg nose down) with an odd, non-square image (37x23) and 130 yaw bins (a
    per-yaw table of two parameter-passed chunks): the scratch's camera tables, built on the device
    and from the host's per-yaw rows, give the regular entry point's results."""
    dev = torch.device("cuda:0")
    p = synth.random_small(77, n_nodes=15, max_depth=4, sensor=synth.Sensor(80, 55, 37, 23, 2.5, 130, 20.0))
    with mig.Context(0) as ctx:
        m = mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin)
        try:
            par, pos = _dev_tree(p, dev)
            md = int(p.tree.depth().max())
            ref = [torch.full((p.tree.n,), -7, dtype=torch.int32, device=dev) for _ in range(3)]
            got = [torch.full((p.tree.n,), -7, dtype=torch.int32, device=dev) for _ in range(3)]
            mig.tree_eval_device(m, par, pos, p.sensor, md, *ref)
            ctx.sync()
            mig.tree_eval_device_noalloc(m, par, pos, p.sensor, md, *got)
            ctx.sync()
            for name, a, b in zip(("abs", "marg", "yaw"), got, ref):
                assert np.array_equal(a.cpu().numpy(), b.cpu().numpy()), name
            assert ref[0].sum().item() > 0
        finally:
            m.close()


def test_noalloc_rejects_trees_above_the_scratch_size():
    dev = torch.device("cuda:0")
    p = synth.tiny()
    with mig.Context(0) as ctx:
        m = mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin)
        try:
            big = synth.Sensor(90, 60, 2048, 2048, 4.0, 8, 0.0)  # 16 MiB of depth buffer per node
            par, pos = _dev_tree(p, dev)
            outs = [torch.empty(p.tree.n, dtype=torch.int32, device=dev) for _ in range(3)]
            with pytest.raises(mig.MigError) as e:
                mig.tree_eval_device_noalloc(m, par, pos, big, 4, *outs)
            assert e.value.status == mig.MIG_EINVAL and "maximum" in str(e.value)
        finally:
            m.close()
