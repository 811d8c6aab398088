"""The random-gather probe behind the benchmark's gather roofline: it measures a positive rate,
L2-resident buffers are served faster than buffers beyond L2, and bad arguments are rejected."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2609_40297_gb300 as mig  # noqa: E402


def test_probe_gather_rates():
    with mig.Context(0) as ctx:
        l2 = mig.probe_gather(ctx, 16 << 20, 1)
        hbm = mig.probe_gather(ctx, 1 << 30, 1)
        tex = mig.probe_gather(ctx, 32 << 20, 4)
        assert l2 > 1e10 and hbm > 1e9 and tex > 1e10
        assert l2 > hbm
        for bad in ((16 << 20, 2), (100, 1), (1 << 33, 1)):
            with pytest.raises(mig.MigError):
                mig.probe_gather(ctx, *bad)
