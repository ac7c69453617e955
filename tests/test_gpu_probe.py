"""The L2 reduction probe (snn_probe_reductions): every operation lands,
scattered or sweeping, and bad arguments are refused before any work."""
import pytest

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("pattern", [0, 1], ids=["scatter", "sweep"])
def test_every_reduction_lands(pattern):
    import torch
    from paper_2109_12855_gb300 import snn
    n_cells, n_ops = (1 << 20) + 7, 3 << 20
    buf = torch.zeros(n_cells, device="cuda")
    ms = snn.snn_probe_reductions(buf, n_ops, pattern)
    assert ms > 0.0
    counts = buf.to(torch.int64)
    assert torch.equal(counts.to(buf.dtype), buf)       # whole numbers
    assert int(counts.sum()) == n_ops
    if pattern == snn.SNN_PROBE_SWEEP:
        # cell c is hit by every k = c mod n_cells
        q, r = divmod(n_ops, n_cells)
        assert int(counts[:r].min()) == int(counts[:r].max()) == q + 1
        assert int(counts[r:].min()) == int(counts[r:].max()) == q
    else:
        # scattered: about n_ops / n_cells per cell, spread over the cells
        assert (counts > 0).float().mean().item() > 0.9
        assert int(counts.max()) < 30


def test_probe_rejects_bad_arguments():
    import torch
    from paper_2109_12855_gb300 import snn
    buf = torch.zeros(1024, device="cuda")
    with pytest.raises(snn.SnnError) as e:
        snn.snn_probe_reductions(buf, 0, 0)
    assert e.value.code == snn.SNN_E_ARG
    with pytest.raises(snn.SnnError):
        snn.snn_probe_reductions(buf, 10, 7)
    with pytest.raises(ValueError):
        snn.snn_probe_reductions(torch.zeros(16), 10, 0)    # host tensor
    assert float(buf.abs().sum()) == 0.0
