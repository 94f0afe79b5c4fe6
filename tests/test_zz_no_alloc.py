"""The allocation-free sub-graph entry point (cortex_subgraph_noalloc), called through the C ABI.

It serves callers that cannot call the device allocator: it builds the incoming synapses of a
target range into buffers the caller owns, using one static device array as working memory.  Its
output must equal what the regular path (cortex_export_synapses on a built network) reports for the
same targets, on two calls in a row (the shared array keeps the previous call's contents).  This
file is collected last so that a first failure here leaves every other test already run."""
import numpy as np
import pytest

from paper_2406_03762_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("spec,t0,t1", [
    (W.NetSpec(800, 200, 80, 20), 100, 350),
    (W.NetSpec(1600, 400, 300, 75, d_min=3, d_max=30, weight_dtype=W.BF16), 0, 2000),
])
def test_noalloc_subgraph_matches_regular_path(cortex, spec, t0, t1):
    import torch

    seed = 31
    with cortex.Network(spec, seed) as net:
        s, t, d, w = net.export_synapses(t0, t1)
    want = sorted(zip(t.tolist(), s.tolist(), d.tolist(), w.tolist()))
    n, nnz = spec.n, (t1 - t0) * spec.k
    for call in range(2):
        row = torch.full((n + 1,), -1, dtype=torch.int32, device="cuda")
        tg = torch.full((nnz,), -1, dtype=torch.int32, device="cuda")
        dl = torch.full((nnz,), -1, dtype=torch.int32, device="cuda")
        wt = torch.full((nnz,), float("nan"), dtype=torch.float32, device="cuda")
        cortex.subgraph_noalloc(spec, seed, t0, t1, row, tg, dl, wt)
        row_h = row.cpu().numpy()
        assert row_h[0] == 0 and row_h[-1] == nnz and np.all(np.diff(row_h) >= 0)
        src = np.repeat(np.arange(n), np.diff(row_h))
        tg_h, dl_h, wt_h = tg.cpu().numpy(), dl.cpu().numpy(), wt.cpu().numpy()
        # rows ordered by target inside each source
        for a in range(0, n, max(1, n // 50)):
            seg = tg_h[row_h[a]:row_h[a + 1]]
            assert np.all(np.diff(seg) >= 0)
        got = sorted(zip(tg_h.tolist(), src.tolist(), dl_h.tolist(), wt_h.tolist()))
        assert got == want, f"call {call}"


def test_noalloc_rejects_sizes_beyond_its_array(cortex):
    import torch

    spec = W.NetSpec(800000, 200000, 9000, 2250)
    nnz = 1000 * spec.k  # buffers of the right size: the library's own limit refuses the request
    row = torch.empty(spec.n + 1, dtype=torch.int32, device="cuda")
    buf = torch.empty(nnz, dtype=torch.int32, device="cuda")
    wt = torch.empty(nnz, dtype=torch.float32, device="cuda")
    with pytest.raises(cortex.CortexError) as e:
        cortex.subgraph_noalloc(spec, 1, 0, 1000, row, buf, buf, wt)
    assert e.value.code == cortex.ERR_UNSUPPORTED
    assert "2^21" in str(e.value)


def test_noalloc_reports_a_source_over_its_per_source_cap(cortex):
    """One inhibitory neuron drawn by every target of a 3,001-target range: that source has 3,001
    synapses in the range, above the 2,048 a source may have.  The device finds it and the call
    returns CORTEX_ERR_UNSUPPORTED with its own message (the outputs are then undefined)."""
    import torch

    spec = W.NetSpec(3000, 1, 1, 1)
    n, nnz = spec.n, spec.n * spec.k
    row = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    tg = torch.empty(nnz, dtype=torch.int32, device="cuda")
    dl = torch.empty(nnz, dtype=torch.int32, device="cuda")
    wt = torch.empty(nnz, dtype=torch.float32, device="cuda")
    with pytest.raises(cortex.CortexError) as e:
        cortex.subgraph_noalloc(spec, 3, 0, n, row, tg, dl, wt)
    assert e.value.code == cortex.ERR_UNSUPPORTED
    assert "2048" in str(e.value)
