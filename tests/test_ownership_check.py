"""The ownership check of Sec. IV-A ("Verification": a synaptic interaction or post-synaptic neuron
accessed by two threads is an error), as a debug mode of the ring delivery.

CPU: the host checker against a synthetic stamp array -- correct stamps pass, a planted stamp of
the wrong warp or block is reported with its cell.  GPU: every parity configuration of the ring
kernel run once in check mode: no cell is written by a second warp (the device count is zero), the
stamps name the plan's owner of every written cell, and the raster still equals the oracle."""
import numpy as np
import pytest

from paper_2406_03762_gb300 import cortex
from paper_2406_03762_gb300 import workloads as W


def _owner_stamps(n, depth, tb, warps, first_block, written):
    tw = -(-tb // warps)
    st = np.zeros((depth, n), np.uint32)
    for s, i in written:
        g, local = i // tb, i % tb
        st[s, i] = (first_block + g) * 16 + local // tw + 1
    return st


def test_host_checker_accepts_the_plan_and_reports_a_planted_overlap():
    n, depth, tb, warps, fb = 1000, 5, 300, 4, 2
    rng = np.random.default_rng(0)
    written = set(zip(rng.integers(0, depth, 3000).tolist(), rng.integers(0, n, 3000).tolist()))
    st = _owner_stamps(n, depth, tb, warps, fb, written)
    assert cortex.check_stamps(st, tb, warps, fb) == (0, -1)
    # a cell of target 310 (block 1, warp 0) stamped by warp 1 of the same block
    bad = st.copy()
    bad[2, 310] = (fb + 1) * 16 + 1 + 1
    assert cortex.check_stamps(bad, tb, warps, fb) == (1, 2 * n + 310)
    # a cell of target 5 (block 0) stamped by block 1's warp 0, and one of the last block's targets
    bad[0, 5] = (fb + 1) * 16 + 0 + 1
    bad[4, 999] = (fb + 0) * 16 + 3 + 1
    nb, first = cortex.check_stamps(bad, tb, warps, fb)
    assert nb == 3 and first == 5
    # the block numbering of a later network in a batch matters
    assert cortex.check_stamps(st, tb, warps, fb + 1)[0] > 0


GPU_CASES = [
    (W.CONFIGS["c0"]["spec"], dict()),
    (W.CONFIGS["c0"]["spec"], dict(ring=2)),
    (W.CONFIGS["c0"]["spec"], dict(mode=1)),
    (W.CONFIGS["c0"]["spec"], dict(warps_per_block=4, steps_per_launch=97)),
    (W.CONFIGS["c0"]["spec"], dict(warps_per_block=16, ring=2)),
    (W.NetSpec(4000, 1000, 400, 100, d_min=5, d_max=40, nu_ext_hz=12000.0), dict()),
    (W.NetSpec(800, 200, 900, 225, weight_dtype=W.BF16), dict()),
    (W.NetSpec(800, 200, 900, 225, weight_dtype=W.BF16), dict(fold=1, ring=2)),
]


@pytest.mark.gpu
@pytest.mark.parametrize("spec,opts", GPU_CASES)
def test_every_ring_configuration_passes_the_ownership_check(cortex, spec, opts):
    import torch
    from helpers import first_mismatch, oracle_run
    seed, steps = 9, 600
    o = cortex.make_options(check_ownership=1, **opts)
    with cortex.Network(spec, seed, o) as net:
        net.simulate(steps)          # raises CortexError(ERR_CHECK) on a violation
        gs, gi = net.spikes()
        st = net.stamps()
    props = torch.cuda.get_device_properties(0)
    tb, _ = cortex.plan([spec], o, n_sm=props.multi_processor_count,
                        smem_per_block=getattr(props, "shared_memory_per_block_optin", 232448))
    assert np.count_nonzero(st) > 0
    assert cortex.check_stamps(st, int(tb[0]), min(opts.get("warps_per_block", 14), 16), 0) == (0, -1)
    _, os_, oi, _ = oracle_run(spec, seed, steps)
    assert first_mismatch(gs, gi, os_, oi) == -1


@pytest.mark.gpu
def test_batch_passes_the_ownership_check(cortex):
    import torch
    specs, seeds = W.small_batch_specs()
    o = cortex.make_options(check_ownership=1, balance=2, net_work=[20.0, 1.0, 0.5, 3.0, 1.0, 8.0])
    props = torch.cuda.get_device_properties(0)
    tb, _ = cortex.plan(specs, o, n_sm=props.multi_processor_count,
                        smem_per_block=getattr(props, "shared_memory_per_block_optin", 232448))
    with cortex.Network(specs, seeds, o) as net:
        net.simulate(500)
        first = 0
        for b, spec in enumerate(specs):
            st = net.stamps(b)
            assert cortex.check_stamps(st, int(tb[b]), 14, first) == (0, -1), b
            first += -(-spec.n // int(tb[b]))
    with pytest.raises(cortex.CortexError) as e:
        cortex.Network(specs, seeds, cortex.make_options(check_ownership=1, delivery=1))
    assert e.value.code == cortex.ERR_UNSUPPORTED
