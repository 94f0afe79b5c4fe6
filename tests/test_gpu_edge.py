"""Degenerate networks and a batch of networks with different delay ranges on the GPU, against the
oracle (the oracle is pinned on the same networks by tests/test_oracle_edge.py), in both delivery
schemes: raster, final state and event count bit for bit."""
import numpy as np
import pytest

from helpers import first_mismatch, oracle_run
from paper_2406_03762_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EDGE = {
    "no_drive": W.NetSpec(800, 200, 80, 20, nu_ext_hz=0.0),
    "indegree_0": W.NetSpec(800, 200, 0, 0),
    "exc_only": W.NetSpec(1000, 0, 100, 0, nu_ext_hz=12000.0),
    "single_delay": W.NetSpec(800, 200, 80, 20, d_min=3, d_max=3),
    "smaller_than_a_warp_share": W.NetSpec(32, 8, 8, 2, nu_ext_hz=18000.0),
    "one_neuron": W.NetSpec(1, 0, 1, 0, nu_ext_hz=20000.0),
}


@pytest.mark.parametrize("name", list(EDGE))
@pytest.mark.parametrize("delivery", [0, 1])
def test_degenerate_network_matches_oracle(cortex, name, delivery):
    spec, seed, steps = EDGE[name], 17, 600
    with cortex.Network(spec, seed, cortex.make_options(delivery=delivery)) as net:
        net.simulate(steps)
        gs, gi = net.spikes()
        gv, gc, gr = net.state()
        st = net.stats()
    ref, os_, oi, _ = oracle_run(spec, seed, steps)
    assert first_mismatch(gs, gi, os_, oi) == -1
    ov, oc, orr = ref.state()
    assert np.array_equal(gv.astype(np.float64), ov) and np.array_equal(gc.astype(np.float64), oc)
    assert np.array_equal(gr, orr)
    assert st["events"] == ref.events
    if name == "no_drive":
        assert len(gs) == 0 and not gc.any()
    if name == "indegree_0":
        assert st["events"] == 0 and len(gs) > 0


MIXED = [W.NetSpec(800, 200, 80, 20, d_min=1, d_max=16),
         W.NetSpec(1200, 300, 120, 30, d_min=3, d_max=20, nu_ext_hz=16000.0),
         W.NetSpec(1600, 400, 160, 40, d_min=5, d_max=40, nu_ext_hz=12000.0),
         W.NetSpec(400, 100, 40, 10, d_min=2, d_max=2, nu_ext_hz=17000.0)]


@pytest.mark.parametrize("opts", [dict(), dict(ring=2), dict(mode=1), dict(delivery=1)])
def test_batch_with_different_delay_ranges(cortex, opts):
    """Networks with d_min 1, 3, 5, 2 and d_max 16, 20, 40, 2 stepped together: every network has its
    own window of d_min + 1 steps, ring depth and barrier; each instance equals the oracle."""
    seeds = [41, 42, 43, 44]
    steps = 700
    with cortex.Network(MIXED, seeds, cortex.make_options(**opts)) as net:
        net.simulate(steps)
        res = [(net.spikes(b), net.state(b)) for b in range(len(MIXED))]
        st = net.stats()
    total = 0
    for b, (spec, seed) in enumerate(zip(MIXED, seeds)):
        ref, os_, oi, _ = oracle_run(spec, seed, steps)
        (gs, gi), (gv, gc, gr) = res[b]
        assert len(os_) > 50
        assert first_mismatch(gs, gi, os_, oi) == -1, f"network {b}"
        ov, _, _ = ref.state()
        assert np.array_equal(gv.astype(np.float64), ov), f"network {b}"
        total += ref.events
    assert st["events"] == total


# Layout limits that only the builder sees, on the device: a source with more than 2,048 synapses
# into one block (a piece over the staging cap; 10 targets in one block, each drawing 5,000 times
# from 10 sources) and a source whose row exceeds 65,535 synapses (16-bit piece offsets; 1,000
# excitatory sources each drawn about 100 times by every one of 100,000 targets).
OVER_LIMITS = {"piece_over_2048": W.NetSpec(10, 0, 5000, 0),
               "row_over_65535": W.NetSpec(1000, 99000, 1000, 0)}


@pytest.mark.parametrize("name", list(OVER_LIMITS))
@pytest.mark.parametrize("delivery", [0, 1])
def test_layout_limits_found_on_the_device_are_refused(cortex, name, delivery):
    """The build returns CORTEX_ERR_UNSUPPORTED with its reason and leaves no handle (nothing reads
    the pieces it did not write), and the context stays usable: the next network matches the
    oracle bit for bit."""
    with pytest.raises(cortex.CortexError) as e:
        cortex.Network(OVER_LIMITS[name], 3, cortex.make_options(delivery=delivery))
    assert e.value.code == cortex.ERR_UNSUPPORTED
    assert "staging capacity" in str(e.value)
    spec, seed, steps = EDGE["single_delay"], 5, 300
    with cortex.Network(spec, seed, cortex.make_options(delivery=delivery)) as net:
        net.simulate(steps)
        gs, gi = net.spikes()
    _, os_, oi, _ = oracle_run(spec, seed, steps)
    assert len(os_) > 0 and first_mismatch(gs, gi, os_, oi) == -1
