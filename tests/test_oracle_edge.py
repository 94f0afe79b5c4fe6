"""Degenerate networks on the oracle (CPU), each pinned by a property that holds exactly."""
import numpy as np

from helpers import oracle_params
from oracle import oracle as orc
from paper_2406_03762_gb300 import workloads as W


def _run(spec, steps, prec=orc.FP64, seed=5):
    net = orc.Network(oracle_params(spec, prec), seed)
    v0, c0, r0 = net.state()
    net.simulate(steps)
    return net, v0


def test_silent_network_decays_freely():
    """No drive: no neuron reaches threshold (V0 < V_th), I stays 0, and every V follows the free
    decay V0 exp(-t h / tau_m) of Eq. 1 (FP64, exact integration) -- recurrent synapses or not."""
    for k in ((0, 0), (8, 2)):
        spec = W.NetSpec(80, 20, k[0], k[1], nu_ext_hz=0.0)
        net, v0 = _run(spec, 200)
        s, _ = net.raster()
        v, c, r = net.state()
        assert len(s) == 0 and not c.any() and not r.any() and not net.ring().any()
        expect = v0 * np.exp(-200 * spec.dt / spec.tau_m)
        assert np.allclose(v, expect, rtol=1e-12, atol=0)


def test_unconnected_network_delivers_nothing():
    """In-degree 0 with drive: neurons spike on their Poisson drive alone, and no synaptic event
    is ever delivered."""
    net, _ = _run(W.NetSpec(80, 20, 0, 0), 500, prec=orc.FP32)
    s, _ = net.raster()
    assert len(s) > 0 and net.events == 0 and not net.ring().any()


def test_excitatory_only_network_has_no_negative_input():
    """Only excitatory sources (J_E > 0): every ring cell is a sum of positive weights."""
    net, _ = _run(W.NetSpec(100, 0, 10, 0), 300, prec=orc.FP32)
    s, _ = net.raster()
    ring = net.ring()
    assert len(s) > 0 and net.events > 0 and ring.min() >= 0.0 and ring.max() > 0.0


def test_single_delay_reaches_only_its_slots():
    """d_min = d_max = 3 (ring depth 4): after T steps the input pending for steps T .. T + 2
    comes from the spikes of steps T - 3 .. T - 1, and the slot of step T + 3 is always empty.
    Checked after every step of 300; the pending slots do fill."""
    spec = W.NetSpec(80, 20, 8, 2, d_min=3, d_max=3)
    net = orc.Network(oracle_params(spec, orc.FP32), 5)
    filled = 0
    for _ in range(300):
        net.simulate(1)
        t, ring = net.step, net.ring()
        assert ring.shape[1] == 4 and not ring[:, (t + 3) % 4].any()
        filled += int(ring[:, [(t + j) % 4 for j in range(3)]].any())
    assert filled > 50
