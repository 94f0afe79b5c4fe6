"""Delay-ordered delivery (Sec. III-B "Varied Synaptic Delays", Sec. III-C spike buffer) against
the oracle, through the C ABI.

The records of every source are sorted by (delay, block, target, draw) and the synapses of delay d
of a spike emitted at step e are read at step e + d into that step's accumulator.  Each accumulator
cell then receives its weights in the order (emission step, source id, draw index) -- the oracle's
order -- so rasters, final states and event counts equal the FP32 oracle bit for bit, with the
ordered fold (FP32 weights) and with the order-free fold (BF16 weights, every partial sum exact)."""
import numpy as np
import pytest

from helpers import first_mismatch, oracle_run
from paper_2406_03762_gb300 import workloads as W

pytestmark = pytest.mark.gpu

C0 = W.CONFIGS["c0"]
DEEP = W.NetSpec(4000, 1000, 400, 100, d_min=5, d_max=40, nu_ext_hz=12000.0)
BF16 = W.NetSpec(800, 200, 900, 225, weight_dtype=W.BF16)


def _run(cortex, spec, seed, steps, **opts):
    with cortex.Network(spec, seed, cortex.make_options(delivery=1, **opts)) as net:
        net.simulate(steps)
        gs, gi = net.spikes()
        st = net.stats()
        state = net.state()
    return gs, gi, st, state


def _check(spec, seed, steps, gs, gi, st, state, min_spikes=100):
    ref, os_, oi, _ = oracle_run(spec, seed, steps)
    assert len(os_) > min_spikes
    fm = first_mismatch(gs, gi, os_, oi)
    assert fm == -1, f"first mismatch at spike {fm} of {len(os_)}"
    ov, oc, orr = ref.state()
    gv, gc, gr = state
    assert np.array_equal(gv.astype(np.float64), ov) and np.array_equal(gc.astype(np.float64), oc)
    assert np.array_equal(gr, orr)
    assert st["events"] == ref.events
    assert st["delivery"] == 1


@pytest.mark.parametrize("opts", [dict(), dict(warps_per_block=8), dict(warps_per_block=16, steps_per_launch=97),
                                  dict(use_graph=-1)])
def test_delay_c0_raster_bit_exact(cortex, opts):
    spec, seed, steps = C0["spec"], C0["seed"], C0["steps"]
    gs, gi, st, state = _run(cortex, spec, seed, steps, **opts)
    assert st["exact_fold"] == 0
    _check(spec, seed, steps, gs, gi, st, state)


def test_delay_deep_delays(cortex):
    """d = 5..40: six steps per window, 41 emission steps per delivery."""
    gs, gi, st, state = _run(cortex, DEEP, 2024, 1500)
    _check(DEEP, 2024, 1500, gs, gi, st, state, min_spikes=1000)


@pytest.mark.parametrize("fold", [0, 1])
def test_delay_bf16_exact_and_ordered_folds(cortex, fold):
    gs, gi, st, state = _run(cortex, BF16, 99, 1500, fold=fold)
    assert st["exact_fold"] == (1 if fold == 0 else 0)
    _check(BF16, 99, 1500, gs, gi, st, state)


def test_delay_batch_every_instance(cortex):
    specs, seeds = W.small_batch_specs()
    steps = 800
    with cortex.Network(specs, seeds, cortex.make_options(delivery=1)) as net:
        net.simulate(steps)
        res = [net.spikes(b) for b in range(len(specs))]
        st = net.stats()
    total = 0
    for b, (spec, seed) in enumerate(zip(specs, seeds)):
        ref, os_, oi, _ = oracle_run(spec, seed, steps)
        assert first_mismatch(*res[b], os_, oi) == -1, f"network {b}"
        total += ref.events
    assert st["events"] == total


def test_delay_in_pieces_equals_one_call_and_ring(cortex):
    spec, seed = C0["spec"], C0["seed"]
    with cortex.Network(spec, seed, cortex.make_options(delivery=1)) as a, \
            cortex.Network(spec, seed, cortex.make_options(delivery=1, steps_per_launch=50)) as b, \
            cortex.Network(spec, seed) as ring:
        a.simulate(700)
        ring.simulate(700)
        for n in (1, 2, 97, 300, 300):
            b.simulate(n)
        for x, y, z in zip(a.spikes(), b.spikes(), ring.spikes()):
            assert np.array_equal(x, y) and np.array_equal(x, z)
        for x, y, z in zip(a.state(), b.state(), ring.state()):
            assert np.array_equal(x, y) and np.array_equal(x, z)


def test_delay_refuses_ring_calls(cortex):
    spec, seed = C0["spec"], C0["seed"]
    with cortex.Network(spec, seed, cortex.make_options(delivery=1)) as net:
        for call in (lambda: net.ring(), lambda: net.set_step(5), lambda: net.deliver([1, 2], 0),
                     lambda: net.set_state(0, v=np.zeros(spec.n, np.float32))):
            with pytest.raises(cortex.CortexError) as e:
                call()
            assert e.value.code == cortex.ERR_UNSUPPORTED
    with pytest.raises(cortex.CortexError) as e:
        cortex.Network(spec, seed, cortex.make_options(delivery=1, mode=1))
    assert e.value.code == cortex.ERR_UNSUPPORTED


def test_delay_barrier_timeout(cortex):
    spec, seed = C0["spec"], C0["seed"]
    opts = cortex.make_options(delivery=1, test_withhold_block=1, barrier_timeout_ms=100.0, use_graph=-1)
    with cortex.Network(spec, seed, opts) as net:
        assert net.simulate_status(20) == -4
        assert net.simulate_status(20) == -4
    gs, gi, st, state = _run(cortex, spec, seed, 300)
    _check(spec, seed, 300, gs, gi, st, state)
