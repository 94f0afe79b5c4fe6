"""The target-partitioned oracle (Sec. III-B "Avoid Data Racing": each thread owns a range of
post-synaptic neurons and the synapses into them) equals the single-threaded oracle bit for bit:
raster, final state, ring and event count, for any number of parts.  It is the form timed on all
host cores for the CPU baseline."""
import numpy as np
import pytest

from helpers import oracle_params
from oracle import oracle as orc
from paper_2406_03762_gb300 import workloads as W

CASES = [
    (W.CONFIGS["c0"]["spec"], W.CONFIGS["c0"]["seed"], 600, orc.FP32),
    (W.NetSpec(1600, 400, 160, 40, d_min=5, d_max=40, nu_ext_hz=12000.0), 7, 500, orc.FP32),
    (W.NetSpec(800, 200, 900, 225, weight_dtype=W.BF16), 99, 400, orc.FP32),
    (W.CONFIGS["c0"]["spec"], 3, 300, orc.FP64),
]


@pytest.mark.parametrize("spec,seed,steps,prec", CASES)
def test_partitioned_oracle_is_bitwise_equal(spec, seed, steps, prec):
    p = oracle_params(spec, prec)
    ref = orc.Network(p, seed)
    ref.simulate(steps)
    rs, ri = ref.raster()
    assert len(rs) > 50
    for parts in (2, 3, 7):
        par = orc.Network(p, seed, threads=parts)
        par.simulate(steps // 2)
        par.set_threads(1)  # the same parts stepped by one thread
        par.simulate(steps - steps // 2)
        ps, pi = par.raster()
        assert np.array_equal(ps, rs) and np.array_equal(pi, ri), parts
        for x, y in zip(par.state(), ref.state()):
            assert np.array_equal(x, y)
        assert np.array_equal(par.ring(), ref.ring())
        assert par.events == ref.events and par.n_syn == ref.n_syn
