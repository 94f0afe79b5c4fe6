"""Pins of the oracle's initial membrane potentials (the paper leaves V(0) open; the reading: V0
uniform on [V_reset, V_th) from the top 24 bits of one Philox word per neuron, one FP32 multiply
and one add).

Checked against the mathematics, not against the formula: with a span V_th - V_reset = 16 mV (a
power of two) every V0 - V_reset must be an exact multiple of 16 * 2^-24 = 2^-20 below 16, and the
values must be uniform on [V_reset, V_th) (Kolmogorov-Smirnov) and uncorrelated between
neighbours.  A wrong shift of the word (range halved or doubled), a missing offset or a wrong scale
fails one of these."""
import numpy as np
from scipy import stats

from helpers import oracle_params
from oracle import oracle as orc
from paper_2406_03762_gb300 import workloads as W


def _v0(spec, seed):
    return orc.Network(oracle_params(spec), seed).state()[0]


def test_v0_on_the_grid_and_uniform():
    spec = W.NetSpec(40000, 10000, 1, 1, v_th=8.0, v_reset=-8.0)
    v = _v0(spec, 12345)
    assert v.min() >= -8.0 and v.max() < 8.0
    m = (v + 8.0) * 2.0**20
    assert np.all(m == np.floor(m)) and m.max() < 2**24
    ks = stats.kstest((v + 8.0) / 16.0, "uniform")
    assert ks.pvalue > 1e-3, ks
    assert abs(np.corrcoef(v[:-1], v[1:])[0, 1]) < 0.02
    # the full range is used: both ends of [V_reset, V_th) are reached within 1%
    assert v.min() < -8.0 + 0.16 and v.max() > 8.0 - 0.16


def test_v0_of_the_benchmark_networks_below_threshold():
    for name in ("c0", "c1"):
        cfg = W.CONFIGS[name]
        spec = W.scaled(cfg["spec"], 20000, 2)
        v = _v0(spec, cfg["seed"])
        assert v.min() >= spec.v_reset and v.max() < spec.v_th
        ks = stats.kstest((v - spec.v_reset) / (spec.v_th - spec.v_reset), "uniform")
        assert ks.pvalue > 1e-3


def test_v0_depends_on_the_seed_not_on_the_network_size():
    a = _v0(W.NetSpec(800, 200, 1, 1), 5)
    b = _v0(W.NetSpec(1600, 400, 1, 1), 5)
    c = _v0(W.NetSpec(800, 200, 1, 1), 6)
    assert np.array_equal(a, b[:1000])
    assert not np.array_equal(a, c)
