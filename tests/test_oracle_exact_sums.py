"""The arithmetic behind the order-free delivery fold, pinned on the CPU.

FP32 addition is not associative, so the summation order (emission step, source id, draw index)
fixes each ring cell's value.  When every weight is an integer multiple of 2^e and the sum of
|w| / 2^e over a target's in-degree stays at or below 2^24, every partial sum is a float and no add
rounds: any order then gives the same bits.  BF16 weights 88 = 11 * 2^3 and -440 = -55 * 2^3 with
K_E = 9,000, K_I = 2,250 (the 1e6-neuron configuration) give 222,750 <= 2^24; the FP32 weight
87.8f has 23 significant bits and sums of three weights already round."""
import numpy as np

from helpers import oracle_params
from oracle import oracle as orc
from paper_2406_03762_gb300 import workloads as W


def _fsum(seq):
    s = np.float32(0.0)
    for x in seq:
        s = np.float32(s + np.float32(x))
    return s


def test_bf16_weight_sums_are_order_free():
    we, wi = np.float32(orc.round_bf16(87.8)), np.float32(orc.round_bf16(-439.0))
    assert we == 88.0 and wi == -440.0
    rng = np.random.default_rng(11)
    for _ in range(300):
        a, b = int(rng.integers(0, 9000)), int(rng.integers(0, 2250))
        seq = np.array([we] * a + [wi] * b, np.float32)
        ref = _fsum(seq)
        assert float(ref) == 88.0 * a - 440.0 * b  # exact: no add rounded
        for _ in range(2):
            assert _fsum(rng.permutation(seq)) == ref


def test_fp32_weight_sums_depend_on_the_order():
    we, wi = np.float32(87.8), np.float32(-439.0)
    assert _fsum([we, we, wi]) != _fsum([wi, we, we])


def test_oracle_bf16_ring_cells_are_exact_sums():
    """Every ring cell of the oracle's BF16 network is an integer multiple of 8 and equals the
    double-precision sum of the same weights (the oracle's accounting shadow), i.e. no add
    rounded."""
    spec = W.NetSpec(800, 200, 900, 225, weight_dtype=W.BF16)
    p = oracle_params(spec)
    net = orc.Network(p, 99, accounting=True)
    net.simulate(400)
    ring = net.ring()
    assert np.count_nonzero(ring) > 0
    assert np.all(np.mod(ring, 8.0) == 0.0)
    events, weight = net.accounting()
    assert events.sum() > 0
