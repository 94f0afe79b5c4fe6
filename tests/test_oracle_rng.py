"""Oracle pins: the counter-based generator and the Poisson drive.

Philox4x32-10 is pinned to the published known-answer vectors; the Poisson table and sampler
are pinned to scipy's Poisson distribution (an independent implementation of the pmf/cdf)."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    assert list(o.philox4x32_10(ctr, key)) == expect


def test_philox_counter_sensitivity():
    # every counter and key word changes the output (no word silently dropped)
    base = o.philox4x32_10([1, 2, 3, 4], [5, 6])
    for pos in range(4):
        c = [1, 2, 3, 4]
        c[pos] ^= 1
        assert not np.array_equal(o.philox4x32_10(c, [5, 6]), base)
    for pos in range(2):
        k = [5, 6]
        k[pos] ^= 1
        assert not np.array_equal(o.philox4x32_10([1, 2, 3, 4], k), base)


@pytest.mark.parametrize("lam", [0.5, 1.0, 1.2, 1.5, 2.0])
def test_poisson_table_matches_cdf(lam):
    thr = o.poisson_table(lam)
    k = np.arange(len(thr))
    cdf = stats.poisson.cdf(k, lam)
    want = np.minimum(np.floor(cdf * 2.0**32), 2.0**32 - 1)
    # tables agree with scipy's cdf to the table resolution (one unit in 2^32)
    assert np.all(np.abs(thr[:-1].astype(np.float64) - want[:-1]) <= 1.0)
    assert thr[-1] == 0xFFFFFFFF
    # the last entry is where the tail mass drops below one unit in 2^32
    assert stats.poisson.sf(len(thr) - 2, lam) * 2.0**32 >= 0.5
    assert np.all(np.diff(thr.astype(np.int64)) >= 0)


@pytest.mark.parametrize("lam", [1.2, 1.5])
def test_poisson_sampler_masses(lam):
    thr = o.poisson_table(lam)
    # the sampler returns k exactly on [thr[k-1], thr[k]) -- check both edges of every bin
    for k in range(len(thr) - 1):
        lo = 0 if k == 0 else int(thr[k - 1])
        if int(thr[k]) > lo:
            assert o.poisson_sample(lo, thr) == k
            assert o.poisson_sample(int(thr[k]) - 1, thr) == k
    assert o.poisson_sample(0xFFFFFFFF, thr) == len(thr) - 1
    # probability mass of each k equals the pmf to 2^-32
    edges = np.concatenate([[0], thr.astype(np.float64)])
    mass = np.diff(edges) / 2.0**32
    pmf = stats.poisson.pmf(np.arange(len(thr)), lam)
    assert np.allclose(mass[:-1], pmf[:-1], atol=2.0**-31)


def test_poisson_drive_empirical_moments():
    lam = 1.5
    thr = o.poisson_table(lam)
    ks = np.array([o.poisson_sample(o.poisson_word(99, i, t), thr) for i in range(50) for t in range(2000)])
    n = len(ks)
    assert abs(ks.mean() - lam) < 5 * np.sqrt(lam / n)
    assert abs(ks.var() - lam) < 0.05 * lam
    # counts against the pmf: chi-square over k = 0..6
    obs = np.array([np.sum(ks == k) for k in range(7)] + [np.sum(ks >= 7)])
    p = np.concatenate([stats.poisson.pmf(np.arange(7), lam), [stats.poisson.sf(6, lam)]])
    chi = stats.chisquare(obs, p * n)
    assert chi.pvalue > 1e-4


def test_bf16_rounding():
    # round-to-nearest-even against numpy's float32 bit layout
    assert o.round_bf16(87.8) == 88.0
    assert o.round_bf16(-439.0) == -440.0
    assert o.round_bf16(1.0) == 1.0
    # tie: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> even (1.0)
    assert o.round_bf16(1.0 + 2.0**-8) == 1.0
    assert o.round_bf16(1.0 + 3 * 2.0**-8) == 1.0 + 2.0**-6
    rng = np.random.default_rng(0)
    for x in rng.normal(0, 100, 200).astype(np.float32):
        y = o.round_bf16(float(x))
        b = np.array([y], np.float32).view(np.uint32)[0]
        assert b & 0xFFFF == 0
        assert abs(y - float(x)) <= abs(float(x)) * 2.0**-8


def test_poisson_word_layout_and_independence_of_the_four_words():
    """Neuron i at step t draws word i mod 4 of Philox(counter = (i / 4, t, 3, 0)); the four
    neurons that share one generator call get uncorrelated drives."""
    seed = 31
    for i, t in [(0, 0), (5, 7), (4099, 12345), (2 ** 20 - 1, 99)]:
        words = o.philox4x32_10([i // 4, t, 3, 0], [seed & 0xffffffff, seed >> 32])
        assert o.poisson_word(seed, i, t) == int(words[i % 4])
    thr = o.poisson_table(1.5)
    ks = np.array([[o.poisson_sample(o.poisson_word(seed, 4 * g + w, t), thr) for w in range(4)]
                   for g in range(8) for t in range(600)], dtype=np.float64)
    c = np.corrcoef(ks.T)
    assert np.all(np.abs(c[np.triu_indices(4, 1)]) < 0.05)
