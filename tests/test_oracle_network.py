"""Oracle pins: fixed in-degree connectivity (Sec. IV-A, Eq. 4-5) and spike delivery (Sec. II-B).

Connectivity is pinned by exact in-degrees, ranges, uniformity tests and the transpose relation
between the per-target draws and the CSR by source.  Delivery is pinned on hand-built graphs whose
ring contents are worked out by hand, on FP32 non-associativity (which exposes the summation
order), and by the invariant that every emitted spike reaches each of its synapses exactly once
at its delay."""
import numpy as np
import pytest
from scipy import stats

from oracle import oracle as o


def _tiny(**kw):
    base = dict(n_exc=40, n_inh=10, k_exc=12, k_inh=3)
    base.update(kw)
    return o.Params(**base)


def test_indegree_exact_and_ranges():
    p = _tiny()
    net = o.Network(p, 11)
    row, tgt, dly = net.outgoing()
    n = p.n_exc + p.n_inh
    assert row[-1] == n * (p.k_exc + p.k_inh) == net.n_syn
    src = np.repeat(np.arange(n), np.diff(row))
    assert np.all((tgt >= 0) & (tgt < n))
    assert np.all((dly >= p.d_min) & (dly <= p.d_max))
    ind_e = np.bincount(tgt[src < p.n_exc], minlength=n)
    ind_i = np.bincount(tgt[src >= p.n_exc], minlength=n)
    assert np.all(ind_e == p.k_exc) and np.all(ind_i == p.k_inh)


def test_csr_is_transpose_of_draws_sorted_by_source_target_draw():
    p = _tiny()
    seed = 5
    net = o.Network(p, seed)
    row, tgt, dly = net.outgoing()
    n, k = p.n_exc + p.n_inh, p.k_exc + p.k_inh
    recs = []
    for i in range(n):
        s, d = o.incoming(seed, p, i)
        for j in range(k):
            recs.append((s[j], i, j, d[j]))
    recs.sort()                                   # (source, target, draw)
    want_tgt = np.array([r[1] for r in recs])
    want_dly = np.array([r[3] for r in recs])
    want_row = np.concatenate([[0], np.cumsum(np.bincount([r[0] for r in recs], minlength=n))])
    assert np.array_equal(row, want_row)
    assert np.array_equal(tgt, want_tgt)
    assert np.array_equal(dly, want_dly)


def test_sources_and_delays_uniform():
    p = o.Params(n_exc=400, n_inh=100, k_exc=400, k_inh=100, d_min=5, d_max=40)
    net = o.Network(p, 3)
    row, tgt, dly = net.outgoing()
    outdeg = np.diff(row)
    n = p.n_exc + p.n_inh
    # out-degree counts are uniform within each population (chi-square)
    for lo, hi, k in ((0, p.n_exc, p.k_exc), (p.n_exc, n, p.k_inh)):
        obs = outdeg[lo:hi]
        assert obs.sum() == n * k
        assert stats.chisquare(obs).pvalue > 1e-4
    counts = np.bincount(dly - p.d_min, minlength=p.d_max - p.d_min + 1)
    assert stats.chisquare(counts).pvalue > 1e-4
    assert abs(outdeg.mean() - (p.k_exc + p.k_inh)) < 1e-9


def test_draws_depend_on_seed_and_target():
    p = _tiny()
    a = o.incoming(1, p, 0)[0]
    assert not np.array_equal(a, o.incoming(2, p, 0)[0])
    assert not np.array_equal(a, o.incoming(1, p, 1)[0])


def _hand_net(edges, n=5, prec=o.FP32, d_max=8):
    p = o.Params(n_exc=n, n_inh=0, k_exc=0, k_inh=0, poisson_on=0, v_th=1e9, d_min=1, d_max=d_max,
                 precision=prec)
    src, tgt, dly, w = zip(*edges)
    net = o.Network(p, 1, edges=(src, tgt, dly, w), accounting=True)
    net.set_state(np.zeros(n), np.zeros(n), np.zeros(n, np.int32))
    return p, net


def test_hand_built_ring_contents():
    edges = [(0, 1, 2, 10.0), (0, 1, 2, 7.0), (0, 2, 5, -3.0), (1, 2, 1, 4.0), (3, 3, 3, 1.0),
             (0, 4, 8, 2.5)]
    p, net = _hand_net(edges)
    D = net.depth
    assert D == p.d_max + 1
    net.simulate(3, forced=([0, 1, 2], [0, 1, 3]))
    ring = net.ring()
    want = np.zeros((5, D))
    want[2, 5 % D] = -3.0            # 0 -> 2 sent at step 0, due at step 5
    want[3, 5 % D] = 1.0             # 3 -> 3 sent at step 2, due at step 5
    want[4, 8 % D] = 2.5             # 0 -> 4 sent at step 0, due at step 8
    # 0 -> 1 (17 at step 2) and 1 -> 2 (4 at step 2) were consumed during step 2
    assert np.array_equal(ring, want)
    _, cur, _ = net.state()
    assert cur[1] == np.float32(17.0) and cur[2] == np.float32(4.0)
    ev, wsum = net.accounting()
    assert list(ev) == [0, 2, 1, 0, 0]


def test_summation_order_is_emission_then_source_then_draw():
    """FP32 addition is not associative: 1e8 + 1 rounds back to 1e8.  Three spikes reach the
    same ring cell; the result shows which order the oracle adds them in."""
    big = 1.0e8
    # sources 0, 1, 2 spike at the same step into target 4 with the same delay
    edges = [(0, 4, 2, big), (1, 4, 2, 1.0), (2, 4, 2, -big)]
    p, net = _hand_net(edges)
    net.simulate(1, forced=([0, 0, 0], [2, 0, 1]))
    assert net.ring()[4, 2] == 0.0   # ((0 + 1e8) + 1) - 1e8 = 0 in float; other orders give 1
    # emission order comes before source order: source 2 sends at step 0 (delay 3), sources 0
    # and 1 at step 1 (delay 2); all due at step 3.  Emission first: ((1 + 1e8) - 1e8) = 0;
    # source order alone would give ((1e8 - 1e8) + 1) = 1.
    edges = [(0, 4, 2, big), (2, 4, 3, 1.0), (1, 4, 2, -big)]
    p, net = _hand_net(edges)
    net.simulate(2, forced=([0, 1, 1], [2, 0, 1]))
    assert net.ring()[4, 3] == 0.0
    # within one source, draw order: multapse onto the same cell
    edges = [(0, 4, 2, big), (0, 4, 2, 1.0), (0, 4, 2, -big)]
    p, net = _hand_net(edges)
    net.simulate(1, forced=([0], [0]))
    assert net.ring()[4, 2] == 0.0


def test_fp64_ring_has_no_rounding_in_the_same_case():
    edges = [(0, 4, 2, 1.0e8), (1, 4, 2, 1.0), (2, 4, 2, -1.0e8)]
    p, net = _hand_net(edges, prec=o.FP64)
    net.simulate(1, forced=([0, 0, 0], [2, 0, 1]))
    assert net.ring()[4, 2] == 1.0


@pytest.mark.parametrize("prec", [o.FP32, o.FP64])
def test_every_spike_reaches_each_synapse_once_at_its_delay(prec):
    p = o.Params(n_exc=160, n_inh=40, k_exc=40, k_inh=10, precision=prec)
    net = o.Network(p, 21, accounting=True)
    T = 600
    net.simulate(T)
    steps, ids = net.raster()
    assert len(steps) > 100
    row, tgt, dly = net.outgoing()
    n = p.n_exc + p.n_inh
    want_ev = np.zeros(n, np.int64)
    want_w = np.zeros(n)
    spikes_of = [[] for _ in range(n)]
    for s, i in zip(steps, ids):
        spikes_of[i].append(s)
    for src in range(n):
        ts = np.array(spikes_of[src], np.int64)
        if len(ts) == 0:
            continue
        w = p.j_exc if src < p.n_exc else p.j_inh
        for q in range(row[src], row[src + 1]):
            # consumed at step t + d if that step has run (t + d < T)
            c = int(np.sum(ts + dly[q] < T))
            want_ev[tgt[q]] += c
            want_w[tgt[q]] += c * w
    ev, wsum = net.accounting()
    assert np.array_equal(ev, want_ev)
    assert np.allclose(wsum, want_w, rtol=1e-12, atol=1e-6)
    assert net.events == int(sum(np.diff(row)[i] for i in ids))


def test_simulate_in_chunks_equals_one_run():
    p = o.Params(n_exc=160, n_inh=40, k_exc=40, k_inh=10)
    a = o.Network(p, 8)
    a.simulate(300)
    b = o.Network(p, 8)
    b.simulate(120)
    b.simulate(180)
    for x, y in zip(a.raster(), b.raster()):
        assert np.array_equal(x, y)
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)
    assert np.array_equal(a.ring(), b.ring())


def _brunel_small(**kw):
    base = dict(n_exc=800, n_inh=200, k_exc=80, k_inh=20)
    base.update(kw)
    return o.Params(**base)


@pytest.mark.parametrize("prec,dmin,dmax", [(o.FP32, 1, 16), (o.FP64, 1, 16), (o.FP32, 5, 40)])
def test_replay_of_targets_reproduces_the_full_simulation(prec, dmin, dmax):
    """A neuron's trajectory is fixed by its incoming synapses and the raster (Eq. 1-3), so
    replaying chosen targets against the full run's raster gives their spikes and final state."""
    p = _brunel_small(precision=prec, d_min=dmin, d_max=dmax)
    seed, steps = 77, 600
    net = o.Network(p, seed)
    net.simulate(steps)
    rs, ri = net.raster()
    assert len(rs) > 500
    v, c, r = net.state()
    rng = np.random.default_rng(3)
    tg = np.unique(np.concatenate([[0, 799, 800, 999], rng.integers(0, 1000, 40)]))
    ps, pi, (pv, pc, pr) = o.replay(p, seed, tg, steps, rs, ri)
    keep = np.isin(ri, tg)
    assert np.array_equal(ps, rs[keep]) and np.array_equal(pi, ri[keep])
    assert np.array_equal(pv, v[tg]) and np.array_equal(pc, c[tg]) and np.array_equal(pr, r[tg])


def test_replay_detects_a_missing_presynaptic_spike():
    """Dropping one raster spike of a source that projects onto a target changes that target's
    replayed state: the replay really consumes the raster."""
    p = _brunel_small()
    seed, steps = 78, 300
    net = o.Network(p, seed)
    net.simulate(steps)
    rs, ri = net.raster()
    target = 5
    src, dly = o.incoming(seed, p, target)
    hit = np.nonzero(np.isin(ri, src) & (rs + dly.max() < steps - 1))[0]
    assert len(hit) > 0
    drop = hit[len(hit) // 2]
    _, _, (v0, c0, _) = o.replay(p, seed, [target], steps, rs, ri)
    _, _, (v1, c1, _) = o.replay(p, seed, [target], steps, np.delete(rs, drop), np.delete(ri, drop))
    assert (v0[0], c0[0]) != (v1[0], c1[0])
