"""The block plan (domain decomposition, Sec. II-B, Eq. 9-10) on the host, through the C ABI's
cortex_plan: no GPU needed.  Properties every plan must have, and the plans of the benchmark
configurations."""
import numpy as np
import pytest

from paper_2406_03762_gb300 import cortex, workloads as W

SMS, SMEM = 152, 232448  # GB300: SMs, opt-in shared memory per block


def _blocks(specs, tb):
    return [-(-s.n // int(t)) for s, t in zip(specs, tb)]


def _check_plan(specs, tb, nb, n_sm=SMS, warps=14):
    assert nb == sum(_blocks(specs, tb)) and nb <= n_sm
    for s, t in zip(specs, tb):
        assert 1 <= t <= s.n
        assert t >= min(s.n, 32 * warps) or -(-s.n // t) > 1  # only a network's last block is short
        assert t <= 65535


def test_single_network_plans():
    """c1 and c3: equal blocks, one per SM."""
    for name, t in (("c1", 741), ("c3", 6580), ("c2", 3290)):
        spec = W.CONFIGS[name]["spec"]
        tb, nb = cortex.plan(spec)
        assert nb == -(-spec.n // int(tb[0])) <= SMS
        assert abs(int(tb[0]) - t) <= 1, (name, tb)


def test_batch_plans_fit_the_sms_and_balance_the_stated_cost():
    """64 uneven networks: every plan fits 152 SMs.  The work-balanced plan (balance 2) lowers
    the largest block cost (targets x cost per target) below the equal-target plan's, and gives
    a costlier network no larger blocks than a cheaper network of the same size would get."""
    specs, _ = W.batch_specs()
    rng = np.random.default_rng(3)
    rate = rng.uniform(10.0, 32.0, len(specs))  # Hz, the spread of the batch's measured rates
    cost = [float(r * 1e-4 * s.k + 0.5) for r, s in zip(rate, specs)]  # events per target and step + update
    loads = {}
    for bal in (0, 1, 2):
        kw = dict(balance=bal, net_work=cost) if bal == 2 else dict(balance=bal)
        tb, nb = cortex.plan(specs, cortex.make_options(**kw))
        _check_plan(specs, tb, nb)
        loads[bal] = max(int(t) * c for t, c in zip(tb, cost))
    assert loads[2] < loads[0]
    tb2, _ = cortex.plan(specs, cortex.make_options(balance=2, net_work=cost))
    for i in range(len(specs)):
        for j in range(len(specs)):
            if specs[i].n == specs[j].n and cost[i] > cost[j]:
                assert tb2[i] <= tb2[j]


def test_uneven_costs_cut_the_costly_network_into_more_blocks():
    """Six small networks, one twenty times costlier per target: the work-balanced plan cuts that
    one into blocks of the smallest size a block may have (32 targets per warp) and keeps every
    other block's cost at or below that block's."""
    specs, _ = W.small_batch_specs()
    cost = [20.0, 1.0, 0.5, 3.0, 1.0, 8.0]
    tb0, nb0 = cortex.plan(specs, cortex.make_options(warps_per_block=10))
    tb2, nb2 = cortex.plan(specs, cortex.make_options(warps_per_block=10, balance=2, net_work=cost))
    _check_plan(specs, tb0, nb0, warps=10)
    _check_plan(specs, tb2, nb2, warps=10)
    b2 = _blocks(specs, tb2)
    assert nb2 > len(specs) and b2[0] == -(-specs[0].n // 320)
    top = int(tb2[0]) * cost[0]
    assert all(int(t) * c <= top for t, c in zip(tb2, cost))
    assert top <= max(int(t) * c for t, c in zip(tb0, cost))


def test_less_shared_memory_never_gives_larger_blocks():
    specs, _ = W.batch_specs()
    for bal in (0, 2):
        kw = dict(balance=2, net_work=[1.0 + s.k / 1000 for s in specs]) if bal == 2 else {}
        big, _ = cortex.plan(specs, cortex.make_options(**kw))
        for smem in (180_000, 140_000):
            try:
                small, nb = cortex.plan(specs, cortex.make_options(**kw), smem_per_block=smem)
            except cortex.CortexError as e:
                assert e.code == -5
                continue
            _check_plan(specs, small, nb)
            assert all(int(s) <= int(b) for s, b in zip(small, big))


def test_targets_per_block_is_an_upper_bound():
    spec = W.CONFIGS["c1"]["spec"]
    tb, nb = cortex.plan(spec, cortex.make_options(targets_per_block=500))
    assert int(tb[0]) <= 500 and nb == -(-spec.n // int(tb[0]))


def test_no_plan_for_more_networks_than_sms():
    """200 networks need at least 200 blocks: refused at once with CORTEX_ERR_UNSUPPORTED."""
    specs = [W.brunel(2000, 200)] * 200
    with pytest.raises(cortex.CortexError) as e:
        cortex.plan(specs)
    assert e.value.code == -5 and "SMs" in str(e.value)


def test_plan_arguments():
    spec = W.CONFIGS["c0"]["spec"]
    for kw in (dict(n_sm=0), dict(smem_per_block=1024)):
        with pytest.raises(cortex.CortexError) as e:
            cortex.plan(spec, **kw)
        assert e.value.code == -1
