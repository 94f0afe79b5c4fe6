"""GPU path at the benchmark's full sizes, and the precision paths against the FP64 oracle.

A neuron's trajectory is fixed by its own incoming synapses and the spikes their sources emitted
(Eq. 1-3), so the oracle's replay of a few targets, driven by the GPU's raster of the whole
network, checks a network far too large for the full oracle one neuron at a time: each sampled
target's spikes and final (V, I, refractory count) must equal the GPU's bit for bit.  The
launch configuration is the one the benchmark times (persistent kernel, 1000 steps per launch,
default warps per block).

Precision (FP32 state and accumulation): potentials within 1e-6 of the FP64 oracle, relative to
max(|V64|, V_th), with the FP64 oracle driven by the GPU's own raster; population rates within 1%
(or the 3-sigma band of the rate fluctuations) of the free-running FP64 oracle.  BF16 weights: rates against the FP64 oracle on the
10,000-neuron network with the statistics of the 1e6-neuron configuration (K = 11,250)."""
import numpy as np
import pytest

from helpers import first_mismatch, fp64_replay_check, oracle_params, oracle_run
from oracle import oracle as orc
from paper_2406_03762_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BENCH_OPTS = dict(steps_per_launch=1000)


def _targets(spec, n_sample, seed, edges=()):
    rng = np.random.default_rng(seed)
    fixed = [0, spec.n_exc - 1, spec.n_exc, spec.n - 1]
    return np.unique(np.concatenate([fixed, np.asarray(edges, np.int64),
                                     rng.integers(0, spec.n, n_sample)])).astype(np.int32)


def layout_edges(cortex, specs, opts):
    """First and last target of every block and of every warp sub-range of each network, in the
    plan the build makes (cortex_plan on this GPU): where the block and warp offsets, the 16-bit
    piece offsets and the 12-bit warp ends of the layout change."""
    import torch
    props = torch.cuda.get_device_properties(0)
    smem = getattr(props, "shared_memory_per_block_optin", 232448)
    tb, _ = cortex.plan(specs, opts, n_sm=props.multi_processor_count, smem_per_block=smem)
    n_warps = min(opts.warps_per_block or 14, 16)
    out = []
    for spec, t in zip(specs, tb):
        t = int(t)
        tw = -(-t // n_warps)
        e = []
        for b0 in range(0, spec.n, t):
            nt = min(t, spec.n - b0)
            e += [b0, b0 + nt - 1]
            for w0 in range(0, nt, tw):
                e += [b0 + w0, b0 + min(w0 + tw, nt) - 1]
        out.append(np.unique(np.asarray(e, np.int64)))
    return out


def _replay_check(net, spec, seed, steps, net_idx=0, n_sample=40, sample_seed=0, edges=()):
    gs, gi = net.spikes(net_idx)
    gv, gc, gr = net.state(net_idx)
    tg = _targets(spec, n_sample, sample_seed, edges)
    ps, pi, (pv, pc, pr) = orc.replay(oracle_params(spec), seed, tg, steps, gs, gi)
    keep = np.isin(gi, tg)
    assert np.array_equal(ps, gs[keep]) and np.array_equal(pi, gi[keep]), "spikes of a sampled target differ"
    assert np.array_equal(pv, gv[tg].astype(np.float64)), "V of a sampled target differs"
    assert np.array_equal(pc, gc[tg].astype(np.float64)), "I of a sampled target differs"
    assert np.array_equal(pr, gr[tg]), "refractory count of a sampled target differs"
    return len(gs), int(keep.sum())


@pytest.mark.parametrize("name,steps,delivery", [("c1", 1000, 0), ("c2", 1000, 0), ("c3", 500, 0),
                                                 ("c2", 1000, 1), ("c3", 500, 1)])
def test_full_size_sampled_targets_bit_exact(cortex, name, steps, delivery):
    """Sampled targets, including the first and last of every block and warp sub-range (4,000+
    targets at 152 blocks x 14 warps), replayed by the oracle from the GPU's raster."""
    cfg = W.CONFIGS[name]
    spec, seed = cfg["spec"], cfg["seed"]
    opts = cortex.make_options(delivery=delivery, **BENCH_OPTS)
    edges = layout_edges(cortex, [spec], opts)[0]
    with cortex.Network(spec, seed, opts) as net:
        st = net.stats()
        assert st["n_synapses"] == spec.n * spec.k
        net.simulate(steps)
        n_spikes, n_sampled = _replay_check(net, spec, seed, steps, edges=edges)
    assert n_spikes > steps, "the network should be active"
    assert len(edges) > 2 * st["n_blocks"]


@pytest.mark.slow
@pytest.mark.parametrize("name,steps,delivery", [("c1", 500, 0), ("c2", 300, 0), ("c2", 300, 1)])
def test_whole_raster_bit_exact_against_the_full_oracle(cortex, name, steps, delivery):
    """The whole raster, final state and event count of the 112,500-neuron network (500 steps) and of
    the 500,000-neuron deep-delay network (2.5e9 synapses, 300 steps = five 6-step windows per 30
    steps) against the full FP32 oracle, run target-partitioned on all host cores (bitwise equal to
    the single-threaded oracle)."""
    import os
    cfg = W.CONFIGS[name]
    spec, seed = cfg["spec"], cfg["seed"]
    with cortex.Network(spec, seed, cortex.make_options(delivery=delivery, **BENCH_OPTS)) as net:
        net.simulate(steps)
        gs, gi = net.spikes()
        gv, gc, gr = net.state()
        st = net.stats()
    ref = orc.Network(oracle_params(spec), seed, threads=max(1, os.cpu_count() or 1))
    ref.simulate(steps)
    os_, oi = ref.raster()
    assert len(os_) > 1000
    assert first_mismatch(gs, gi, os_, oi) == -1
    ov, oc, orr = ref.state()
    assert np.array_equal(gv.astype(np.float64), ov) and np.array_equal(gc.astype(np.float64), oc)
    assert np.array_equal(gr, orr)
    assert st["events"] == ref.events


def test_batch_64_networks_sampled_targets_bit_exact(cortex):
    """The 64 uneven networks stepped together for 500 ms in the plan the autotuner picks (the one
    the benchmark times); the first and last target of every block and warp sub-range of every
    instance, and random ones."""
    specs, seeds = W.batch_specs()
    steps = W.CONFIGS["c4"]["steps"]
    best, _, _ = cortex.autotune(specs, seeds, cortex.make_options(**BENCH_OPTS), trial_steps=500)
    edges = layout_edges(cortex, specs, best)
    with cortex.Network(specs, seeds, best) as net:
        assert net.stats()["n_nets"] == 64
        net.simulate(steps)
        for b, (spec, seed) in enumerate(zip(specs, seeds)):
            _replay_check(net, spec, seed, steps, net_idx=b, n_sample=2, sample_seed=b, edges=edges[b])


def _rate_check(spec, s_a, i_a, s_b, i_b, t0, t1, block=250):
    """Relative error of each population's mean rate over [t0, t1) and the 3-sigma band from
    block-to-block fluctuations (blocks of `block` steps) of both runs."""
    out = []
    for lo, hi in ((0, spec.n_exc), (spec.n_exc, spec.n)):
        edges = np.arange(t0, t1 + 1, block)
        def per_block(s, i):
            m = (i >= lo) & (i < hi)
            return np.histogram(s[m], bins=edges)[0].astype(np.float64)
        a, b = per_block(s_a, i_a), per_block(s_b, i_b)
        mean_b = b.mean()
        rel = (a.mean() - mean_b) / mean_b
        sig = np.sqrt(a.var(ddof=1) / len(a) + b.var(ddof=1) / len(b)) / mean_b
        out.append((rel, sig))
    return out


def test_fp32_potentials_and_rates_against_fp64_oracle(cortex):
    """N = 2,500, FP32 on the GPU against the FP64 oracle.
    Potentials: every neuron after every step of the first 100 ms within 1e-6 of the FP64 oracle
    replaying that neuron with the GPU's raster as presynaptic input, relative to max(|V64|, V_th),
    up to the neuron's own first spike-time difference.
    Rates: the free-running FP64 oracle over 200 ms, after its raster first departs from the GPU's."""
    cfg = W.CONFIGS["c0"]
    spec, seed, steps = cfg["spec"], cfg["seed"], cfg["steps"]
    n_v = 1000
    gv = np.zeros((n_v, spec.n), np.float64)
    with cortex.Network(spec, seed) as net:
        for t in range(n_v):
            net.simulate(1)
            gv[t] = net.state()[0]
        net.simulate(steps - n_v)
        gs, gi = net.spikes()
    err, agree = fp64_replay_check(spec, seed, n_v, gs, gi, gv)
    assert agree >= 0.99, f"only {agree:.4f} of the neurons keep their spike times"
    assert err <= 1e-6, f"max relative V error {err:.3g}"
    _, os_, oi, _ = oracle_run(spec, seed, steps, precision=orc.FP64)
    fm = first_mismatch(gs, gi, os_, oi)
    t_star = int(min(gs[fm], os_[fm])) if 0 <= fm < min(len(gs), len(os_)) else steps
    if t_star < steps - 500:
        for rel, sig in _rate_check(spec, gs, gi, os_, oi, t_star, steps):
            assert abs(rel) <= max(0.01, 3 * sig)


def test_bf16_rates_against_fp64_oracle_on_10k_network(cortex):
    """BF16 weights (J_E 87.8 -> 88, J_I -439 -> -440, +0.23%), FP32 accumulation and state, on
    N = 10,000 with K = 11,250 (the statistics of the 1e6-neuron configuration), against the FP64
    oracle with the exact weights:
    - rates: each population's rate over 500 ms within 2%, or within the 3-sigma band of the rate
      fluctuations;
    - raster error: the first step at which the rasters differ, and per-neuron spike counts (their
      correlation across neurons and the mean absolute difference), printed and bounded loosely;
    - the 1e6-neuron BF16 network's rates against these 10k FP64 rates (the same in-degree, so the
      same mean input; finite-size differences allowed up to 5%)."""
    spec = W.NetSpec(8000, 2000, 9000, 2250, weight_dtype=W.BF16)
    seed, steps = W.CONFIGS["c3"]["seed"], 5000
    with cortex.Network(spec, seed) as net:
        net.simulate(steps)
        gs, gi = net.spikes()
    _, os_, oi, _ = oracle_run(spec, seed, steps, precision=orc.FP64)
    n = min(len(gs), len(os_))
    assert n > 10000
    for rel, sig in _rate_check(spec, gs, gi, os_, oi, 0, steps):
        assert abs(rel) <= max(0.02, 3 * sig), f"rate error {rel:.4f} (3 sigma {3 * sig:.4f})"
    fm = first_mismatch(gs, gi, os_, oi)
    first_step = int(min(gs[fm], os_[fm])) if 0 <= fm < n else steps
    cg = np.bincount(gi, minlength=spec.n).astype(np.float64)
    co = np.bincount(oi, minlength=spec.n).astype(np.float64)
    corr = float(np.corrcoef(cg, co)[0, 1])
    mad = float(np.mean(np.abs(cg - co)))
    # two independent Poisson counts of the same means differ by about E|X - Y|; sampled here
    pois = np.random.default_rng(0)
    indep = float(np.mean(np.abs(pois.poisson(co) - pois.poisson(co))))
    print(f"BF16 vs FP64 (10k): first raster difference at step {first_step}; per-neuron spike counts over "
          f"{steps} steps: correlation {corr:.3f}, mean |difference| {mad:.2f} spikes (mean count {co.mean():.1f}; "
          f"independent Poisson counts of the same means: {indep:.2f})")
    # the +0.23% weights change the raster within milliseconds (a chaotic network): afterwards it is
    # another realisation with the same statistics, no farther from the FP64 one than an
    # independent realisation would be
    assert first_step < steps
    assert corr > -0.05 and mad <= 1.1 * indep
    big = W.CONFIGS["c3"]
    with cortex.Network(big["spec"], big["seed"]) as net:
        net.simulate(steps)
        bs, bi = net.spikes()
    for lo, hi, lo_s, hi_s in ((0, big["spec"].n_exc, 0, spec.n_exc), (big["spec"].n_exc, big["spec"].n, spec.n_exc, spec.n)):
        r_big = np.count_nonzero((bi >= lo) & (bi < hi) & (bs >= 1000)) / ((hi - lo) * (steps - 1000) * 1e-4)
        r_10k = np.count_nonzero((oi >= lo_s) & (oi < hi_s) & (os_ >= 1000)) / ((hi_s - lo_s) * (steps - 1000) * 1e-4)
        print(f"population [{lo}, {hi}): 1e6-neuron BF16 {r_big:.3f} Hz, 10k FP64 {r_10k:.3f} Hz")
        assert abs(r_big - r_10k) <= 0.05 * r_10k


@pytest.mark.slow
def test_c2_fp32_against_fp64_potentials_and_rates(cortex):
    """The headline network (500,000 neurons, K = 5,000, delays 5..40) in FP32 on the GPU against the
    FP64 oracle (readings 15-16):
    - potentials: 256 targets (the ends of every 19th block and random ones), after every step of the
      first 100 ms, within 1e-6 of the FP64 oracle replaying them with the GPU's raster as
      presynaptic input, relative to max(|V64|, V_th), up to each target's own first spike-time
      difference; at least 99% of the targets keep all their spike times;
    - rates: each population's rate over 100 ms .. 1 s within 1% (or the 3-sigma band) of the
      free-running FP64 oracle, run target-partitioned on all host cores."""
    import os
    cfg = W.CONFIGS["c2"]
    spec, seed, n_v, steps = cfg["spec"], cfg["seed"], 1000, 10000
    rng = np.random.default_rng(5)
    tb = -(-spec.n // 152)
    tg = np.unique(np.concatenate([np.arange(0, spec.n, 19 * tb), np.arange(tb - 1, spec.n, 19 * tb),
                                   rng.integers(0, spec.n, 220)]))[:256].astype(np.int32)
    gv = np.zeros((n_v, len(tg)), np.float64)
    with cortex.Network(spec, seed, cortex.make_options(**BENCH_OPTS)) as net:
        for t in range(n_v):
            net.simulate(1)
            gv[t] = net.state()[0][tg]
        net.simulate(steps - n_v)
        gs, gi = net.spikes()
    ps, pi, _, v64 = orc.replay(oracle_params(spec, orc.FP64, bf16=0), seed, tg, n_v, gs, gi, trace=True)
    first = np.full(len(tg), n_v)
    keep = gs < n_v
    for q, i in enumerate(tg):
        a, b = gs[keep][gi[keep] == i], ps[pi == i]
        m = min(len(a), len(b))
        d = np.nonzero(a[:m] != b[:m])[0]
        if len(d):
            first[q] = min(a[d[0]], b[d[0]])
        elif len(a) != len(b):
            first[q] = (a if len(a) > len(b) else b)[m]
    ok = np.arange(n_v)[:, None] < first[None, :]
    err = np.abs(gv - v64) / np.maximum(np.abs(v64), spec.v_th)
    print(f"c2 potentials: max relative error {err[ok].max():.3g}, targets keeping their spike times "
          f"{np.mean(first >= n_v):.3f}")
    assert err[ok].max() <= 1e-6
    assert np.mean(first >= n_v) >= 0.99
    ref = orc.Network(oracle_params(spec, orc.FP64, bf16=0), seed, threads=max(1, os.cpu_count() or 1))
    ref.simulate(steps)
    os_, oi = ref.raster()
    for rel, sig in _rate_check(spec, gs, gi, os_, oi, n_v, steps):
        print(f"c2 rate error {rel:+.4f} (3 sigma {3 * sig:.4f})")
        assert abs(rel) <= max(0.01, 3 * sig)


def test_barrier_wait_times_out_with_an_error_status(cortex):
    """One block never publishes its spikes (test hook), so every block's bounded wait at the
    window barrier runs out: cortex_simulate returns CORTEX_ERR_TIMEOUT, further calls on the
    handle return it at once, and the CUDA context stays usable for a new network."""
    cfg = W.CONFIGS["c0"]
    spec, seed = cfg["spec"], cfg["seed"]
    opts = cortex.make_options(test_withhold_block=1, barrier_timeout_ms=100.0, use_graph=-1)
    with cortex.Network(spec, seed, opts) as net:
        assert net.simulate_status(20) == -4
        assert net.simulate_status(20) == -4
    with cortex.Network(spec, seed) as net:
        net.simulate(300)
        gs, gi = net.spikes()
    _, os_, oi, _ = oracle_run(spec, seed, 300)
    assert first_mismatch(gs, gi, os_, oi) == -1
