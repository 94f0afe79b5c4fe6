"""GPU path vs the oracle, through the C ABI.

Bit-exact: Philox words, FP32 propagators and Poisson thresholds, initial potentials, the
connectivity (multiset of (source, target, delay, weight)), and -- in FP32 with the summation
order (emission step, source, draw) on both sides -- the whole spike raster and final state."""
import numpy as np
import pytest

from helpers import first_mismatch, oracle_params, oracle_run
from oracle import oracle as orc
from paper_2406_03762_gb300 import workloads as W

pytestmark = pytest.mark.gpu

C0 = W.CONFIGS["c0"]


def _kat():
    import os
    rows = []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            w = [int(x, 16) for x in line.split()]
            rows.append(w)
    return np.array(rows, dtype=np.uint64).astype(np.uint32)


def test_philox_device_known_answers(cortex):
    k = _kat()
    out = cortex.philox(k[:, 0:4], k[:, 4:6])
    assert np.array_equal(out, k[:, 6:10])


def test_philox_device_matches_oracle(cortex):
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2**32, size=(500, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(500, 2), dtype=np.uint64).astype(np.uint32)
    out = cortex.philox(ctr, key)
    for q in range(0, 500, 7):
        assert np.array_equal(out[q], orc.philox4x32_10(ctr[q], key[q]))


SPECS = [C0["spec"], W.NetSpec(4000, 1000, 400, 100, d_min=5, d_max=40, nu_ext_hz=12000.0),
         W.NetSpec(800, 200, 900, 225, weight_dtype=W.BF16), W.brunel(3000, 300, nu_ext_hz=17321.5)]


@pytest.mark.parametrize("spec", SPECS)
def test_constants_bit_equal(cortex, spec):
    with cortex.Network(spec, 1) as net:
        c6, thr, nref = net.constants()
    ref = orc.Network(oracle_params(spec), 1)
    c8, othr, onref = ref.constants_f32()
    assert c6[0] == c8[0] and c6[1] == c8[1] and c6[2] == c8[2]          # P11, P21, P22 - 1
    assert c6[3] == c8[4] and c6[4] == c8[5] and c6[5] == c8[6]          # weights, J_ext
    assert np.array_equal(thr, othr) and nref == onref


def test_initial_state_bit_equal(cortex):
    spec, seed = C0["spec"], C0["seed"]
    with cortex.Network(spec, seed) as net:
        v, i, r = net.state()
    ov, oi, orr = orc.Network(oracle_params(spec), seed).state()
    assert np.array_equal(v.astype(np.float64), ov)
    assert np.all(i == 0) and np.all(r == 0)


def _oracle_incoming(spec, seed, t_begin, t_end):
    p = oracle_params(spec)
    ref = orc.Network(p, seed)
    row, tgt, dly = ref.outgoing()
    src = np.repeat(np.arange(len(row) - 1), np.diff(row)).astype(np.int64)
    keep = (tgt >= t_begin) & (tgt < t_end)
    rec = np.stack([tgt[keep], src[keep], dly[keep]], axis=1)
    order = np.lexsort((rec[:, 2], rec[:, 1], rec[:, 0]))
    return rec[order], ref


@pytest.mark.parametrize("spec,warps", [(C0["spec"], 8), (SPECS[1], 4), (SPECS[2], 14)])
def test_connectivity_bit_exact(cortex, spec, warps):
    seed = 77
    n = spec.n
    with cortex.Network(spec, seed, cortex.make_options(warps_per_block=warps)) as net:
        s, t, d, w = net.export_synapses(0, n)
        c6, _, _ = net.constants()
    want, _ = _oracle_incoming(spec, seed, 0, n)
    got = np.stack([t, s, d], axis=1).astype(np.int64)
    assert got.shape == want.shape
    assert np.array_equal(got, want)
    exp_w = np.where(s < spec.n_exc, c6[3], c6[4]).astype(np.float32)
    assert np.array_equal(w, exp_w)
    # in-degree exactly K_E / K_I for every target
    assert np.all(np.bincount(t[s < spec.n_exc], minlength=n) == spec.k_exc)
    assert np.all(np.bincount(t[s >= spec.n_exc], minlength=n) == spec.k_inh)


MODES = [
    dict(),                                            # persistent, automatic ring placement
    dict(ring=2),                                      # persistent, ring in global memory
    dict(mode=1),                                      # split update / delivery launches
    dict(warps_per_block=4, steps_per_launch=97),      # other warp split, odd launch chunks
    dict(warps_per_block=14, use_graph=-1),
    dict(warps_per_block=16, ring=2),                  # the widest block: 16 sub-range ends per header
    dict(helper_warp=1),                               # one more warp builds the descriptors
    dict(helper_warp=1, warps_per_block=13, ring=2),
    dict(helper_warp=1, mode=1, warps_per_block=6),
]


@pytest.mark.parametrize("opts", MODES)
def test_raster_c0_bit_exact(cortex, opts):
    spec, seed, steps = C0["spec"], C0["seed"], C0["steps"]
    with cortex.Network(spec, seed, cortex.make_options(**opts)) as net:
        net.simulate(steps)
        gs, gi = net.spikes()
        gv, gc, gr = net.state()
        st = net.stats()
    ref, os_, oi, _ = oracle_run(spec, seed, steps)
    assert first_mismatch(gs, gi, os_, oi) == -1, f"first mismatch at spike {first_mismatch(gs, gi, os_, oi)}"
    ov, oc, orr = ref.state()
    assert np.array_equal(gv.astype(np.float64), ov)
    assert np.array_equal(gc.astype(np.float64), oc)
    assert np.array_equal(gr, orr)
    assert st["events"] == ref.events
    assert st["spikes"] == len(os_)


def test_raster_deep_delays_window(cortex):
    """d = 5..40: six steps per barrier window (d_min + 1), ring depth 41."""
    spec, seed, steps = SPECS[1], 2024, 1500
    for opts in (dict(), dict(mode=1)):
        with cortex.Network(spec, seed, cortex.make_options(**opts)) as net:
            net.simulate(steps)
            gs, gi = net.spikes()
            gv, _, _ = net.state()
        ref, os_, oi, _ = oracle_run(spec, seed, steps)
        assert len(os_) > 1000
        assert first_mismatch(gs, gi, os_, oi) == -1
        assert np.array_equal(gv.astype(np.float64), ref.state()[0])


def test_simulate_in_pieces_equals_one_call(cortex):
    spec, seed = C0["spec"], C0["seed"]
    with cortex.Network(spec, seed) as a, cortex.Network(spec, seed, cortex.make_options(steps_per_launch=50)) as b:
        a.simulate(700)
        for n in (1, 2, 97, 300, 300):
            b.simulate(n)
        for x, y in zip(a.spikes(), b.spikes()):
            assert np.array_equal(x, y)
        for x, y in zip(a.state(), b.state()):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("opts", [dict(), dict(fold=1), dict(ring=2, l2_persist=1), dict(ring=2, fold=1, l2_persist=-1),
                                  dict(mode=1, ring=2)])
def test_bf16_weights_match_oracle_with_bf16_weights(cortex, opts):
    """BF16 storage with FP32 accumulation is deterministic: equal to the FP32 oracle run with the
    weights rounded to bfloat16 (J_E 87.8 -> 88, J_I -439 -> -440).  These weights are multiples of
    8 with K_E 88 + K_I 440 far below 2^24 * 8, so the build proves every partial sum exact and
    folds without ordering (unless fold=1 asks for the ordered fold); both give the oracle's bits."""
    spec, seed, steps = SPECS[2], 99, 1500
    with cortex.Network(spec, seed, cortex.make_options(**opts)) as net:
        net.simulate(steps)
        gs, gi = net.spikes()
        gv, gc, gr = net.state()
        c6, _, _ = net.constants()
        st = net.stats()
    assert c6[3] == 88.0 and c6[4] == -440.0
    assert st["exact_fold"] == (0 if opts.get("fold") == 1 else 1)
    if st["ring_in_smem"] == 0:
        assert (st["l2_persist_bytes"] > 0) == (opts.get("l2_persist", 0) > 0)
    ref, os_, oi, _ = oracle_run(spec, seed, steps)
    assert len(os_) > 100
    assert first_mismatch(gs, gi, os_, oi) == -1
    ov, oc, orr = ref.state()
    assert np.array_equal(gv.astype(np.float64), ov) and np.array_equal(gc.astype(np.float64), oc)
    assert np.array_equal(gr, orr)


def test_exact_fold_is_refused_when_sums_can_round(cortex):
    """FP32 weights 87.8 / -439 (87.8f has 23 significant bits): partial sums of a cell round, so
    the order-free fold is not proven and fold=2 is refused; the default keeps the ordered fold."""
    spec, seed = C0["spec"], C0["seed"]
    with pytest.raises(cortex.CortexError) as e:
        cortex.Network(spec, seed, cortex.make_options(fold=2))
    assert e.value.code == cortex.ERR_UNSUPPORTED
    with cortex.Network(spec, seed) as net:
        assert net.stats()["exact_fold"] == 0


@pytest.mark.parametrize("opts", [dict(), dict(ring=2)])
def test_restore_of_a_ring_off_the_weight_grid_keeps_results(cortex, opts):
    """A restored ring whose values are not sums of the network's weights (here 0.1 pA) cannot use
    the order-free fold: the handle returns to the ordered fold, whose shared-memory layout (with
    the duplicate-detection tags) it recomputes, and still equals the oracle started from the same
    state; with the ring in shared memory and in global memory."""
    spec, seed = SPECS[2], 99
    ref = orc.Network(oracle_params(spec), seed)
    ref.simulate(100)
    v, c, r = ref.state()
    ring = ref.ring().T.copy()
    ring[3, 7] += np.float32(0.1)
    ref.set_ring(ring.T)
    ref.simulate(300)
    s_all, i_all = ref.raster()
    keep = s_all >= 100
    with cortex.Network(spec, seed, cortex.make_options(**opts)) as net:
        assert net.stats()["exact_fold"] == 1
        net.set_state(0, v=v.astype(np.float32), i_syn=c.astype(np.float32), refr=r, ring=ring.astype(np.float32))
        st = net.stats()
        assert st["exact_fold"] == 0
        if opts.get("ring") == 2:
            assert st["ring_in_smem"] == 0
        net.set_step(100)
        net.simulate(300)
        gs, gi = net.spikes()
    assert first_mismatch(gs, gi, s_all[keep], i_all[keep]) == -1


def test_batch_every_instance_matches_oracle(cortex):
    specs, seeds = W.small_batch_specs()
    steps = 800
    with cortex.Network(specs, seeds) as net:
        net.simulate(steps)
        res = [net.spikes(b) for b in range(len(specs))]
        st = net.stats()
    assert st["n_nets"] == len(specs)
    total = 0
    for b, (spec, seed) in enumerate(zip(specs, seeds)):
        ref, os_, oi, _ = oracle_run(spec, seed, steps)
        gs, gi = res[b]
        assert first_mismatch(gs, gi, os_, oi) == -1, f"network {b}"
        total += ref.events
    assert st["events"] == total


def test_deliver_counts_out_degree(cortex):
    spec, seed = W.NetSpec(8000, 2000, 800, 200), 5
    rng = np.random.default_rng(1)
    ids = np.unique(rng.integers(0, spec.n, 300))
    with cortex.Network(spec, seed) as net:
        src, tgt, dly, w = net.export_synapses(0, spec.n)
        ms, ev = net.deliver(ids, t_emit=0, reps=1)
    outdeg = np.bincount(src, minlength=spec.n)
    assert ev == int(outdeg[ids].sum())
    assert ms > 0


def test_autotune_plan_does_not_change_results(cortex):
    """The autotuner times candidate plans (warps per block x block balance, including plans
    balanced by the measured work of each network).  Every plan gives the same rasters, because
    the summation order does not depend on the partition, and the oracle's.  A work-balanced plan
    with uneven costs cuts the costly networks into several blocks."""
    specs, seeds = W.small_batch_specs()
    best, ms, n = cortex.autotune(specs, seeds, trial_steps=200)
    assert n >= 20 and ms > 0
    assert best.warps_per_block in (8, 10, 12, 14, 16) and best.balance in (0, 1, 2)
    if best.balance == 2:
        assert len(best.work()) == len(specs) and min(best.work()) > 0
    uneven = cortex.make_options(warps_per_block=10, balance=2, net_work=[20.0, 1.0, 0.5, 3.0, 1.0, 8.0])
    rasters = []
    for opts in (best, cortex.make_options(warps_per_block=8, balance=1), uneven, cortex.make_options()):
        with cortex.Network(specs, seeds, opts) as net:
            if opts is uneven:
                assert net.stats()["n_blocks"] > len(specs)
            net.simulate(600)
            rasters.append([net.spikes(b) for b in range(len(specs))])
    for r in rasters[1:]:
        for (s0, i0), (s1, i1) in zip(rasters[0], r):
            assert np.array_equal(s0, s1) and np.array_equal(i0, i1)
    _, os_, oi, _ = oracle_run(specs[0], seeds[0], 600)
    assert first_mismatch(*rasters[0][0], os_, oi) == -1


def test_ring_matches_the_oracle_ring(cortex):
    """The ring of future input after 300 steps (cortex_get_ring, slot-major) equals the oracle's
    ring (neuron-major, slot = step mod D) element by element; shared-memory and global ring."""
    cfg = W.CONFIGS["c0"]
    spec, seed, steps = cfg["spec"], cfg["seed"], 300
    ref, _, _, _ = oracle_run(spec, seed, steps)
    oring = ref.ring()
    assert np.count_nonzero(oring) > 0
    for ring_mode in (1, 2):
        with cortex.Network(spec, seed, cortex.make_options(ring=ring_mode)) as net:
            net.simulate(steps)
            g = net.ring()
        assert g.shape == (spec.d_max + 1, spec.n)
        assert np.array_equal(g.T.astype(np.float64), oring)


def test_checkpoint_restore_continues_bit_exact(cortex):
    """State (V, I, refractory counts, ring) and step of a batch of networks after 300 steps,
    restored into fresh handles built from the same params and seeds: the next 300 steps give
    the same rasters and final states as the uninterrupted run, in both ring modes."""
    specs, seeds = W.small_batch_specs(n_nets=3)
    for ring_mode in (1, 2):
        opts = cortex.make_options(ring=ring_mode)
        with cortex.Network(specs, seeds, opts) as a:
            a.simulate(300)
            ck = [(a.state(b), a.ring(b)) for b in range(len(specs))]
            a.clear_spikes()
            a.simulate(300)
            ra = [a.spikes(b) for b in range(len(specs))]
            sa = [a.state(b) for b in range(len(specs))]
        with cortex.Network(specs, seeds, opts) as b_net:
            for b, ((v, c, r), g) in enumerate(ck):
                b_net.set_state(b, v=v, i_syn=c, refr=r, ring=g)
            b_net.set_step(300)
            b_net.simulate(300)
            for b in range(len(specs)):
                s1, i1 = b_net.spikes(b)
                assert np.array_equal(s1, ra[b][0]) and np.array_equal(i1, ra[b][1])
                assert len(s1) > 0 and s1.min() >= 300
                for x, y in zip(b_net.state(b), sa[b]):
                    assert np.array_equal(x, y)


def test_restore_from_the_oracle_state(cortex):
    """The oracle's FP32 state and ring after 200 steps, loaded into a fresh GPU handle at step
    200: the GPU's next 200 steps equal the oracle's continuation bit for bit.  This pins the
    checkpoint layout and the step convention against the oracle, not only against the GPU."""
    cfg = W.CONFIGS["c0"]
    spec, seed = cfg["spec"], cfg["seed"]
    ref = orc.Network(oracle_params(spec), seed)
    ref.simulate(200)
    v, c, r = ref.state()
    ring = ref.ring().T
    s0, _ = ref.raster()
    ref.simulate(200)
    s_all, i_all = ref.raster()
    keep = s_all >= 200
    with cortex.Network(spec, seed) as net:
        net.set_state(0, v=v.astype(np.float32), i_syn=c.astype(np.float32), refr=r, ring=ring.astype(np.float32))
        net.set_step(200)
        net.simulate(200)
        gs, gi = net.spikes()
        gv, gc, gr = net.state()
    assert len(s0) > 0 and keep.sum() > 0
    assert first_mismatch(gs, gi, s_all[keep], i_all[keep]) == -1
    ov, oc, orr = ref.state()
    assert np.array_equal(gv.astype(np.float64), ov) and np.array_equal(gc.astype(np.float64), oc)
    assert np.array_equal(gr, orr)


def test_set_state_refuses_bad_refractory_counts(cortex):
    cfg = W.CONFIGS["c0"]
    with cortex.Network(cfg["spec"], cfg["seed"]) as net:
        _, _, r = net.state()
        bad = r.copy()
        bad[5] = 10_000
        with pytest.raises(cortex.CortexError):
            net.set_state(0, refr=bad)
        with pytest.raises(cortex.CortexError):
            net.set_step(-1)


def test_host_plan_matches_the_build(cortex):
    """cortex_plan (host only) gives the block count the build makes on this GPU."""
    import torch
    props = torch.cuda.get_device_properties(0)
    smem = getattr(props, "shared_memory_per_block_optin", 232448)
    specs, seeds = W.small_batch_specs()
    for kw in (dict(), dict(balance=1), dict(balance=2, net_work=[20.0, 1.0, 0.5, 3.0, 1.0, 8.0]),
               dict(warps_per_block=8)):
        opts = cortex.make_options(**kw)
        _, nb = cortex.plan(specs, opts, n_sm=props.multi_processor_count, smem_per_block=smem)
        with cortex.Network(specs, seeds, opts) as net:
            assert net.stats()["n_blocks"] == nb, kw


def test_autotune_cache_answers_the_second_call(cortex, tmp_path):
    """cortex_autotune_cached: the first call tunes and appends the winner to the cache file, the
    second returns the same plan without building anything; another network set misses."""
    specs, seeds = W.small_batch_specs(n_nets=3)
    path = tmp_path / "autotune.cache"
    b1, ms1, n1, hit1 = cortex.autotune(specs, seeds, trial_steps=100, cache=path, with_hit=True)
    assert not hit1 and n1 > 0 and path.exists()
    b2, ms2, n2, hit2 = cortex.autotune(specs, seeds, trial_steps=100, cache=path, with_hit=True)
    assert hit2 and n2 == 0 and abs(ms2 - ms1) <= 1e-6 * ms1
    assert (b2.warps_per_block, b2.balance) == (b1.warps_per_block, b1.balance)
    if b1.balance == 2:
        assert np.allclose(b2.work(), b1.work())
    _, _, _, hit3 = cortex.autotune(specs, [s + 1 for s in seeds], trial_steps=100, cache=path, with_hit=True)
    assert not hit3
    assert len(path.read_text().splitlines()) == 2
