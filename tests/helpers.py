"""Shared test helpers: converting a workload spec into oracle parameters, running both sides."""
import numpy as np

from oracle import oracle as orc


def oracle_params(spec, precision=orc.FP32, bf16=None):
    d = {k: v for k, v in spec.as_dict().items() if k in orc.Params.__dataclass_fields__}
    d["precision"] = precision
    d["bf16_weights"] = int(spec.weight_dtype == 1) if bf16 is None else int(bf16)
    return orc.Params(**d)


def oracle_run(spec, seed, steps, precision=orc.FP32, trace_ids=None):
    net = orc.Network(oracle_params(spec, precision), seed)
    tr = net.simulate(steps, trace_ids=trace_ids)
    s, i = net.raster()
    return net, s, i, tr


def first_mismatch(s1, i1, s2, i2):
    n = min(len(s1), len(s2))
    bad = np.nonzero((np.asarray(s1[:n]) != np.asarray(s2[:n])) | (np.asarray(i1[:n]) != np.asarray(i2[:n])))[0]
    if len(bad):
        return int(bad[0])
    if len(s1) != len(s2):
        return n
    return -1


def fp64_replay_check(spec, seed, steps, s32, i32, v32):
    """FP32 potentials against FP64: the FP64 oracle replays every neuron driven by the FP32 run's
    own raster (same presynaptic spikes), so each neuron's V differs only by its own arithmetic.
    A neuron is compared up to the first step where its own spikes differ between the two.
    Returns (max |V32 - V64| / max(|V64|, V_th), fraction of neurons whose spikes all agree)."""
    n = spec.n
    p64 = oracle_params(spec, orc.FP64, bf16=0)
    ps, pi, _, v64 = orc.replay(p64, seed, np.arange(n), steps, s32, i32, trace=True)
    first = np.full(n, steps, dtype=np.int64)
    s32, i32 = np.asarray(s32), np.asarray(i32)
    by32 = [[] for _ in range(n)]
    by64 = [[] for _ in range(n)]
    for s, i in zip(s32[s32 < steps], i32[s32 < steps]):
        by32[i].append(int(s))
    for s, i in zip(ps, pi):
        by64[i].append(int(s))
    for i in range(n):
        a, b = by32[i], by64[i]
        m = min(len(a), len(b))
        d = [k for k in range(m) if a[k] != b[k]]
        if d:
            first[i] = min(a[d[0]], b[d[0]])
        elif len(a) != len(b):
            first[i] = (a if len(a) > len(b) else b)[m]
    t = np.arange(steps)[:, None]
    ok = t < first[None, :]
    err = np.abs(np.asarray(v32)[:steps] - v64) / np.maximum(np.abs(v64), spec.v_th)
    return float(err[ok].max()), float(np.mean(first >= steps))
