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
