"""Seeded synthetic workloads: the Brunel balanced random networks used for parity tests and
benchmarks.  This module only holds parameter sets and the seeded recipe for the batched
instances; it contains none of the model's arithmetic and imports neither the CUDA library nor
the oracle, so both sides can take their inputs from it.

The networks stand in for the paper's evaluation workloads (Sec. IV: balanced random network,
LIF neurons with exponential synaptic currents), which need external connectome data that is not
used here.  Every configuration: tau_m = 10 ms, C_m = 250 pF, tau_syn = 0.5 ms, V_th = 20 mV,
V_reset = 0 mV, E_L = 0, t_ref = 2 ms, dt = 0.1 ms, J_E = 87.8 pA, J_I = -5 J_E, external Poisson
drive at weight J_E, uniform integer delays, fixed in-degree with an 80/20 E/I split.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, asdict, replace

import numpy as np

BASE_SEED = 20240606

F32 = 0
BF16 = 1


@dataclass(frozen=True)
class NetSpec:
    """One network: sizes, delays, drive and weight storage.  Units: ms, pF, mV, pA, Hz."""
    n_exc: int
    n_inh: int
    k_exc: int
    k_inh: int
    d_min: int = 1
    d_max: int = 16
    nu_ext_hz: float = 15000.0
    weight_dtype: int = F32
    tau_m: float = 10.0
    c_m: float = 250.0
    tau_syn: float = 0.5
    v_th: float = 20.0
    v_reset: float = 0.0
    e_l: float = 0.0
    t_ref: float = 2.0
    dt: float = 0.1
    j_exc: float = 87.8
    j_inh: float = -439.0
    j_ext: float = 87.8

    @property
    def n(self) -> int:
        return self.n_exc + self.n_inh

    @property
    def k(self) -> int:
        return self.k_exc + self.k_inh

    def as_dict(self) -> dict:
        return asdict(self)


def brunel(n: int, k: int, **kw) -> NetSpec:
    """80/20 split of n neurons and of the in-degree k (rounded to nearest)."""
    n_exc = int(round(0.8 * n))
    k_exc = int(round(0.8 * k))
    return NetSpec(n_exc=n_exc, n_inh=n - n_exc, k_exc=k_exc, k_inh=k - k_exc, **kw)


# The five benchmark configurations (sizes, delays, drive, precision, simulated time).
CONFIGS = {
    "c0": dict(spec=NetSpec(2000, 500, 200, 50), steps=2000, seed=BASE_SEED + 0,
               name="brunel_n2500_k250_fp32"),
    "c1": dict(spec=NetSpec(90000, 22500, 9000, 2250), steps=10000, seed=BASE_SEED + 1,
               name="brunel_n112500_k11250_fp32"),
    "c2": dict(spec=NetSpec(400000, 100000, 4000, 1000, d_min=5, d_max=40, nu_ext_hz=12000.0),
               steps=10000, seed=BASE_SEED + 2, name="brunel_n500k_k5000_d5-40_fp32"),
    "c3": dict(spec=NetSpec(800000, 200000, 9000, 2250, weight_dtype=BF16), steps=10000,
               seed=BASE_SEED + 3, name="brunel_n1m_k11250_bf16"),
    "c4": dict(spec=None, steps=5000, seed=BASE_SEED + 4, n_nets=64,
               name="batch64_brunel_n2k-50k"),
}

# Profiling cases: the c1, c2 and c3 models at a quarter of the neurons and of the in-degree (same
# K/N, so the same per-block segment structure per source), small enough for ncu replay.
PROFILE = {
    "c1q": dict(spec=NetSpec(22500, 5625, 2250, 562), steps=2000, seed=BASE_SEED + 11,
                name="brunel_n28125_k2812_fp32"),
    "c2q": dict(spec=NetSpec(100000, 25000, 1000, 250, d_min=5, d_max=40, nu_ext_hz=12000.0), steps=2000,
                seed=BASE_SEED + 12, name="brunel_n125k_k1250_d5-40_fp32"),
    "c3q": dict(spec=NetSpec(200000, 50000, 2250, 562, weight_dtype=BF16), steps=2000, seed=BASE_SEED + 13,
                name="brunel_n250k_k2812_bf16"),
    # DRAM-traffic cases: fewer neurons at the full in-degree, so a source's piece per block (K over
    # the blocks) and the header share per synaptic event are those of the full configuration
    "c1r": dict(spec=NetSpec(22500, 5625, 9000, 2250), steps=2000, seed=BASE_SEED + 21,
                name="brunel_n28125_k11250_fp32"),
    "c2r": dict(spec=NetSpec(100000, 25000, 4000, 1000, d_min=5, d_max=40, nu_ext_hz=12000.0), steps=2000,
                seed=BASE_SEED + 22, name="brunel_n125k_k5000_d5-40_fp32"),
    "c3r": dict(spec=NetSpec(40000, 10000, 9000, 2250, weight_dtype=BF16), steps=2000, seed=BASE_SEED + 23,
                name="brunel_n50k_k11250_bf16"),
}

# Same statistics as c3 at 10,000 neurons (K = 11,250 > N, so sources repeat).
C3_SUBSAMPLE = dict(spec=NetSpec(8000, 2000, 9000, 2250, weight_dtype=BF16), steps=10000,
                    seed=BASE_SEED + 3, name="brunel_n10k_k11250_bf16")


def batch_specs(master_seed: int = BASE_SEED + 4, n_nets: int = 64):
    """The batched workload: n_nets independent Brunel networks.
    N_b = round(exp(U(ln 2000, ln 50000))), N_E = round(0.8 N_b), K = min(floor(N_b / 10), 5000),
    K_E = round(0.8 K), nu_ext ~ U(10, 20) kHz, seed_b = master_seed + 1 + b."""
    rng = np.random.default_rng(master_seed)
    specs, seeds = [], []
    for b in range(n_nets):
        n = int(round(math.exp(rng.uniform(math.log(2000.0), math.log(50000.0)))))
        k = min(n // 10, 5000)
        nu = float(rng.uniform(10000.0, 20000.0))
        specs.append(brunel(n, k, nu_ext_hz=nu))
        seeds.append(master_seed + 1 + b)
    return specs, seeds


def small_batch_specs(master_seed: int = 7, n_nets: int = 6, n_lo: int = 200, n_hi: int = 3000):
    """A small batch with the same recipe at test sizes (several nets, uneven sizes)."""
    rng = np.random.default_rng(master_seed)
    specs, seeds = [], []
    for b in range(n_nets):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        k = max(2, min(n // 10, 5000))
        nu = float(rng.uniform(10000.0, 20000.0))
        specs.append(brunel(n, k, nu_ext_hz=nu))
        seeds.append(master_seed + 1 + b)
    return specs, seeds


def scaled(spec: NetSpec, n: int, k: int | None = None) -> NetSpec:
    """Same model at another size (keeps delays, drive, precision)."""
    k = spec.k if k is None else k
    n_exc = int(round(0.8 * n))
    k_exc = int(round(0.8 * k))
    return replace(spec, n_exc=n_exc, n_inh=n - n_exc, k_exc=k_exc, k_inh=k - k_exc)
