"""ctypes wrapper of the CPU oracle (``cortex_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of the benchmark
use it; the CUDA library never imports it.  The oracle is a plain single-threaded simulator of
the paper's model (LIF neurons, Eq. 1-2; exponential synaptic current, Eq. 3; the simulation
loop of Sec. II-B) and of the fixed in-degree connectivity, written without any blocking or
reordering so it can be checked against the paper by eye.

Pins (see ``tests/test_oracle_*.py``): Philox known-answer vectors, the analytic PSP, ODE
integration with an independent solver, step halving, the analytic inter-spike interval, the
Poisson pmf, hand-built graphs worked out by hand, and delivery invariants.  The whole-network
raster has no printed counterpart in the paper: parity with the paper is unpinned there.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cortex_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

FP32 = 0
FP64 = 1
POISSON_TABLE_CAP = 64


def build(force: bool = False) -> str:
    """Compile the oracle with gcc: no FP contraction, no fast-math (IEEE round-to-nearest)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp",
           "-o", tmp, _SRC, "-lm"]
    if subprocess.run(cmd, capture_output=True).returncode != 0:
        # no OpenMP runtime: the target-partitioned form then runs its parts one after another
        cmd.remove("-fopenmp")
        subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("n_exc", ctypes.c_int32), ("n_inh", ctypes.c_int32),
        ("k_exc", ctypes.c_int32), ("k_inh", ctypes.c_int32),
        ("tau_m", ctypes.c_double), ("c_m", ctypes.c_double), ("tau_syn", ctypes.c_double),
        ("v_th", ctypes.c_double), ("v_reset", ctypes.c_double), ("e_l", ctypes.c_double),
        ("t_ref", ctypes.c_double), ("dt", ctypes.c_double),
        ("j_exc", ctypes.c_double), ("j_inh", ctypes.c_double),
        ("d_min", ctypes.c_int32), ("d_max", ctypes.c_int32),
        ("nu_ext_hz", ctypes.c_double), ("j_ext", ctypes.c_double),
        ("i_e", ctypes.c_double),
        ("precision", ctypes.c_int32), ("bf16_weights", ctypes.c_int32),
        ("poisson_on", ctypes.c_int32),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        L.oracle_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
        L.oracle_philox4x32_10.restype = None
        L.oracle_round_bf16.argtypes = [ctypes.c_float]
        L.oracle_round_bf16.restype = ctypes.c_float
        L.oracle_propagators.argtypes = [P(_Params), P(ctypes.c_double), P(ctypes.c_float), P(ctypes.c_int32)]
        L.oracle_propagators.restype = None
        L.oracle_poisson_table.argtypes = [ctypes.c_double, P(ctypes.c_uint32), ctypes.c_int]
        L.oracle_poisson_table.restype = ctypes.c_int
        L.oracle_poisson_sample.argtypes = [ctypes.c_uint32, P(ctypes.c_uint32), ctypes.c_int]
        L.oracle_poisson_sample.restype = ctypes.c_int
        L.oracle_draw.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                  ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                  P(ctypes.c_int32), P(ctypes.c_int32)]
        L.oracle_draw.restype = None
        L.oracle_build.argtypes = [P(_Params), ctypes.c_uint64, P(vp)]
        L.oracle_build.restype = ctypes.c_int
        L.oracle_build_edges.argtypes = [P(_Params), ctypes.c_uint64, ctypes.c_int64, P(ctypes.c_int32),
                                         P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_double), P(vp)]
        L.oracle_build_edges.restype = ctypes.c_int
        L.oracle_build_par.argtypes = [P(_Params), ctypes.c_uint64, ctypes.c_int32, P(vp)]
        L.oracle_build_par.restype = ctypes.c_int
        L.oracle_set_threads.argtypes = [vp, ctypes.c_int32]
        L.oracle_set_threads.restype = ctypes.c_int
        L.oracle_free.argtypes = [vp]
        L.oracle_free.restype = None
        L.oracle_enable_accounting.argtypes = [vp]
        L.oracle_enable_accounting.restype = ctypes.c_int
        L.oracle_simulate.argtypes = [vp, ctypes.c_int64, ctypes.c_int64, P(ctypes.c_int64), P(ctypes.c_int32),
                                      ctypes.c_int64, P(ctypes.c_int32), P(ctypes.c_double)]
        L.oracle_simulate.restype = ctypes.c_int
        for name in ("oracle_n", "oracle_n_syn", "oracle_step", "oracle_events", "oracle_raster_size"):
            getattr(L, name).argtypes = [vp]
            getattr(L, name).restype = ctypes.c_int64
        L.oracle_depth.argtypes = [vp]
        L.oracle_depth.restype = ctypes.c_int32
        L.oracle_raster.argtypes = [vp, P(ctypes.c_int64), P(ctypes.c_int32)]
        L.oracle_raster.restype = None
        L.oracle_state.argtypes = [vp, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_int32)]
        L.oracle_state.restype = None
        L.oracle_ring.argtypes = [vp, P(ctypes.c_double)]
        L.oracle_ring.restype = None
        L.oracle_out_row.argtypes = [vp, P(ctypes.c_int64)]
        L.oracle_out_row.restype = None
        L.oracle_out_edges.argtypes = [vp, P(ctypes.c_int32), P(ctypes.c_int32)]
        L.oracle_out_edges.restype = None
        L.oracle_accounting.argtypes = [vp, P(ctypes.c_int64), P(ctypes.c_double)]
        L.oracle_accounting.restype = None
        L.oracle_constants_f32.argtypes = [vp, P(ctypes.c_float), P(ctypes.c_uint32), P(ctypes.c_int32),
                                           P(ctypes.c_int32)]
        L.oracle_constants_f32.restype = None
        L.oracle_set_state.argtypes = [vp, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_int32)]
        L.oracle_set_state.restype = None
        L.oracle_set_ring.argtypes = [vp, P(ctypes.c_double)]
        L.oracle_set_ring.restype = None
        L.oracle_v0_word.argtypes = [ctypes.c_uint64, ctypes.c_int64]
        L.oracle_v0_word.restype = ctypes.c_uint32
        L.oracle_poisson_word.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64]
        L.oracle_poisson_word.restype = ctypes.c_uint32
        L.oracle_replay.argtypes = [P(_Params), ctypes.c_uint64, ctypes.c_int64, P(ctypes.c_int32), ctypes.c_int64,
                                    ctypes.c_int64, P(ctypes.c_int64), P(ctypes.c_int32), ctypes.c_int64,
                                    P(ctypes.c_int64), P(ctypes.c_int32), P(ctypes.c_int64), P(ctypes.c_double),
                                    P(ctypes.c_double), P(ctypes.c_int32), P(ctypes.c_double)]
        L.oracle_replay.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


@dataclass
class Params:
    """Model parameters (units: ms, pF, mV, pA, Hz).  Defaults: the Brunel network of the
    benchmark configurations."""
    n_exc: int = 2000
    n_inh: int = 500
    k_exc: int = 200
    k_inh: int = 50
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
    d_min: int = 1
    d_max: int = 16
    nu_ext_hz: float = 15000.0
    j_ext: float = 87.8
    i_e: float = 0.0
    precision: int = FP32
    bf16_weights: int = 0
    poisson_on: int = 1

    def c(self) -> _Params:
        return _Params(**{f: getattr(self, f) for f, _ in _Params._fields_})


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def round_bf16(x: float) -> float:
    return float(lib().oracle_round_bf16(float(x)))


def propagators(p: Params):
    """Returns (p64[P11, P21, P22, P20, P22 - 1] float64, p32[...] float32, n_ref)."""
    o64 = np.zeros(5, dtype=np.float64)
    o32 = np.zeros(5, dtype=np.float32)
    nref = ctypes.c_int32(0)
    cp = p.c()
    lib().oracle_propagators(ctypes.byref(cp), _ptr(o64, ctypes.c_double), _ptr(o32, ctypes.c_float),
                             ctypes.byref(nref))
    return o64, o32, int(nref.value)


def poisson_table(lam: float) -> np.ndarray:
    thr = np.zeros(POISSON_TABLE_CAP, dtype=np.uint32)
    n = lib().oracle_poisson_table(float(lam), _ptr(thr, ctypes.c_uint32), POISSON_TABLE_CAP)
    if n < 1:
        raise ValueError("Poisson table does not saturate")
    return thr[:n].copy()


def poisson_sample(u: int, thr: np.ndarray) -> int:
    t = np.ascontiguousarray(thr, dtype=np.uint32)
    return int(lib().oracle_poisson_sample(int(u), _ptr(t, ctypes.c_uint32), len(t)))


def draw(seed: int, p: Params, i: int, j: int):
    s = ctypes.c_int32(0)
    d = ctypes.c_int32(0)
    lib().oracle_draw(seed, p.n_exc, p.n_inh, p.k_exc, p.d_min, p.d_max, i, j, ctypes.byref(s), ctypes.byref(d))
    return int(s.value), int(d.value)


def incoming(seed: int, p: Params, i: int):
    """All K draws of target i as arrays (sources, delays), in draw order."""
    k = p.k_exc + p.k_inh
    src = np.empty(k, dtype=np.int32)
    dly = np.empty(k, dtype=np.int32)
    for j in range(k):
        src[j], dly[j] = draw(seed, p, i, j)
    return src, dly


def v0_word(seed: int, i: int) -> int:
    return int(lib().oracle_v0_word(seed, i))


def poisson_word(seed: int, i: int, t: int) -> int:
    return int(lib().oracle_poisson_word(seed, i, t))


def replay(p: Params, seed: int, targets, n_steps: int, raster_steps, raster_ids, trace: bool = False):
    """Simulate only the given targets of the Philox network, driven by a given raster of the whole
    network (its (step, id) pairs sorted by step, then id).  Returns (spike steps, spike ids) of the
    targets, in (step, id) order, and their final (V, I, refractory count) as arrays in target
    order; with trace=True also V of every target after every step ([n_steps, targets]).  A target's trajectory depends only on its own incoming synapses and the raster, so
    this checks a large simulation one neuron at a time."""
    t = np.ascontiguousarray(np.unique(np.asarray(targets, dtype=np.int32)))
    rs = np.ascontiguousarray(np.asarray(raster_steps, dtype=np.int64))
    ri = np.ascontiguousarray(np.asarray(raster_ids, dtype=np.int32))
    cap = max(1024, 4 * len(t) * max(1, n_steps // 20))
    while True:
        os_ = np.empty(cap, dtype=np.int64)
        oi = np.empty(cap, dtype=np.int32)
        n_out = ctypes.c_int64(0)
        v = np.empty(len(t), dtype=np.float64)
        c = np.empty(len(t), dtype=np.float64)
        r = np.empty(len(t), dtype=np.int32)
        tr = np.empty((n_steps, len(t)), dtype=np.float64) if trace else None
        pc = p.c()
        rc = lib().oracle_replay(ctypes.byref(pc), seed, len(t), _ptr(t, ctypes.c_int32), n_steps, len(rs),
                                 _ptr(rs, ctypes.c_int64), _ptr(ri, ctypes.c_int32), cap,
                                 _ptr(os_, ctypes.c_int64), _ptr(oi, ctypes.c_int32), ctypes.byref(n_out),
                                 _ptr(v, ctypes.c_double), _ptr(c, ctypes.c_double), _ptr(r, ctypes.c_int32),
                                 _ptr(tr, ctypes.c_double) if trace else None)
        if rc != 0:
            raise RuntimeError(f"oracle_replay failed ({rc})")
        if n_out.value <= cap:
            if trace:
                return os_[:n_out.value], oi[:n_out.value], (v, c, r), tr
            return os_[:n_out.value], oi[:n_out.value], (v, c, r)
        cap = int(n_out.value)


class Network:
    """One oracle network (Philox connectivity or a hand-built edge list)."""

    def __init__(self, p: Params, seed: int, edges=None, accounting: bool = False, threads: int = 1):
        """threads > 1: the target-partitioned form (same results bit for bit; no forced spikes,
        traces or accounting)."""
        self.p = p
        self.seed = seed
        h = ctypes.c_void_p(None)
        cp = p.c()
        if edges is None and threads > 1:
            rc = lib().oracle_build_par(ctypes.byref(cp), seed, int(threads), ctypes.byref(h))
        elif edges is None:
            rc = lib().oracle_build(ctypes.byref(cp), seed, ctypes.byref(h))
        else:
            src, tgt, dly, w = (np.ascontiguousarray(edges[0], np.int32), np.ascontiguousarray(edges[1], np.int32),
                                np.ascontiguousarray(edges[2], np.int32), np.ascontiguousarray(edges[3], np.float64))
            rc = lib().oracle_build_edges(ctypes.byref(cp), seed, len(src), _ptr(src, ctypes.c_int32),
                                          _ptr(tgt, ctypes.c_int32), _ptr(dly, ctypes.c_int32),
                                          _ptr(w, ctypes.c_double), ctypes.byref(h))
        if rc != 0:
            raise RuntimeError(f"oracle build failed: {rc}")
        self._h = h
        if accounting and lib().oracle_enable_accounting(h) != 0:
            raise MemoryError("oracle accounting")

    def close(self):
        if self._h:
            lib().oracle_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n(self) -> int:
        return int(lib().oracle_n(self._h))

    @property
    def n_syn(self) -> int:
        return int(lib().oracle_n_syn(self._h))

    @property
    def step(self) -> int:
        return int(lib().oracle_step(self._h))

    @property
    def events(self) -> int:
        return int(lib().oracle_events(self._h))

    @property
    def depth(self) -> int:
        return int(lib().oracle_depth(self._h))

    def simulate(self, n_steps: int, forced=None, trace_ids=None):
        """Advance n_steps.  forced: (steps, ids) spikes emitted in addition to the neurons' own.
        trace_ids: neurons whose V is recorded after every step; returns [n_steps, len] or None."""
        fs = np.zeros(0, np.int64)
        fi = np.zeros(0, np.int32)
        if forced is not None:
            order = np.argsort(np.asarray(forced[0]), kind="stable")
            fs = np.ascontiguousarray(np.asarray(forced[0], np.int64)[order])
            fi = np.ascontiguousarray(np.asarray(forced[1], np.int32)[order])
        tr = None
        tid = np.zeros(0, np.int32)
        if trace_ids is not None:
            tid = np.ascontiguousarray(trace_ids, np.int32)
            tr = np.zeros((n_steps, len(tid)), np.float64)
        rc = lib().oracle_simulate(self._h, n_steps, len(fs), _ptr(fs, ctypes.c_int64), _ptr(fi, ctypes.c_int32),
                                   len(tid), _ptr(tid, ctypes.c_int32),
                                   _ptr(tr, ctypes.c_double) if tr is not None else None)
        if rc != 0:
            raise RuntimeError(f"oracle simulate failed: {rc}")
        return tr

    def set_threads(self, threads: int):
        """Threads that step a target-partitioned network (results do not depend on it)."""
        if lib().oracle_set_threads(self._h, int(threads)) != 0:
            raise ValueError("set_threads: only for a network built with threads > 1")

    def raster(self):
        n = int(lib().oracle_raster_size(self._h))
        s = np.zeros(n, np.int64)
        i = np.zeros(n, np.int32)
        if n:
            lib().oracle_raster(self._h, _ptr(s, ctypes.c_int64), _ptr(i, ctypes.c_int32))
        return s, i

    def state(self):
        n = self.n
        v = np.zeros(n, np.float64)
        c = np.zeros(n, np.float64)
        r = np.zeros(n, np.int32)
        lib().oracle_state(self._h, _ptr(v, ctypes.c_double), _ptr(c, ctypes.c_double), _ptr(r, ctypes.c_int32))
        return v, c, r

    def set_state(self, v, cur, refr):
        v = np.ascontiguousarray(v, np.float64)
        c = np.ascontiguousarray(cur, np.float64)
        r = np.ascontiguousarray(refr, np.int32)
        lib().oracle_set_state(self._h, _ptr(v, ctypes.c_double), _ptr(c, ctypes.c_double), _ptr(r, ctypes.c_int32))

    def set_ring(self, ring):
        """Overwrite the ring ([n, D], as ring() returns it)."""
        g = np.ascontiguousarray(ring, np.float64)
        if g.shape != (self.n, self.depth):
            raise ValueError(f"expected shape {(self.n, self.depth)}, got {g.shape}")
        lib().oracle_set_ring(self._h, _ptr(g, ctypes.c_double))

    def ring(self) -> np.ndarray:
        out = np.zeros((self.n, self.depth), np.float64)
        lib().oracle_ring(self._h, _ptr(out, ctypes.c_double))
        return out

    def outgoing(self):
        """CSR by source: (row[n+1], tgt[n_syn], delay[n_syn]) sorted by (source, target, draw)."""
        row = np.zeros(self.n + 1, np.int64)
        lib().oracle_out_row(self._h, _ptr(row, ctypes.c_int64))
        tgt = np.zeros(self.n_syn, np.int32)
        dly = np.zeros(self.n_syn, np.int32)
        lib().oracle_out_edges(self._h, _ptr(tgt, ctypes.c_int32), _ptr(dly, ctypes.c_int32))
        return row, tgt, dly

    def accounting(self):
        ev = np.zeros(self.n, np.int64)
        w = np.zeros(self.n, np.float64)
        lib().oracle_accounting(self._h, _ptr(ev, ctypes.c_int64), _ptr(w, ctypes.c_double))
        return ev, w

    def constants_f32(self):
        c8 = np.zeros(8, np.float32)
        thr = np.zeros(POISSON_TABLE_CAP, np.uint32)
        nthr = ctypes.c_int32(0)
        nref = ctypes.c_int32(0)
        lib().oracle_constants_f32(self._h, _ptr(c8, ctypes.c_float), _ptr(thr, ctypes.c_uint32),
                                   ctypes.byref(nthr), ctypes.byref(nref))
        return c8, thr[:nthr.value].copy(), int(nref.value)
