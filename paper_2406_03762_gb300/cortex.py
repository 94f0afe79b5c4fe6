"""Python binding of the C ABI in include/cortex.h (argument marshalling only).

Every step of the simulation runs in the CUDA library; this module only converts arguments.
There is no CPU fallback: if the library is missing or no GPU is present, load() raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

OK = 0
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_OVERFLOW, ERR_CHECK = -1, -2, -3, -4, -5, -6, -7
F32, BF16 = 0, 1
RING_AUTO, RING_SMEM, RING_GLOBAL = 0, 1, 2
MODE_PERSISTENT, MODE_SPLIT = 0, 1
FOLD_AUTO, FOLD_ORDERED, FOLD_EXACT = 0, 1, 2
DELIVERY_RING, DELIVERY_DELAY = 0, 1


class CortexError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where}: {detail} (status {code})")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("n_exc", ctypes.c_int32), ("n_inh", ctypes.c_int32), ("k_exc", ctypes.c_int32), ("k_inh", ctypes.c_int32),
        ("tau_m", ctypes.c_float), ("c_m", ctypes.c_float), ("tau_syn", ctypes.c_float), ("v_th", ctypes.c_float),
        ("v_reset", ctypes.c_float), ("e_l", ctypes.c_float), ("t_ref", ctypes.c_float), ("dt", ctypes.c_float),
        ("j_exc", ctypes.c_float), ("j_inh", ctypes.c_float),
        ("d_min", ctypes.c_int32), ("d_max", ctypes.c_int32),
        ("nu_ext_hz", ctypes.c_float), ("j_ext", ctypes.c_float),
        ("weight_dtype", ctypes.c_int32),
    ]


class Options(ctypes.Structure):
    _fields_ = [
        ("ring", ctypes.c_int32), ("mode", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
        ("targets_per_block", ctypes.c_int32), ("steps_per_launch", ctypes.c_int32), ("use_graph", ctypes.c_int32),
        ("raster_capacity", ctypes.c_int64), ("barrier_timeout_ms", ctypes.c_double),
        ("spikes_per_round", ctypes.c_int32), ("balance", ctypes.c_int32), ("test_withhold_block", ctypes.c_int32),
        ("net_work", ctypes.POINTER(ctypes.c_float)),
        ("fold", ctypes.c_int32), ("l2_persist", ctypes.c_int32), ("delivery", ctypes.c_int32),
        ("check_ownership", ctypes.c_int32), ("helper_warp", ctypes.c_int32),
    ]

    def work(self):
        """The per-network costs of a balance-2 plan (list of floats), or None."""
        keep = getattr(self, "_work", None)
        return None if keep is None or not self.net_work else list(keep)


class Stats(ctypes.Structure):
    _fields_ = [
        ("n_nets", ctypes.c_int64), ("n_neurons", ctypes.c_int64), ("n_synapses", ctypes.c_int64),
        ("step", ctypes.c_int64), ("spikes", ctypes.c_int64), ("events", ctypes.c_int64),
        ("build_ms", ctypes.c_double), ("simulate_ms", ctypes.c_double), ("simulate_steps", ctypes.c_int64),
        ("simulate_events", ctypes.c_int64), ("n_blocks", ctypes.c_int32), ("threads_per_block", ctypes.c_int32),
        ("ring_in_smem", ctypes.c_int32), ("mode", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
        ("spikes_per_round", ctypes.c_int32), ("smem_bytes", ctypes.c_int32),
        ("exact_fold", ctypes.c_int32), ("l2_persist_bytes", ctypes.c_int64), ("delivery", ctypes.c_int32),
        ("build_h2d_bytes", ctypes.c_int64), ("helper_warp", ctypes.c_int32),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


EXPORTED = [
    "cortex_build", "cortex_build_batch", "cortex_simulate", "cortex_spikes", "cortex_clear_spikes",
    "cortex_stats", "cortex_export_synapses", "cortex_get_state", "cortex_constants", "cortex_deliver",
    "cortex_philox", "cortex_free", "cortex_strerror", "cortex_last_error", "cortex_subgraph_noalloc",
    "cortex_autotune", "cortex_get_ring", "cortex_set_state", "cortex_set_step", "cortex_plan",
    "cortex_get_stamps", "cortex_check_stamps", "cortex_autotune_cached",
]

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load the CUDA library.  Raises if it is not built (no silent fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    L.cortex_build.argtypes = [P(Params), ctypes.c_uint64, P(Options), vp, P(vp)]
    L.cortex_build_batch.argtypes = [P(Params), P(ctypes.c_uint64), ctypes.c_int32, P(Options), vp, P(vp)]
    L.cortex_simulate.argtypes = [vp, ctypes.c_int64]
    L.cortex_spikes.argtypes = [vp, ctypes.c_int32, P(ctypes.c_int64), P(ctypes.c_int32), P(ctypes.c_int32)]
    L.cortex_clear_spikes.argtypes = [vp]
    L.cortex_stats.argtypes = [vp, P(Stats)]
    L.cortex_export_synapses.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P(ctypes.c_int64),
                                         P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_float)]
    L.cortex_get_state.argtypes = [vp, ctypes.c_int32, P(ctypes.c_float), P(ctypes.c_float), P(ctypes.c_int32)]
    L.cortex_constants.argtypes = [vp, ctypes.c_int32, P(ctypes.c_float), P(ctypes.c_uint32), P(ctypes.c_int32),
                                   P(ctypes.c_int32)]
    L.cortex_deliver.argtypes = [vp, ctypes.c_int32, P(ctypes.c_int32), ctypes.c_int64, ctypes.c_int64,
                                 ctypes.c_int32, P(ctypes.c_double), P(ctypes.c_int64)]
    L.cortex_philox.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), ctypes.c_int64, P(ctypes.c_uint32)]
    L.cortex_subgraph_noalloc.argtypes = [P(Params), ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, vp, vp, vp, vp, vp]
    L.cortex_get_ring.argtypes = [vp, ctypes.c_int32, P(ctypes.c_float)]
    L.cortex_set_state.argtypes = [vp, ctypes.c_int32, P(ctypes.c_float), P(ctypes.c_float), P(ctypes.c_int32),
                                   P(ctypes.c_float)]
    L.cortex_set_step.argtypes = [vp, ctypes.c_int64]
    L.cortex_autotune_cached.argtypes = [P(Params), P(ctypes.c_uint64), ctypes.c_int32, P(Options), ctypes.c_int32, vp,
                                         ctypes.c_char_p, P(Options), P(ctypes.c_double), P(ctypes.c_int32),
                                         P(ctypes.c_float), P(ctypes.c_int32)]
    L.cortex_get_stamps.argtypes = [vp, ctypes.c_int32, P(ctypes.c_uint32)]
    L.cortex_check_stamps.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      P(ctypes.c_uint32), P(ctypes.c_int64), P(ctypes.c_int64)]
    L.cortex_plan.argtypes = [P(Params), ctypes.c_int32, P(Options), ctypes.c_int32, ctypes.c_int64, P(ctypes.c_int32),
                              P(ctypes.c_int32)]
    L.cortex_autotune.argtypes = [P(Params), P(ctypes.c_uint64), ctypes.c_int32, P(Options), ctypes.c_int32, vp,
                                  P(Options), P(ctypes.c_double), P(ctypes.c_int32), P(ctypes.c_float)]
    for name in EXPORTED:
        if name not in ("cortex_free", "cortex_strerror", "cortex_last_error"):
            getattr(L, name).restype = ctypes.c_int
    L.cortex_free.argtypes = [vp]
    L.cortex_free.restype = None
    L.cortex_strerror.argtypes = [ctypes.c_int]
    L.cortex_strerror.restype = ctypes.c_char_p
    L.cortex_last_error.argtypes = []
    L.cortex_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(rc: int, where: str):
    if rc != OK:
        L = load()
        raise CortexError(rc, where, f"{L.cortex_strerror(rc).decode()}: {L.cortex_last_error().decode()}")


def _p(a: np.ndarray | None, ct):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ct))


def params_from_spec(spec) -> Params:
    """NetSpec (workloads) or any object with the same attribute names -> Params."""
    return Params(n_exc=spec.n_exc, n_inh=spec.n_inh, k_exc=spec.k_exc, k_inh=spec.k_inh, tau_m=spec.tau_m,
                  c_m=spec.c_m, tau_syn=spec.tau_syn, v_th=spec.v_th, v_reset=spec.v_reset, e_l=spec.e_l,
                  t_ref=spec.t_ref, dt=spec.dt, j_exc=spec.j_exc, j_inh=spec.j_inh, d_min=spec.d_min,
                  d_max=spec.d_max, nu_ext_hz=spec.nu_ext_hz, j_ext=spec.j_ext, weight_dtype=spec.weight_dtype)


def make_options(**kw) -> Options:
    """Options with the given fields set; net_work takes a sequence of floats (kept alive by the
    returned object)."""
    o = Options()
    for k, v in kw.items():
        if k == "net_work":
            _set_work(o, v)
        else:
            setattr(o, k, v)
    return o


def _set_work(o: Options, values):
    arr = (ctypes.c_float * len(values))(*[float(x) for x in values])
    o._work = arr
    o.net_work = ctypes.cast(arr, ctypes.POINTER(ctypes.c_float))


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


def autotune(specs, seeds, base: Options | None = None, trial_steps: int = 1000, stream=None, cache=None,
             with_hit: bool = False):
    """cortex_autotune (or cortex_autotune_cached with a cache file path): the fastest plan (warps
    per block x block balance) for these networks.  Returns (Options, ms per simulation step,
    number of candidates built) and, with with_hit, whether the cache answered; a balance-2 plan
    keeps its per-network costs alive with the returned Options."""
    L = load()
    if not isinstance(specs, (list, tuple)):
        specs, seeds = [specs], [seeds]
    arr = (Params * len(specs))(*[params_from_spec(s) for s in specs])
    sd = (ctypes.c_uint64 * len(specs))(*[int(x) for x in seeds])
    best = Options()
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int32(0)
    hit = ctypes.c_int32(0)
    work = (ctypes.c_float * len(specs))()
    if cache is None:
        rc = L.cortex_autotune(arr, sd, len(specs), ctypes.byref(base) if base is not None else None,
                               int(trial_steps), _stream_handle(stream), ctypes.byref(best), ctypes.byref(ms),
                               ctypes.byref(n), work)
    else:
        rc = L.cortex_autotune_cached(arr, sd, len(specs), ctypes.byref(base) if base is not None else None,
                                      int(trial_steps), _stream_handle(stream), str(cache).encode(), ctypes.byref(best),
                                      ctypes.byref(ms), ctypes.byref(n), work, ctypes.byref(hit))
    _check(rc, "cortex_autotune")
    if best.balance == 2:
        best._work = work  # best.net_work points into it
    else:
        best.net_work = None
    if with_hit:
        return best, float(ms.value), int(n.value), bool(hit.value)
    return best, float(ms.value), int(n.value)


def plan(specs, options: Options | None = None, n_sm: int = 152, smem_per_block: int = 232448):
    """cortex_plan: (targets per block of each network, block count) for a GPU with n_sm SMs and
    smem_per_block bytes of opt-in shared memory per block; host only."""
    L = load()
    if not isinstance(specs, (list, tuple)):
        specs = [specs]
    arr = (Params * len(specs))(*[params_from_spec(s) for s in specs])
    tb = np.zeros(len(specs), np.int32)
    nb = ctypes.c_int32(0)
    _check(L.cortex_plan(arr, len(specs), ctypes.byref(options) if options is not None else None, int(n_sm),
                         int(smem_per_block), _p(tb, ctypes.c_int32), ctypes.byref(nb)), "cortex_plan")
    return tb, int(nb.value)


class Network:
    """A handle of one or more networks on the GPU (cortex_build / cortex_build_batch)."""

    def __init__(self, specs, seeds, options: Options | None = None, stream=None):
        L = load()
        if not isinstance(specs, (list, tuple)):
            specs, seeds = [specs], [seeds]
        self.specs = list(specs)
        self.seeds = [int(s) for s in seeds]
        arr = (Params * len(specs))(*[params_from_spec(s) for s in specs])
        sd = (ctypes.c_uint64 * len(specs))(*self.seeds)
        h = ctypes.c_void_p(None)
        opt = ctypes.byref(options) if options is not None else None
        rc = L.cortex_build_batch(arr, sd, len(specs), opt, _stream_handle(stream), ctypes.byref(h))
        _check(rc, "cortex_build_batch")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().cortex_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def simulate(self, n_steps: int):
        _check(load().cortex_simulate(self._h, int(n_steps)), "cortex_simulate")

    def simulate_status(self, n_steps: int) -> int:
        return int(load().cortex_simulate(self._h, int(n_steps)))

    def spikes(self, net_idx: int = 0):
        L = load()
        n = ctypes.c_int64(0)
        rc = L.cortex_spikes(self._h, net_idx, ctypes.byref(n), None, None)
        if rc not in (OK, ERR_OVERFLOW):
            _check(rc, "cortex_spikes")
        steps = np.zeros(n.value, np.int32)
        ids = np.zeros(n.value, np.int32)
        if n.value:
            _check(L.cortex_spikes(self._h, net_idx, ctypes.byref(n), _p(steps, ctypes.c_int32), _p(ids, ctypes.c_int32)),
                   "cortex_spikes")
        return steps, ids

    def clear_spikes(self):
        _check(load().cortex_clear_spikes(self._h), "cortex_clear_spikes")

    def stats(self) -> dict:
        st = Stats()
        _check(load().cortex_stats(self._h, ctypes.byref(st)), "cortex_stats")
        return st.as_dict()

    def state(self, net_idx: int = 0):
        n = self.specs[net_idx].n_exc + self.specs[net_idx].n_inh
        v = np.zeros(n, np.float32)
        c = np.zeros(n, np.float32)
        r = np.zeros(n, np.int32)
        _check(load().cortex_get_state(self._h, net_idx, _p(v, ctypes.c_float), _p(c, ctypes.c_float),
                                       _p(r, ctypes.c_int32)), "cortex_get_state")
        return v, c, r

    def ring(self, net_idx: int = 0) -> np.ndarray:
        """cortex_get_ring: [D, n] float32, row s = input at the step t' in [t, t + D) with
        t' mod D == s (t the current step)."""
        spec = self.specs[net_idx]
        out = np.zeros((spec.d_max + 1, spec.n), np.float32)
        _check(load().cortex_get_ring(self._h, net_idx, _p(out, ctypes.c_float)), "cortex_get_ring")
        return out

    def set_state(self, net_idx: int = 0, v=None, i_syn=None, refr=None, ring=None):
        """cortex_set_state: restore any of V, I, refractory counts and the ring ([D, n])."""
        n = self.specs[net_idx].n
        def arr(x, dt, shape):
            if x is None:
                return None
            a = np.ascontiguousarray(x, dt)
            if a.shape != shape:
                raise ValueError(f"expected shape {shape}, got {a.shape}")
            return a
        v = arr(v, np.float32, (n,))
        c = arr(i_syn, np.float32, (n,))
        r = arr(refr, np.int32, (n,))
        g = arr(ring, np.float32, (self.specs[net_idx].d_max + 1, n))
        _check(load().cortex_set_state(self._h, net_idx, _p(v, ctypes.c_float), _p(c, ctypes.c_float),
                                       _p(r, ctypes.c_int32), _p(g, ctypes.c_float)), "cortex_set_state")

    def stamps(self, net_idx: int = 0) -> np.ndarray:
        """cortex_get_stamps: [D, n] uint32, the warp that wrote each ring cell (check mode)."""
        spec = self.specs[net_idx]
        out = np.zeros((spec.d_max + 1, spec.n), np.uint32)
        _check(load().cortex_get_stamps(self._h, net_idx, _p(out, ctypes.c_uint32)), "cortex_get_stamps")
        return out

    def set_step(self, step: int):
        _check(load().cortex_set_step(self._h, int(step)), "cortex_set_step")

    def constants(self, net_idx: int = 0):
        out6 = np.zeros(6, np.float32)
        thr = np.zeros(64, np.uint32)
        nthr = ctypes.c_int32(0)
        nref = ctypes.c_int32(0)
        _check(load().cortex_constants(self._h, net_idx, _p(out6, ctypes.c_float), _p(thr, ctypes.c_uint32),
                                       ctypes.byref(nthr), ctypes.byref(nref)), "cortex_constants")
        return out6, thr[:nthr.value].copy(), int(nref.value)

    def export_synapses(self, t_begin: int, t_end: int, net_idx: int = 0):
        L = load()
        n = ctypes.c_int64(0)
        rc = L.cortex_export_synapses(self._h, net_idx, t_begin, t_end, ctypes.byref(n), None, None, None, None)
        if rc not in (OK, ERR_OVERFLOW):
            _check(rc, "cortex_export_synapses")
        src = np.zeros(n.value, np.int32)
        tgt = np.zeros(n.value, np.int32)
        dly = np.zeros(n.value, np.int32)
        w = np.zeros(n.value, np.float32)
        if n.value:
            _check(L.cortex_export_synapses(self._h, net_idx, t_begin, t_end, ctypes.byref(n), _p(src, ctypes.c_int32),
                                            _p(tgt, ctypes.c_int32), _p(dly, ctypes.c_int32), _p(w, ctypes.c_float)),
                   "cortex_export_synapses")
        return src, tgt, dly, w

    def deliver(self, ids, t_emit: int, reps: int = 1, net_idx: int = 0):
        a = np.ascontiguousarray(ids, np.int32)
        ms = ctypes.c_double(0)
        ev = ctypes.c_int64(0)
        _check(load().cortex_deliver(self._h, net_idx, _p(a, ctypes.c_int32), len(a), int(t_emit), int(reps),
                                     ctypes.byref(ms), ctypes.byref(ev)), "cortex_deliver")
        return ms.value, ev.value


def check_stamps(stamps: np.ndarray, targets_per_block: int, warps: int, first_block: int = 0):
    """cortex_check_stamps (host only): (cells stamped by a warp that does not own them, index of
    the first, -1 if none) for stamps [D, n] of one network."""
    st = np.ascontiguousarray(stamps, np.uint32)
    depth, n = st.shape
    bad = ctypes.c_int64(0)
    first = ctypes.c_int64(0)
    _check(load().cortex_check_stamps(int(n), int(depth), int(targets_per_block), int(warps), int(first_block),
                                      _p(st, ctypes.c_uint32), ctypes.byref(bad), ctypes.byref(first)),
           "cortex_check_stamps")
    return int(bad.value), int(first.value)


def philox(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, np.uint32).reshape(-1, 2)
    out = np.zeros_like(c)
    _check(load().cortex_philox(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), len(c), _p(out, ctypes.c_uint32)),
           "cortex_philox")
    return out


def _check_device_buffer(name: str, t, dtype: str, min_numel: int):
    """A caller-owned output of cortex_subgraph_noalloc: the C side cannot see the size or the type
    of a device buffer, so a wrong one is refused here, before any launch (CortexError ERR_ARG)."""
    if t is None:
        if min_numel > 0:
            raise CortexError(ERR_ARG, "cortex_subgraph_noalloc", f"{name} is None")
        return
    if not getattr(t, "is_cuda", False):
        raise CortexError(ERR_ARG, "cortex_subgraph_noalloc", f"{name} must be a CUDA tensor")
    if str(getattr(t, "dtype", "")).replace("torch.", "") != dtype:
        raise CortexError(ERR_ARG, "cortex_subgraph_noalloc", f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise CortexError(ERR_ARG, "cortex_subgraph_noalloc", f"{name} must be contiguous")
    if t.numel() < min_numel:
        raise CortexError(ERR_ARG, "cortex_subgraph_noalloc", f"{name} holds {t.numel()} elements, needs {min_numel}")
    dev = getattr(t, "device", None)
    idx = getattr(dev, "index", None)
    if idx is not None:
        import torch
        if idx != torch.cuda.current_device():
            raise CortexError(ERR_ARG, "cortex_subgraph_noalloc", f"{name} is on cuda:{idx}, not the current device")


def subgraph_noalloc(spec, seed: int, t_begin: int, t_end: int, row_ptr, tgt, delay, weight, stream=None):
    """cortex_subgraph_noalloc: the caller passes contiguous CUDA tensors on the current device:
    int32 row_ptr[n + 1], int32 tgt/delay[nnz], float32 weight[nnz], nnz = (t_end - t_begin) * K.
    Each is checked (type, device, size) before the call, since the library writes into them."""
    n, k = spec.n_exc + spec.n_inh, spec.k_exc + spec.k_inh
    nnz = max(0, int(t_end) - int(t_begin)) * k
    _check_device_buffer("row_ptr", row_ptr, "int32", n + 1)
    _check_device_buffer("tgt", tgt, "int32", nnz)
    _check_device_buffer("delay", delay, "int32", nnz)
    _check_device_buffer("weight", weight, "float32", nnz)
    p = params_from_spec(spec)
    ptr = lambda t: ctypes.c_void_p(int(t.data_ptr())) if t is not None else None
    _check(load().cortex_subgraph_noalloc(ctypes.byref(p), int(seed), int(t_begin), int(t_end), _stream_handle(stream),
                                          ptr(row_ptr), ptr(tgt), ptr(delay), ptr(weight)), "cortex_subgraph_noalloc")
