"""Benchmark: synaptic events/s and real-time factor of the spike-delivery hot path on one GB300.

One benchmark step = one cortex_simulate call of --sim-steps simulation steps (default 10,000 steps
= 1 s of simulated time) of the deep-delay balanced random network N = 500,000, K = 5,000, delays
5..40 steps, FP32 weights (2.5e9 synapses, 15 GB of records on the device, so every step reads far
more than the 129 MB L2).  Each simulation step runs the whole hot path: neuron update, spike
compaction, publication, grid barrier and delivery.  Inputs are synthetic (a seeded network), built
on the device before timing.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank simulates its own replica (weak scaling, no collective on the data
path); rank 0 prints one JSON line.  At one GPU the line also carries "forms": the same metric for
the 112,500-neuron network, the BF16-weight network (N = 1e6, K = 11,250), the batch of 64 networks
(500 ms), the delay-ordered delivery on the deep-delay and BF16 networks, and the delivery kernel
alone, each timed after the main measurement on the same GPU with its own clock record.
--impl reference times the CPU oracle, target-partitioned over all host cores, on bounded samples
of the same network and prints the same metric.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "synaptic events/s"
UNIT = "events/s"
BYTES_PER_EVENT = {0: 7, 1: 5}   # FP32: w 4 B + local target 2 B + delay 1 B; BF16: 2 + 2 + 1
HEADLINE = "c2"


def replica_seed(base_seed: int, rank: int) -> int:
    """Seed of rank's replica: every rank simulates its own network (weak scaling)."""
    return int(base_seed) + 1000 * int(rank)


def replica_aggregate(ms: float, events: float, dist, device: str = "cuda"):
    """Whole-job numbers over the ranks: the slowest rank's time and the sum of the events
    (no collective on the data path; one max and one sum after the timed region)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    e = torch.tensor([float(events)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), float(e.item())


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload_config(cfg) -> dict:
    """The workload as both arms name it: what is simulated, not how."""
    spec = cfg["spec"]
    if spec is None:  # the batch of uneven networks
        from paper_2406_03762_gb300 import workloads as W
        specs, _ = W.batch_specs()
        return {"workload": cfg["name"], "n_nets": len(specs), "n_neurons": sum(x.n for x in specs),
                "synapses": sum(x.n * x.k for x in specs), "weights": "f32", "dt_ms": specs[0].dt,
                "l2": "inputs larger than L2 (records %.1f GB)" % (sum(x.n * x.k for x in specs) * 6 / 1e9)}
    return {"workload": cfg["name"], "n_neurons": spec.n, "k": spec.k, "synapses": spec.n * spec.k,
            "d_min": spec.d_min, "d_max": spec.d_max, "weights": "bf16" if spec.weight_dtype == 1 else "f32",
            "dt_ms": spec.dt, "l2": "inputs larger than L2 (records %.1f GB)" % (
                spec.n * spec.k * (4 if spec.weight_dtype == 1 else 6) / 1e9)}


def host_info() -> dict:
    mem = None
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemTotal:"):
                mem = round(int(line.split()[1]) / 1e6, 1)
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "host_memory_gb": mem}


# ---------------------------------------------------------------------------------------------
# CPU oracle runs (a spawned process: no CUDA state is inherited)
# ---------------------------------------------------------------------------------------------
def _oracle_job(cfg_name: str, threads: int, samples, q):
    """Build the oracle target-partitioned over `threads` parts (untimed), then time each
    (n_steps, n_threads) sample in turn."""
    sys.path.insert(0, ROOT)
    from oracle import oracle as orc
    from paper_2406_03762_gb300 import workloads as W
    cfg = W.CONFIGS[cfg_name] if cfg_name in W.CONFIGS else W.PROFILE[cfg_name]
    spec = cfg["spec"]
    d = {k: v for k, v in spec.as_dict().items() if k in orc.Params.__dataclass_fields__}
    d["bf16_weights"] = int(spec.weight_dtype == 1)
    t0 = time.perf_counter()
    net = orc.Network(orc.Params(**d), cfg["seed"], threads=threads)
    build_s = time.perf_counter() - t0
    out = []
    for n_steps, n_threads in samples:
        net.set_threads(n_threads)
        e0 = net.events
        t0 = time.perf_counter()
        net.simulate(n_steps)
        out.append((net.events - e0, time.perf_counter() - t0, n_steps, n_threads))
    q.put(dict(build_s=build_s, samples=out, step=net.step))


def run_oracle(cfg_name, threads, samples, timeout):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_oracle_job, args=(cfg_name, threads, samples, q), daemon=True)
    p.start()
    try:
        return q.get(timeout=timeout)
    finally:
        p.join(timeout=10)
        if p.is_alive():
            p.terminate()


# ---------------------------------------------------------------------------------------------
# clocks during a timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples every 20 ms; stop() keeps those taken inside [mark_start, mark_end]."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"cortex_clocks_{os.getpid()}_{id(self)}.csv")
        self.t0 = self.t1 = None

    def start(self):
        try:
            with open(self.path, "w") as out:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                     "-lms", "20"], stdout=out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            try:
                os.remove(self.path)  # no sampler on this machine: leave nothing behind
            except OSError:
                pass
            return self
        # wait (at most 3 s) for the first sample so that sampling covers the timed region
        t_end = time.time() + 3.0
        while time.time() < t_end:
            try:
                if os.path.getsize(self.path) > 0:
                    break
            except OSError:
                pass
            time.sleep(0.01)
        return self

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        import datetime
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            rows.append((ts, parts[1:]))
        try:
            os.remove(self.path)
        except OSError:
            pass
        inside = [r for ts, r in rows if ts is not None and self.t0 is not None and self.t1 is not None
                  and self.t0 - 0.02 <= ts <= self.t1 + 0.02]
        use = inside if inside else [r for _, r in rows]
        if not use:
            return None
        sm = sorted(float(r[1]) for r in use if r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in use if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in use for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(use), "samples_in_timed_region": len(inside)}


# ---------------------------------------------------------------------------------------------
def reference_arm(args):
    """The oracle, target-partitioned over all host cores, on bounded samples of the same network."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfg = _config(args.config)
    cores = os.cpu_count() or 1
    res = run_oracle(args.config, cores, [(args.ref_sample_steps, cores)] * (args.warmup + args.steps),
                     args.cpu_timeout)
    timed = res["samples"][args.warmup:]
    ev = sum(x[0] for x in timed)
    sec = sum(x[1] for x in timed)
    value = ev / sec if sec > 0 else 0.0
    spec = cfg["spec"]
    sim_s = args.ref_sample_steps * spec.dt * 1e-3 * len(timed)
    sample = (f"{cfg['name']}: oracle build {res['build_s']:.1f} s (untimed, {cores} parts), then {args.warmup} + "
              f"{args.steps} samples of {args.ref_sample_steps} simulation steps each on {cores} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / max(1, len(timed)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if spec.weight_dtype == 0 else "bf16", "data": "synthetic",
        "config": workload_config(cfg), "sim_steps_per_step": args.ref_sample_steps,
        "rtf": sec / sim_s if sim_s > 0 else None,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         **host_info()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def our_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    import torch
    from paper_2406_03762_gb300 import cortex
    from paper_2406_03762_gb300 import workloads as W

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    cortex.load()
    cfg = _config(args.config)
    spec = cfg["spec"]
    seed = replica_seed(cfg["seed"], rank)
    net_spec, net_seed = spec, seed
    if spec is None:  # the batch of uneven networks (library's default plan; the form autotunes it)
        specs, seeds = W.batch_specs()
        net_spec, net_seed = specs, [replica_seed(x, rank) for x in seeds]
        spec = specs[0]  # per-network values below (weight type, dt) are common to the batch
    stream = torch.cuda.Stream()
    opts = cortex.make_options(steps_per_launch=args.steps_per_launch, warps_per_block=args.warps,
                               delivery=args.delivery)
    net = cortex.Network(net_spec, net_seed, opts, stream=stream)
    st0 = net.stats()

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        net.simulate(args.sim_steps)
        net.clear_spikes()
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local).start()
    ev_a = torch.cuda.Event(enable_timing=True)
    ev_b = torch.cuda.Event(enable_timing=True)
    st_b = net.stats()
    e_before, s_before = st_b["events"], st_b["spikes"]
    clocks.mark_start()
    ev_a.record(stream)
    kern_ms = 0.0
    for _ in range(args.steps):
        net.simulate(args.sim_steps)          # launches on `stream`
        kern_ms += net.stats()["simulate_ms"]
        net.clear_spikes()                    # the device raster keeps one step's spikes
    ev_b.record(stream)
    torch.cuda.synchronize()
    clocks.mark_end()
    barrier()
    clk = clocks.stop()
    ms = ev_a.elapsed_time(ev_b)
    st = net.stats()
    events = st["events"] - e_before
    spikes = st["spikes"] - s_before
    ms_max, events_all = replica_aggregate(ms, events, dist, "cuda")
    value = events_all / (ms_max * 1e-3)
    sim_s = args.steps * args.sim_steps * spec.dt * 1e-3
    rtf = (ms_max * 1e-3) / sim_s
    net.close()

    # end to end through the public API, every step: build the network from its parameters (the
    # step's inputs, copied host -> device by the build), simulate, read the raster back, free
    d2h = h2d = 0
    e2e_events = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        with cortex.Network(net_spec, net_seed, opts, stream=stream) as n2:
            n2.simulate(args.sim_steps)
            s_, i_ = n2.spikes()
            st2 = n2.stats()
            d2h += s_.nbytes + i_.nbytes
            h2d += st2["build_h2d_bytes"]
            e2e_events += st2["events"]
    e2e_s = time.perf_counter() - t0
    e2e_value = e2e_events * world / e2e_s

    # roofline of the dominant kernel (the persistent step kernel): algorithmic record bytes
    launches_per_step = max(1, -(-args.sim_steps // args.steps_per_launch))
    launches = args.steps * launches_per_step
    bpe = BYTES_PER_EVENT[spec.weight_dtype]
    per_launch_bytes = events * bpe / launches
    launch_ms = kern_ms / launches
    peak, peak_kind = _peaks()
    achieved = per_launch_bytes / (launch_ms * 1e-3) / 1e9
    kname = "k_dstep (persistent, delay-ordered)" if args.delivery == 1 else "k_step (persistent)"
    traffic = _traffic(per_launch_bytes / bpe, TRAFFIC_RECORDS.get((args.config, args.delivery)))

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if spec.weight_dtype == 0 else "bf16", "data": "synthetic",
        "config": workload_config(cfg), "sim_steps_per_step": args.sim_steps,
        "plan": {"replicas": world, "blocks": st0["n_blocks"], "threads_per_block": st0["threads_per_block"],
                 "ring_in_smem": st0["ring_in_smem"], "spikes_per_round": st0["spikes_per_round"],
                 "smem_bytes": st0["smem_bytes"], "delivery": "delay" if args.delivery == 1 else "ring",
                 "exact_fold": st0["exact_fold"], "helper_warp": st0["helper_warp"]},
        "rtf": rtf,
        "spikes": spikes, "events": events,
        "build_ms": st0["build_ms"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_kind": peak_kind, "bytes_per_event": bpe,
                     "kernel": kname, "launch_ms": launch_ms},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d // args.steps,
                "d2h_bytes_per_step": d2h // args.steps,
                "includes": "cortex_build, cortex_simulate, cortex_spikes and cortex_free every step"},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if world == 1 and not args.no_forms:
        line["forms"] = {}
        for key, name, kw, n_steps in FORMS:
            line["forms"][key] = _form(cortex, W, name, kw, args, stream, peak, peak_kind,
                                       n_steps or args.form_steps)
        line["forms"]["deliver_only"] = _deliver_form(cortex, W, args, stream, peak, peak_kind)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _cpu_baseline(args):
    """The oracle on the host cores: target-partitioned over all of them (bitwise equal to the
    single-threaded oracle), and the same parts stepped by one thread, on bounded samples."""
    cores = os.cpu_count() or 1
    name = _config(args.config)["name"]
    try:
        res = run_oracle(args.config, cores, [(args.cpu_sample_steps, cores), (args.cpu_single_steps, 1)],
                         args.cpu_timeout)
    except Exception as ex:  # noqa: BLE001
        return {"value": None, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": f"not finished: {ex!r}"}
    (ev_m, s_m, n_m, _), (ev_1, s_1, n_1, _) = res["samples"]
    return {"value": ev_m / s_m, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{name}: oracle built in {res['build_s']:.0f} s (untimed, {cores} target ranges), then "
                      f"{n_m} simulation steps on {cores} threads; single-core figure: the next {n_1} steps on 1 thread",
            "single_core_value": ev_1 / s_1, "rtf": s_m / (n_m * 1e-4), **host_info()}


# (form key, configuration, options, simulation steps timed: None = --form-steps)
FORMS = [
    ("fp32_n112k", "c1", {}, None),
    ("bf16", "c3", {}, None),
    ("batched", "c4", {}, 5000),
    ("fp32_deep_delay_ordered", "c2", {"delivery": 1}, 1000),
    ("bf16_delay_ordered", "c3", {"delivery": 1}, None),
]

# ncu DRAM records per (configuration, delivery): bytes per event captured at full size (profiles/),
# valid while the kernel's code is the one captured
TRAFFIC_RECORDS = {("c1", 0): "k_step_c1_traffic.json", ("c2", 0): "k_step_c2_traffic.json",
                   ("c3", 0): "k_step_c3_traffic.json", ("c4", 0): "k_step_c4_traffic.json",
                   ("c3", 1): "k_dstep_c3_traffic.json", ("c2", 1): "k_dstep_c2_traffic.json"}


def _form(cortex, W, name, kw, args, stream, peak, peak_kind, n_steps):
    """events/s, RTF and kernel roofline of another configuration on the same GPU.  One untimed
    launch, then n_steps simulation steps, with the clocks sampled meanwhile."""
    cfg = W.CONFIGS[name]
    plan = None
    base = cortex.make_options(steps_per_launch=args.steps_per_launch, **kw)
    if name == "c4":
        specs, seeds = W.batch_specs()
        best, tune_ms, n_tried = cortex.autotune(specs, seeds, base, trial_steps=args.steps_per_launch, stream=stream)
        plan = {"autotuned": True, "warps_per_block": best.warps_per_block, "balance": best.balance,
                "candidates": n_tried, "trial_ms_per_step": tune_ms}
        net = cortex.Network(specs, seeds, best, stream=stream)
        bpe = BYTES_PER_EVENT[0]
    else:
        net = cortex.Network(cfg["spec"], cfg["seed"], base, stream=stream)
        bpe = BYTES_PER_EVENT[cfg["spec"].weight_dtype]
    st0 = net.stats()
    net.simulate(args.steps_per_launch)
    e0 = net.stats()["events"]
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))).start()
    clocks.mark_start()
    t0 = time.perf_counter()
    net.simulate(n_steps)
    wall = time.perf_counter() - t0
    clocks.mark_end()
    clk = clocks.stop()
    st = net.stats()
    ev = st["events"] - e0
    ms = st["simulate_ms"]
    launches = max(1, -(-n_steps // args.steps_per_launch))
    achieved = ev * bpe / (ms * 1e-3) / 1e9
    sim_s = n_steps * 0.1e-3
    delivery = kw.get("delivery", 0)
    out = {"workload": cfg["name"], "value": ev / (ms * 1e-3), "unit": UNIT, "rtf": (ms * 1e-3) / sim_s,
           "sim_steps": n_steps, "wall_value": ev / wall, "n_nets": st0["n_nets"],
           "neurons": st0["n_neurons"], "synapses": st0["n_synapses"], "build_ms": st0["build_ms"],
           "blocks": st0["n_blocks"], "threads_per_block": st0["threads_per_block"],
           "ring_in_smem": st0["ring_in_smem"], "spikes_per_round": st0["spikes_per_round"],
           "smem_bytes": st0["smem_bytes"], "delivery": "delay" if delivery == 1 else "ring",
           "exact_fold": st0["exact_fold"], "helper_warp": st0.get("helper_warp"), "dtype": "bf16" if bpe == 5 else "f32",
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "peak_kind": peak_kind, "bytes_per_event": bpe,
                        "kernel": "k_dstep (persistent, delay-ordered)" if delivery == 1 else "k_step (persistent)",
                        "launch_ms": ms / launches,
                        "traffic": _traffic(ev / launches, TRAFFIC_RECORDS.get((name, delivery)))},
           "clocks": clk}
    if plan is not None:
        out["plan"] = plan
    net.close()
    return out


def _deliver_record(config: str, spikes: int) -> str:
    """profiles/ record of the delivery kernel alone on `spikes` sources of a configuration."""
    return f"k_step_deliver_{config}_s{spikes}_traffic.json"


def _deliver_form(cortex, W, args, stream, peak, peak_kind):
    """The ring delivery kernel alone (cortex_deliver, one launch per repetition) on a fixed set of
    spiking sources (default: 10,000 of the 112,500-neuron network), repeated long enough for the
    clock samples."""
    import numpy as np
    cfg = W.CONFIGS[args.deliver_config]
    spec = cfg["spec"]
    with cortex.Network(spec, cfg["seed"], cortex.make_options(), stream=stream) as net:
        rng = np.random.default_rng(1)
        ids = np.unique(rng.choice(spec.n, size=min(args.spikes, spec.n), replace=False))
        net.deliver(ids, t_emit=0, reps=3)
        clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))).start()
        clocks.mark_start()
        ms, ev = net.deliver(ids, t_emit=0, reps=args.deliver_reps)
        clocks.mark_end()
        clk = clocks.stop()
    bpe = BYTES_PER_EVENT[spec.weight_dtype]
    achieved = ev * bpe / (ms * 1e-3) / 1e9
    return {"workload": cfg["name"], "value": ev / (ms * 1e-3), "unit": UNIT, "spikes_per_launch": int(len(ids)),
            "events_per_launch": ev, "launch_ms": ms, "reps": args.deliver_reps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "bytes_per_event": bpe, "kernel": "k_step (delivery phase)",
                         "traffic": _traffic(ev, _deliver_record(args.deliver_config, len(ids)))},
            "clocks": clk}


def code_digest(texts) -> str:
    """sha256 of C/C++/CUDA sources with comments removed and blank space collapsed (string
    literals kept as written): it changes when the code does, not when a comment does."""
    import hashlib
    import re
    tok = re.compile(r'"(?:\\.|[^"\\])*"|//[^\n]*|/\*.*?\*/', re.S)
    h = hashlib.sha256()
    for text in texts:
        text = tok.sub(lambda m: m.group(0) if m.group(0).startswith('"') else " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


KERNEL_SOURCES = {"k_step": ("step.cu", "step_common.cuh", "cortex_internal.cuh"),
                  "k_dstep": ("step_delay.cu", "step_common.cuh", "cortex_internal.cuh")}


def kernel_digest(kernel: str = "k_step") -> str:
    """code_digest of a step kernel's sources."""
    texts = []
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2406_03762_gb300", "csrc", name)) as g:
            texts.append(g.read())
    return code_digest(texts)


def _traffic(events_per_launch, record):
    """DRAM bytes per launch from a committed ncu record (profiles/<record>: bytes per synaptic event
    of the same workload at full size), scaled by the launch's events, if the kernel's code is
    unchanged since the capture; else None."""
    if record is None:
        return None
    path = os.path.join(ROOT, "profiles", record)
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("kernel_code_sha256") != kernel_digest(d.get("kernel_name", "k_step")):
            return None
        return d["dram_bytes_per_event"] * events_per_launch
    except Exception:
        return None


def deliver_arm(args):
    """Delivery kernel alone (split phase) on a fixed set of spiking sources."""
    import torch
    from paper_2406_03762_gb300 import cortex
    from paper_2406_03762_gb300 import workloads as W
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cortex.load()
    peak, peak_kind = _peaks()
    line = _deliver_form(cortex, W, args, torch.cuda.Stream(), peak, peak_kind)
    line.update({"metric": "delivery events/s", "n_gpus": 1, "higher_is_better": True})
    print(json.dumps(line), flush=True)
    return 0


def _config(name):
    from paper_2406_03762_gb300 import workloads as W
    if name in W.CONFIGS:
        return W.CONFIGS[name]
    return W.PROFILE[name]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=HEADLINE)
    ap.add_argument("--delivery", type=int, default=0, help="0: ring, 1: delay-ordered")
    ap.add_argument("--sim-steps", type=int, default=10000)
    ap.add_argument("--steps-per-launch", type=int, default=1000)
    ap.add_argument("--cpu-sample-steps", type=int, default=2000)
    ap.add_argument("--cpu-single-steps", type=int, default=200)
    ap.add_argument("--cpu-timeout", type=float, default=900.0)
    ap.add_argument("--ref-sample-steps", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="simulate", choices=["simulate", "deliver"])
    ap.add_argument("--spikes", type=int, default=10000, help="--mode deliver: spiking sources per launch")
    ap.add_argument("--deliver-config", default="c1", choices=["c1", "c2", "c3"],
                    help="--mode deliver: the network whose connectivity is read")
    ap.add_argument("--deliver-reps", type=int, default=300)
    ap.add_argument("--warps", type=int, default=0, help="warps per block (0: library default)")
    ap.add_argument("--no-forms", action="store_true", help="skip the other configurations")
    ap.add_argument("--form-steps", type=int, default=3000, help="simulation steps timed per form")
    args = ap.parse_args()
    if args.mode == "deliver":
        return deliver_arm(args)
    if args.impl == "reference":
        return reference_arm(args)
    return our_arm(args)


if __name__ == "__main__":
    sys.exit(main())
