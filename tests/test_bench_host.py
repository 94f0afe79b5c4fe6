"""Host-side pieces of the benchmark that need no GPU: the digest that ties the committed DRAM
traffic record to the kernel code it was measured on."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

SRC = '''// header comment
#include "x.h"
/* block
   comment */
__global__ void k(float* p) {  // trailing
  const char* s = "a // not a comment /* nor this */";
  p[0] += 1.0f;
}
'''


def test_digest_ignores_comments_and_blank_space():
    d = bench.code_digest([SRC])
    recommented = SRC.replace("// trailing", "// another remark").replace("header comment", "x")
    reflowed = SRC.replace("  p[0] += 1.0f;", "\n\n    p[0]   +=   1.0f;")
    assert bench.code_digest([recommented]) == d
    assert bench.code_digest([reflowed]) == d


def test_digest_sees_every_code_change():
    d = bench.code_digest([SRC])
    for edit in (("+= 1.0f", "+= 2.0f"), ("p[0]", "p[1]"), ('"a // not', '"b // not'), ("#include", "#define Y\n#include")):
        assert bench.code_digest([SRC.replace(*edit)]) != d, edit


def test_traffic_is_reported_only_for_the_measured_kernel():
    """The bench scales a committed record's DRAM bytes per event while the record's digest is the
    current code of the kernel it names, and reports null otherwise (or when there is no record)."""
    found = 0
    deliver = [bench._deliver_record(c, s) for c in ("c1", "c2", "c3") for s in (1000, 10000)]
    assert bench._deliver_record("c1", 10000) == "k_step_deliver_c1_s10000_traffic.json"
    for name in sorted(set(bench.TRAFFIC_RECORDS.values()) | set(deliver)):
        path = os.path.join(ROOT, "profiles", name)
        if not os.path.exists(path):
            assert bench._traffic(1e6, name) is None
            continue
        found += 1
        with open(path) as f:
            rec = json.load(f)
        assert 3.0 < rec["dram_bytes_per_event"] < 60.0
        if rec["kernel_code_sha256"] == bench.kernel_digest(rec.get("kernel_name", "k_step")):
            assert bench._traffic(1e6, name) == rec["dram_bytes_per_event"] * 1e6
        else:
            assert bench._traffic(1e6, name) is None
    assert bench._traffic(1e6, None) is None


def test_both_arms_name_the_same_workload():
    """The reference arm and ours put the same workload description in "config"."""
    from paper_2406_03762_gb300 import workloads as W
    c = bench.workload_config(W.CONFIGS[bench.HEADLINE])
    assert c["workload"] == W.CONFIGS["c2"]["name"] and c["synapses"] == 500000 * 5000
    assert c["d_min"] == 5 and c["d_max"] == 40 and c["weights"] == "f32"


class _FakeNet:
    """Stands in for cortex.Network: counts steps and reports fixed per-step events and time."""

    def __init__(self, *a, **k):
        self.steps, self.last = 0, 0

    def stats(self):
        return {"events": 5_818_217 * self.steps, "simulate_ms": 0.0605 * self.last, "n_nets": 1,
                "n_neurons": 1_000_000, "n_synapses": 11_250_000_000, "build_ms": 1.0, "n_blocks": 152,
                "ring_in_smem": 0, "spikes_per_round": 26, "smem_bytes": 230_272, "threads_per_block": 448,
                "exact_fold": 1}

    def simulate(self, n):
        self.steps += n
        self.last = n

    def close(self):
        pass


class _FakeCortex:
    Network = _FakeNet

    @staticmethod
    def make_options(**kw):
        return kw


def test_bench_form_line_without_gpu():
    """The BF16 form's dictionary builds (including its traffic lookup) with a stand-in library."""
    import types
    from paper_2406_03762_gb300 import workloads as W
    args = types.SimpleNamespace(steps_per_launch=1000, form_steps=2000)
    out = bench._form(_FakeCortex, W, "c3", {}, args, None, 6785.2, "measured", 2000)
    r = out["roofline"]
    assert out["dtype"] == "bf16" and abs(out["rtf"] - 0.605) < 1e-9
    assert abs(r["achieved"] - 5_818_217 * 1000 * 5 / 0.0605e-3 / 1e9 / 1000) < 1e-6 * r["achieved"]
    assert out["delivery"] == "ring" and out["exact_fold"] == 1


def test_batch_workload_is_described_without_a_single_spec():
    """The 64-network batch has no single network spec: the bench names it by its sizes, summed
    over the batch, and every form's configuration has a traffic record at full size."""
    from paper_2406_03762_gb300 import workloads as W
    cfg = W.CONFIGS["c4"]
    specs, seeds = W.batch_specs()
    c = bench.workload_config(cfg)
    assert c["workload"] == cfg["name"] and c["n_nets"] == len(specs) == len(seeds) == 64
    assert c["n_neurons"] == sum(s.n for s in specs)
    assert c["synapses"] == sum(s.n * s.k for s in specs)
    for key, name, kw, _ in bench.FORMS:
        assert (name, kw.get("delivery", 0)) in bench.TRAFFIC_RECORDS, key
