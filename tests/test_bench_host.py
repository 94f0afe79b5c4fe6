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
    """The bench scales the committed record's DRAM bytes per event while the record's digest is
    the current kernel code's, and reports null otherwise."""
    with open(os.path.join(ROOT, "profiles", "k_step_traffic.json")) as f:
        rec = json.load(f)
    assert 6.0 < rec["dram_bytes_per_event"] < 8.0  # 6 stored bytes per synapse plus headers
    if rec["kernel_code_sha256"] == bench.kernel_digest():
        assert bench._traffic(1e6, None) == rec["dram_bytes_per_event"] * 1e6
    else:
        assert bench._traffic(1e6, None) is None
