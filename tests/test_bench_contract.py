"""Host-side pieces of bench.py that its JSON line depends on: the defaults
(one GPU, at least three warm-up steps), the measured peak it divides by, and
the DRAM traffic record, which must describe the kernel sources in the tree
(bench.py reports `traffic` only then)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_defaults(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse_args()
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1 and a.impl == "ours" and a.precision == "fp64"


def test_peak_is_the_measured_copy_bandwidth():
    peak, kind = bench.measured_peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            assert (peak, kind) == (float(json.load(f)["hbm_gbs"]), "measured")
    else:
        assert kind == "fallback"


def test_traffic_is_reported_only_for_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    """bench.py reports a kernel's DRAM traffic only while the step kernels'
    code hashes to the value recorded with it (the ncu capture was taken on
    those sources); on other sources, or another workload, it reports null."""
    workload = "zipf-lp m=1e6 n=3e6 nnz~3e7 FP64"
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    sha = bench.kernel_source_sha()
    for kernel in ("primal half-step (FP64)", "k_dual_step"):
        e = rec.get(kernel)
        t = bench.profiled_traffic(kernel, workload)
        if e and e["source_sha"] == sha and e["workload"] == workload:
            assert t == e["dram_bytes_per_launch"] and 0.9e8 < t < 2e9
        else:
            assert t is None
        assert bench.profiled_traffic(kernel, "another workload") is None
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "0" * 16)
    assert bench.profiled_traffic("k_dual_step", workload) is None


def test_code_hash_ignores_comments_and_layout_only():
    a = "int f(int x) { return x + 1; } // one\n"
    b = "/* doc */\nint f(int x)  {\n  return x + 1;  // another\n}\n"
    c = "int f(int x) { return x + 2; }"
    assert bench.code_tokens(a) == bench.code_tokens(b) != bench.code_tokens(c)
    assert bench.code_tokens('s = "/* kept */ // kept"; t = \'/\';') == 's = "/* kept */ // kept"; t = \'/\';'
