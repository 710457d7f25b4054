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


def test_traffic_record_matches_the_kernel_sources():
    """The record of the benchmarked half-steps was taken on these sources:
    after a change to the step kernels, capture it again (the command is in the
    FP64 step-kernel summary under profiles/)."""
    workload = "zipf-lp m=1e6 n=3e6 nnz~3e7 FP64"
    for kernel in ("primal half-step (FP64)", "k_dual_step"):
        t = bench.profiled_traffic(kernel, workload)
        assert t is not None, f"{kernel}: traffic record stale or missing"
        assert 0.9e8 < t < 2e9


def test_code_hash_ignores_comments_and_layout_only():
    a = "int f(int x) { return x + 1; } // one\n"
    b = "/* doc */\nint f(int x)  {\n  return x + 1;  // another\n}\n"
    c = "int f(int x) { return x + 2; }"
    assert bench.code_tokens(a) == bench.code_tokens(b) != bench.code_tokens(c)
    assert bench.code_tokens('s = "/* kept */ // kept"; t = \'/\';') == 's = "/* kept */ // kept"; t = \'/\';'
