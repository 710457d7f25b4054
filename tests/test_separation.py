"""The oracle and the CUDA path share no code, and only test infrastructure
uses the oracle: the package never imports it, the oracle imports nothing from
the package (its inputs are passed in as arrays), and bench.py imports it only
inside the functions of its CPU-baseline and reference legs. Nothing committed
refers to the untracked working folder."""
import ast
import os
import pathlib
import re
import subprocess

ROOT = pathlib.Path(__file__).resolve().parent.parent
PKG = ROOT / "paper_2510_24429_b300"


def _imports(path: pathlib.Path, top_level_only: bool = False) -> set[str]:
    tree = ast.parse(path.read_text())
    nodes = tree.body if top_level_only else list(ast.walk(tree))
    out = set()
    for node in nodes:
        if isinstance(node, ast.Import):
            out.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            out.add(node.module.split(".")[0])
    return out


def test_package_never_imports_the_oracle():
    for f in PKG.rglob("*.py"):
        assert "oracle" not in _imports(f), f
    for f in list(PKG.rglob("*.cu")) + list(PKG.rglob("*.cuh")) + [ROOT / "include" / "pdhg.h"]:
        includes = re.findall(r'#include\s+"([^"]+)"', f.read_text())
        assert not any("oracle" in i for i in includes), (f, includes)


def test_oracle_imports_only_the_standard_library_numpy_and_scipy():
    allowed = {"__future__", "dataclasses", "math", "numpy", "scipy", "typing", "itertools", "functools"}
    for f in (ROOT / "oracle").rglob("*.py"):
        extra = _imports(f) - allowed
        assert not extra, (f, extra)
    assert not list((ROOT / "oracle").rglob("*.cu*")) and not list((ROOT / "oracle").rglob("*.h"))


def test_bench_imports_the_oracle_only_inside_its_cpu_legs():
    bench = ROOT / "bench.py"
    assert "oracle" not in _imports(bench, top_level_only=True)
    tree = ast.parse(bench.read_text())
    users = set()
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                if isinstance(node, ast.ImportFrom) and node.module and node.module.split(".")[0] == "oracle":
                    users.add(fn.name)
    assert users == {"oracle_seconds_per_iteration", "_oracle_replica", "run_reference"}, users


def test_nothing_committed_uses_the_working_folder():
    files = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True).stdout.split()
    if not files:  # not a git checkout
        files = [str(p.relative_to(ROOT)) for p in ROOT.rglob("*") if p.is_file() and "_work" not in p.parts]
    for rel in files:
        p = ROOT / rel
        if p.suffix not in (".py", ".cu", ".cuh", ".h", ".sh", ".txt", ".cfg", ".toml") or not p.exists():
            continue
        text = p.read_text(errors="replace")
        assert not re.search(r"(^|[\s'\"/(])_work/", text), rel
