"""The CUDA path and the oracle stay independent.

- Nothing in the package (binding, build script, CUDA sources) imports,
  includes or loads the oracle.
- Nothing in the oracle imports or loads the package or its header.
- The seeded input generators (workloads/) import neither.
- bench.py runs the oracle only in its CPU-baseline leg, its `--impl
  reference` arm, and the precision study of the FP32 path's error against
  the FP64 oracle; each imports it inside its own function, outside any
  timed region of the GPU path.
"""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2002_02211_gb300")
ORACLE = os.path.join(ROOT, "oracle")
WORKLOADS = os.path.join(ROOT, "workloads")

SOURCE_EXT = (".py", ".cu", ".cuh", ".h", ".c", ".cpp")


def _sources(top):
    for dirpath, dirnames, files in os.walk(top):
        dirnames[:] = [d for d in dirnames if d not in ("__pycache__", "_build")]
        for f in files:
            if f.endswith(SOURCE_EXT):
                yield os.path.join(dirpath, f)


def _hits(top, pattern):
    rx = re.compile(pattern)
    out = []
    for path in _sources(top):
        with open(path, errors="replace") as fh:
            for n, line in enumerate(fh, 1):
                if rx.search(line):
                    out.append(f"{os.path.relpath(path, ROOT)}:{n}: {line.strip()}")
    return out


def test_package_does_not_use_the_oracle():
    hits = _hits(PKG, r"^\s*(import\s+oracle|from\s+oracle\b)|#\s*include\s*[<\"].*oracle|liboracle|pic_oracle")
    assert not hits, hits


def test_oracle_does_not_use_the_package():
    hits = _hits(ORACLE, r"paper_2002_02211_gb300|libpic|#\s*include\s*[<\"]pic\.h|pic_kernels|pic_device")
    assert not hits, hits


def test_input_generators_import_neither():
    hits = _hits(WORKLOADS, r"^\s*(import|from)\s+(oracle|paper_2002_02211_gb300)\b")
    assert not hits, hits


def test_bench_runs_the_oracle_only_in_its_oracle_legs():
    allowed = {"cpu_sample", "cpu_baseline", "main_reference", "main_precision"}
    with open(os.path.join(ROOT, "bench.py")) as fh:
        tree = ast.parse(fh.read())
    found = set()

    def visit(node, func):
        for child in ast.iter_child_nodes(node):
            name = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else func
            if isinstance(child, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in child.names):
                found.add(func)
            if isinstance(child, ast.ImportFrom) and (child.module or "").split(".")[0] == "oracle":
                found.add(func)
            visit(child, name)

    visit(tree, None)
    assert None not in found, "bench.py imports the oracle at module level"
    assert found <= allowed, found - allowed
    assert {"cpu_baseline", "main_reference"} <= found
