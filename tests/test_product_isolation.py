"""The product path never reaches the oracle.

The oracle is test infrastructure: the package (binding, autograd wrapper, build script and CUDA
sources) neither imports nor includes it, importing the package leaves it unloaded, and bench.py
imports it only inside its CPU-baseline leg (`oracle_rate`, used by the CPU baseline, the accuracy
rows and the reference arm).
"""

import ast
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1004_5076_gb300")


def _package_files():
    for d, dirs, files in os.walk(PKG):
        dirs[:] = [x for x in dirs if x not in ("_build", "__pycache__")]
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                yield os.path.join(d, f)


def test_package_sources_do_not_reference_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b|#\s*include\s*[<\"][^>\"]*oracle)", re.M)
    hits = [p for p in _package_files() if pat.search(open(p, encoding="utf-8").read())]
    assert not hits, hits


def test_importing_the_package_leaves_the_oracle_unloaded():
    code = ("import sys; sys.path.insert(0, %r); import paper_1004_5076_gb300, paper_1004_5076_gb300.autograd; "
            "bad = [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]; "
            "assert not bad, bad" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]


def test_bench_imports_the_oracle_only_in_its_cpu_leg():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py"), encoding="utf-8").read())
    where = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            name = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else fn
            if isinstance(child, ast.ImportFrom) and (child.module or "").split(".")[0] == "oracle":
                where.append(fn)
            if isinstance(child, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in child.names):
                where.append(fn)
            visit(child, name)

    visit(tree, None)
    # the CPU baselines: O1 on every host core (pool workers and driver) and O2 on one core
    assert where and set(where) <= {"_o1_init", "_o1_edge", "oracle_rate_allcores", "o2_rate"}, where
