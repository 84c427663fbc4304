"""The oracle is test infrastructure: no module of the package imports it, and
the benchmark driver imports it only inside its host-baseline and reference
functions; the package's binding refuses to run without the CUDA library
rather than fall back to anything else."""
import ast
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1509_08391_gb300")
ALLOWED_IN_BENCH = {"cpu_baseline", "run_reference", "cpu_baseline_configs"}


def _oracle_imports(tree):
    """(enclosing function name or None, line) of every import of oracle."""
    found = []

    def visit(node, func):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else func
            if isinstance(child, ast.Import):
                if any(a.name == "oracle" or a.name.startswith("oracle.") for a in child.names):
                    found.append((func, child.lineno))
            elif isinstance(child, ast.ImportFrom):
                if child.module and (child.module == "oracle" or child.module.startswith("oracle.")):
                    found.append((func, child.lineno))
            visit(child, f)

    visit(tree, None)
    return found


def test_package_never_imports_the_oracle():
    for name in sorted(os.listdir(PKG)):
        if name.endswith(".py"):
            tree = ast.parse(open(os.path.join(PKG, name)).read())
            assert _oracle_imports(tree) == [], name


def test_bench_imports_the_oracle_only_in_its_baseline_legs():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    uses = _oracle_imports(tree)
    assert uses, "the cpu_baseline leg times the oracle"
    for func, line in uses:
        assert func in ALLOWED_IN_BENCH, (func, line)


def test_binding_raises_without_the_library(tmp_path):
    from paper_1509_08391_gb300 import llr
    saved = llr._lib
    llr._lib = None
    try:
        with pytest.raises(RuntimeError, match="missing"):
            llr.load(str(tmp_path / "absent.so"))
    finally:
        llr._lib = saved
