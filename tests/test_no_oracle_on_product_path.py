"""The product path never routes through the oracle: the library package
imports nothing from oracle/, and bench.py touches the oracle only in its
reference arm, in the oracle's child process and in the branches guarded by
`not args.no_cpu_baseline` (the CPU baseline and parity blocks)."""

import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_HELPERS = {"oracle_data", "oracle_slice_baseline", "run_oracle_sample"}
ORACLE_FUNCTIONS = {"bench_reference", "oracle_sample_main"} | ORACLE_HELPERS


def test_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1705_07497_gb300")
    for dirpath, _, files in os.walk(pkg):
        for name in files:
            if name.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                text = open(os.path.join(dirpath, name)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", text, re.M), name
                assert "oracle/" not in text.replace("oracle/ ", ""), name


def _guarded(test):
    """True for `not args.no_cpu_baseline` (possibly inside an `and`)."""
    src = ast.unparse(test)
    return "not args.no_cpu_baseline" in src


def _violations(node, fn, guarded, out):
    for child in ast.iter_child_nodes(node):
        g = guarded
        if isinstance(child, ast.If) and _guarded(child.test):
            for stmt in child.body:
                _violations(stmt, fn, True, out)
            for stmt in child.orelse:
                _violations(stmt, fn, guarded, out)
            continue
        if isinstance(child, ast.ImportFrom) and child.module and child.module.split(".")[0] == "oracle":
            if not g and fn not in ORACLE_FUNCTIONS:
                out.append((fn, child.lineno, "import"))
        if isinstance(child, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in child.names):
            if not g and fn not in ORACLE_FUNCTIONS:
                out.append((fn, child.lineno, "import"))
        if isinstance(child, ast.Call) and isinstance(child.func, ast.Name) and child.func.id in ORACLE_HELPERS:
            if not g and fn not in ORACLE_FUNCTIONS:
                out.append((fn, child.lineno, child.func.id))
        _violations(child, fn, g, out)


def test_bench_touches_the_oracle_only_in_its_oracle_legs():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    out = []
    for node in tree.body:
        if isinstance(node, (ast.Import, ast.ImportFrom)):
            names = [node.module or ""] if isinstance(node, ast.ImportFrom) else [a.name for a in node.names]
            assert not any(n.split(".")[0] == "oracle" for n in names), "module-level oracle import"
        if isinstance(node, ast.FunctionDef):
            _violations(node, node.name, False, out)
    assert out == [], out
    # and the guarded legs exist: the check is not vacuous
    text = open(os.path.join(ROOT, "bench.py")).read()
    assert text.count("not args.no_cpu_baseline") >= 5


def test_oracle_does_not_import_the_library():
    """The other direction: nothing under oracle/ imports the package or
    includes its CUDA sources or headers (the two share no code; the oracle
    takes its inputs as arguments)."""
    odir = os.path.join(ROOT, "oracle")
    for name in os.listdir(odir):
        if name.endswith((".py", ".c", ".h")):
            text = open(os.path.join(odir, name)).read()
            assert "paper_1705_07497_gb300" not in text, name
            assert not re.search(r'#include\s+"', text), name
