"""The oracle and the CUDA path share no code. The product package never
imports the oracle; the oracle never imports the package or includes its
headers; the benchmark reaches the oracle only in its CPU-baseline and
reference legs, and the entry point only to build it and in the smoke check."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1303_5164_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _py_files(d):
    for dp, dn, fn in os.walk(d):
        dn[:] = [x for x in dn if not x.startswith(("_build", "__pycache__"))]
        for f in fn:
            if f.endswith(".py"):
                yield os.path.join(dp, f)


def _imports(path):
    tree = ast.parse(open(path).read())
    out = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out += [(a.name, node) for a in node.names]
        elif isinstance(node, ast.ImportFrom) and node.module:
            out.append((node.module, node))
    return tree, out


def test_product_never_imports_the_oracle():
    for p in _py_files(PKG):
        _, imps = _imports(p)
        assert not [m for m, _ in imps if m == "oracle" or m.startswith("oracle.")], p


def test_oracle_never_uses_the_product():
    for p in _py_files(ORACLE):
        _, imps = _imports(p)
        assert not [m for m, _ in imps if m.startswith("paper_1303_5164_gb300")], p
        txt = open(p).read()
        assert "csrc" not in txt and "kernelet.h" not in txt, p
    for f in os.listdir(ORACLE):
        if f.endswith((".c", ".h")):
            inc = re.findall(r'#include\s+[<"]([^>"]+)[>"]', open(os.path.join(ORACLE, f)).read())
            assert all(i in ("math.h", "stdint.h", "stdlib.h", "string.h", "stddef.h", "stdio.h") for i in inc), (f, inc)
    for p in _py_files(PKG):
        assert "oracle/" not in open(p).read(), p  # no path into the oracle either


def _functions_importing_oracle(path):
    tree, imps = _imports(path)
    owners = set()
    for fn in ast.walk(tree):
        if isinstance(fn, (ast.FunctionDef, ast.AsyncFunctionDef)):
            for node in ast.walk(fn):
                if isinstance(node, (ast.Import, ast.ImportFrom)):
                    mods = [a.name for a in node.names] if isinstance(node, ast.Import) else [node.module or ""]
                    if any(m == "oracle" or m.startswith("oracle.") for m in mods):
                        owners.add(fn.name)
    top = [m for m, node in imps if (m == "oracle" or m.startswith("oracle.")) and node in tree.body]
    return owners, top


def test_benchmark_and_entry_point_reach_the_oracle_only_where_allowed():
    owners, top = _functions_importing_oracle(os.path.join(ROOT, "bench.py"))
    assert not top and owners <= {"_oracle_one", "cpu_oracle_sample", "cpu_oracle_all_cores", "run_reference"}, owners
    owners, top = _functions_importing_oracle(os.path.join(ROOT, "__graft_entry__.py"))
    assert not top and owners <= {"build", "smoke"}, owners


def test_product_fails_loudly_without_its_library(tmp_path):
    # no fallback: a missing libkernelet.so raises instead of computing anything on the CPU
    import subprocess
    import sys
    code = ("import paper_1303_5164_gb300.kernelet as K\n"
            f"K.lib_path = lambda: {str(tmp_path / 'absent.so')!r}\n"
            "K._lib = None\n"
            "try:\n"
            "    K.lib()\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n"
            "    raise SystemExit(0)\n"
            "raise SystemExit(1)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert r.returncode == 0 and "no fallback" in r.stdout, r.stdout + r.stderr
