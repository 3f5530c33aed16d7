"""The oracle and the product path share no code: the package (binding, generators, CUDA
sources) never imports or includes the oracle, the oracle never imports the package's solver,
and bench.py reaches the oracle only from its CPU-baseline and reference-arm functions."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_0901_1110_gb300")


def _imports(path):
    tree = ast.parse(open(path).read())
    out = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out += [(a.name, node) for a in node.names]
        elif isinstance(node, ast.ImportFrom) and node.module:
            out.append((node.module, node))
    return tree, out


def test_package_never_imports_the_oracle():
    for name in os.listdir(PKG):
        if name.endswith(".py"):
            _, imps = _imports(os.path.join(PKG, name))
            assert not [m for m, _ in imps if m.split(".")[0] == "oracle"], name
    csrc = os.path.join(PKG, "csrc")
    for name in os.listdir(csrc):
        text = open(os.path.join(csrc, name)).read()
        assert not re.search(r"#\s*include\s*[<\"][^>\"]*oracle", text), name


def test_oracle_never_imports_the_solver():
    odir = os.path.join(ROOT, "oracle")
    for name in os.listdir(odir):
        if name.endswith(".py"):
            _, imps = _imports(os.path.join(odir, name))
            bad = [m for m, _ in imps if m.split(".")[0] in ("paper_0901_1110_gb300", "bench",
                                                            "torch", "ctypes")]
            assert not bad, (name, bad)


def test_input_generators_import_neither_side():
    _, imps = _imports(os.path.join(PKG, "inputs.py"))
    assert {m.split(".")[0] for m, _ in imps} <= {"dataclasses", "numpy"}


def test_bench_reaches_the_oracle_only_from_its_cpu_legs():
    tree, _ = _imports(os.path.join(ROOT, "bench.py"))
    allowed = {"_oracle_subbox", "reference_arm", "cpu_baseline_sample"}
    for fn in [n for n in tree.body if isinstance(n, ast.FunctionDef)]:
        for node in ast.walk(fn):
            mods = []
            if isinstance(node, ast.Import):
                mods = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom) and node.module:
                mods = [node.module]
            if any(m.split(".")[0] == "oracle" for m in mods):
                assert fn.name in allowed, fn.name
    top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
    for node in top:
        names = [a.name for a in node.names] if isinstance(node, ast.Import) else [node.module]
        assert not any(str(m).split(".")[0] == "oracle" for m in names)
