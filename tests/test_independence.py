"""The oracle and the CUDA path share no code (CPU, static): the product package never
imports or includes anything under oracle/, the oracle never imports the product package
nor includes its headers, and the only module both sides are fed from is the input
generator `media`, which importing does not load the CUDA library."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1303_2470_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(top, exts):
    for d, _, names in os.walk(top):
        if "__pycache__" in d or "_build" in d:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def _imports(path):
    mods = set()
    for node in ast.walk(ast.parse(open(path).read())):
        if isinstance(node, ast.Import):
            mods.update(a.name for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            mods.add(("." * node.level) + (node.module or ""))
    return mods


def _includes(path):
    return re.findall(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', open(path).read(), flags=re.M)


def test_product_never_imports_or_includes_the_oracle():
    for f in _files(PKG, (".py",)):
        for m in _imports(f):
            assert m.split(".")[0] != "oracle", f"{f} imports {m}"
    for f in _files(PKG, (".cu", ".cuh", ".h", ".c", ".cpp")):
        for inc in _includes(f):
            assert "oracle" not in inc, f"{f} includes {inc}"


def test_oracle_never_imports_or_includes_the_product():
    for f in _files(ORACLE, (".py",)):
        for m in _imports(f):
            assert not m.startswith("paper_1303_2470_gb300"), f"{f} imports {m}"
    for f in _files(ORACLE, (".c", ".h", ".cpp")):
        for inc in _includes(f):
            assert "csrc" not in inc and "mp.h" not in inc and "surrogate.h" not in inc, f"{f} includes {inc}"


def test_input_generators_hold_no_library_import():
    # media.py feeds both sides: it may use numpy only, and importing the package does not
    # load libmp (only importing paper_1303_2470_gb300.mp does)
    mods = _imports(os.path.join(PKG, "media.py"))
    assert mods <= {"__future__", "numpy"}, mods
    init = _imports(os.path.join(PKG, "__init__.py"))
    assert not any(m.lstrip(".").startswith("mp") for m in init), init
