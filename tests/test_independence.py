"""The oracle and the CUDA path share no code: no module of the product
package (Python or CUDA/C++) refers to the oracle, and no oracle module imports
the product package.  The seeded input generators (paper_1401_6749_gb300/synth.py)
hold no arithmetic of the method and import nothing but numpy and torch (whose
matrix_exp makes the seeded SU(3) links)."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1401_6749_gb300")


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            mods.add(node.module.split(".")[0])
    return mods


def _files(top, exts):
    for d, _, names in os.walk(top):
        if "__pycache__" in d or "_build" in d:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def test_product_package_does_not_use_the_oracle():
    for f in _files(PKG, (".py",)):
        assert "oracle" not in _imports(f), f
    for f in _files(os.path.join(PKG, "csrc"), (".cu", ".cuh", ".h", ".cpp")):
        assert not re.search(r"#\s*include\s*[<\"][^>\"]*oracle", open(f).read()), f


def test_oracle_does_not_import_the_product():
    for f in _files(os.path.join(ROOT, "oracle"), (".py",)):
        assert "paper_1401_6749_gb300" not in _imports(f), f


def test_input_generators_import_only_numpy_and_torch():
    assert _imports(os.path.join(PKG, "synth.py")) <= {"numpy", "torch"}
