"""The oracle and the CUDA path share no code, and the product has no CPU
fallback (checked on the CPU, no GPU needed):

- nothing under oracle/ imports or names the product package or its sources;
- nothing in the product package (binding, build script, CUDA sources, header)
  imports or names the oracle;
- workloads/ (the seeded generators both sides use) imports neither;
- importing the binding from a copy without libascg.so raises ImportError.
"""
import ast
import glob
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_1701_03989_gb300"


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module:
            names.add(node.module.split(".")[0])
    return names


def test_oracle_does_not_use_the_product():
    files = glob.glob(os.path.join(ROOT, "oracle", "*.py"))
    assert files
    for f in files:
        assert not (_imports(f) & {PKG, "bench", "__graft_entry__"}), f
        text = open(f).read()
        assert PKG not in text and "libascg" not in text and "csrc" not in text, f


def test_product_does_not_use_the_oracle():
    files = (glob.glob(os.path.join(ROOT, PKG, "*.py")) + glob.glob(os.path.join(ROOT, PKG, "csrc", "*")) +
             glob.glob(os.path.join(ROOT, "include", "*.h")))
    assert files
    for f in files:
        if f.endswith(".py"):
            assert "oracle" not in _imports(f), f
        text = open(f, errors="replace").read()
        assert "ascg_oracle" not in text and "oracle/" not in text, f


def test_workloads_import_neither_side():
    for f in glob.glob(os.path.join(ROOT, "workloads", "*.py")):
        assert not (_imports(f) & {PKG, "oracle"}), f


def test_binding_without_library_raises(tmp_path):
    pkg = tmp_path / PKG
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, PKG, "__init__.py"), pkg / "__init__.py")
    code = f"import sys; sys.path.insert(0, {str(tmp_path)!r}); import {PKG}"
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=str(tmp_path))
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "no CPU fallback" in r.stderr
