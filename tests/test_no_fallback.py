"""The product path has no CPU fallback: the binding refuses to import
without the built CUDA library, and no module of the package imports the
oracle or executes anything under oracle/."""

import ast
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1611_08494_gb300")


def test_binding_refuses_to_import_without_the_library(tmp_path):
    pkg = tmp_path / "paper_1611_08494_gb300"
    pkg.mkdir()
    (pkg / "__init__.py").write_text("")
    shutil.copy(os.path.join(PKG, "xm.py"), pkg / "xm.py")  # no _lib/ beside it
    code = ("import sys; sys.path.insert(0, %r)\n"
            "try:\n"
            "    from paper_1611_08494_gb300 import xm\n"
            "except ImportError as e:\n"
            "    print('refused:', e)\n"
            "else:\n"
            "    print('imported')\n") % str(tmp_path)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.startswith("refused:") and "no CPU fallback" in out.stdout


def _imports(path):
    tree = ast.parse(open(path).read())
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module:
            names.add(node.module.split(".")[0])
        elif isinstance(node, ast.Call) and getattr(node.func, "id", "") == "__import__":
            names.add("__import__")
    return names


def test_package_never_imports_the_oracle():
    for f in sorted(os.listdir(PKG)):
        if f.endswith(".py"):
            names = _imports(os.path.join(PKG, f))
            assert "oracle" not in names, f
            assert "__import__" not in names, f
            src = open(os.path.join(PKG, f)).read()
            assert "oracle/" not in src and "xm_oracle" not in src, f
