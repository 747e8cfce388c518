"""The oracle and the CUDA path stay apart, and the product path has no fallback.

* Nothing in the product package imports the oracle, and the oracle imports nothing
  from the product package; the seeded generators (datagen) import neither.
* Without the built library the binding raises instead of computing anything.
"""
import ast
import glob
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_2602_04551_b300"


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            if node.level == 0 and node.module:
                names.add(node.module.split(".")[0])
    return names


def test_product_package_never_imports_the_oracle():
    files = glob.glob(os.path.join(ROOT, PKG, "**", "*.py"), recursive=True)
    assert files
    for f in files:
        assert "oracle" not in _imports(f), f
    for f in glob.glob(os.path.join(ROOT, PKG, "csrc", "*")):
        assert "oracle" not in open(f, errors="replace").read().lower(), f


def test_oracle_and_generators_never_import_the_product():
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.py")) + glob.glob(os.path.join(ROOT, "datagen", "*.py")):
        imp = _imports(f)
        assert PKG not in imp and "torch" not in imp, f
    for f in glob.glob(os.path.join(ROOT, "datagen", "*.py")):
        assert "oracle" not in _imports(f), f


def test_missing_library_fails_loudly(tmp_path):
    """A copy of the binding without libbnb.so raises on first use."""
    dst = tmp_path / PKG
    dst.mkdir()
    for f in glob.glob(os.path.join(ROOT, PKG, "*.py")):
        shutil.copy(f, dst)
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import %s as b\n"
            "try:\n"
            "    b.bnb_options_default()\n"
            "except ImportError as e:\n"
            "    print('raised', e)\n"
            "else:\n"
            "    print('no error')\n") % (str(tmp_path), PKG)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120,
                         cwd=str(tmp_path))
    assert out.stdout.startswith("raised"), out.stdout + out.stderr
    assert "not built" in out.stdout
