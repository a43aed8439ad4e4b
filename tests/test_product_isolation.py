"""The product package never imports the oracle (no GPU).  The oracle is test infrastructure; the
library's path must stand on its own kernels.  Checked twice: statically (no import statement in
any module of the package names the oracle) and dynamically (importing every module of the package
in a fresh interpreter leaves no oracle module in sys.modules)."""
import ast
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2404_16245_gb300")


def _modules():
    for dirpath, dirnames, filenames in os.walk(PKG):
        dirnames[:] = [d for d in dirnames if not d.startswith(("_", "."))]
        for fn in sorted(filenames):
            if fn.endswith(".py"):
                yield os.path.join(dirpath, fn)


def test_no_module_of_the_package_imports_the_oracle():
    offenders = []
    for path in _modules():
        tree = ast.parse(open(path).read(), filename=path)
        for node in ast.walk(tree):
            names = []
            if isinstance(node, ast.Import):
                names = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom) and node.level == 0 and node.module:
                names = [node.module]
            offenders += [(os.path.relpath(path, ROOT), n) for n in names if n == "oracle" or n.startswith("oracle.")]
    assert not offenders, offenders


def test_importing_the_package_loads_no_oracle_module():
    mods = []
    for path in _modules():
        rel = os.path.relpath(path, ROOT)[:-3].replace(os.sep, ".")
        if rel.endswith("__init__"):
            rel = rel[: -len(".__init__")]
        mods.append(rel)
    code = ("import importlib, sys\n"
            f"mods = {mods!r}\n"
            "for m in mods:\n"
            "    try:\n"
            "        importlib.import_module(m)\n"
            "    except ImportError as e:\n"
            "        if 'libshgo.so is not built' not in str(e):\n"
            "            raise\n"
            "bad = [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]\n"
            "assert not bad, bad\n"
            "print('isolated', len(mods))\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "isolated" in r.stdout
