"""The product path has no CPU fallback: the package refuses to import
without its compiled library, and nothing outside the test infrastructure
(tests/, the smoke check, the bench's CPU-baseline and reference legs)
imports the oracle; the oracle and the inputs module import nothing of the
library."""
import ast
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1712_06121_gb300")


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    out = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out += [(a.name, node) for a in node.names]
        elif isinstance(node, ast.ImportFrom) and node.module:
            out.append((node.module, node))
    return tree, out


def _py_files(d):
    for base, _, files in os.walk(d):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def test_package_refuses_to_import_without_its_library(tmp_path):
    dst = tmp_path / "paper_1712_06121_gb300"
    dst.mkdir()
    shutil.copy(os.path.join(PKG, "__init__.py"), dst / "__init__.py")
    r = subprocess.run([sys.executable, "-c", "import paper_1712_06121_gb300"], cwd=tmp_path,
                       capture_output=True, text=True)
    assert r.returncode != 0 and "ImportError" in r.stderr and "libcube.so is not built" in r.stderr


def test_library_package_and_inputs_never_import_the_oracle():
    for d in (PKG, os.path.join(ROOT, "synth")):
        for path in _py_files(d):
            for name, _ in _imports(path)[1]:
                assert not name.startswith("oracle"), (path, name)


def test_oracle_imports_nothing_of_the_library():
    for path in _py_files(os.path.join(ROOT, "oracle")):
        for name, _ in _imports(path)[1]:
            assert not name.startswith("paper_1712_06121_gb300") and not name.startswith("synth"), (path, name)


def test_oracle_imports_in_entry_points_are_confined():
    """bench.py and __graft_entry__.py import the oracle only inside the
    functions that time it (CPU baseline, reference arm) or check the smoke
    run against it, never at module level."""
    allowed = {"bench.py": {"oracle_state"}, "__graft_entry__.py": {"smoke"}}
    for fname, funcs in allowed.items():
        tree, _ = _imports(os.path.join(ROOT, fname))
        for node in tree.body:
            if isinstance(node, (ast.Import, ast.ImportFrom)):
                names = [a.name for a in node.names] if isinstance(node, ast.Import) else [node.module or ""]
                assert not any(n.startswith("oracle") for n in names), (fname, names)
        for node in ast.walk(tree):
            if isinstance(node, ast.FunctionDef):
                uses = [n for n, _ in _imports_in(node) if n.startswith("oracle")]
                if uses:
                    assert node.name in funcs, (fname, node.name)


def _imports_in(fn):
    out = []
    for node in ast.walk(fn):
        if isinstance(node, ast.Import):
            out += [(a.name, node) for a in node.names]
        elif isinstance(node, ast.ImportFrom) and node.module:
            out.append((node.module, node))
    return out
