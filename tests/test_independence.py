"""The oracle and the CUDA path share no code: nothing under oracle/ imports
the library package, and the library package never imports the oracle (only
tests/, __graft_entry__.smoke() and bench.py's CPU legs may)."""

import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_1104_4475_gb300"


def _imports(path):
    """(module names imported, enclosing function name or None) of a file."""
    tree = ast.parse(open(path).read(), filename=path)
    out = []

    def visit(node, func):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else func
            if isinstance(child, ast.Import):
                out.extend((a.name, f) for a in child.names)
            elif isinstance(child, ast.ImportFrom):
                mod = child.module or ""
                out.append(("." * child.level + mod, f))
            visit(child, f)

    visit(tree, None)
    return out


def _py_files(folder):
    for dirpath, _, files in os.walk(os.path.join(ROOT, folder)):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(dirpath, f)


def test_oracle_imports_nothing_from_the_library():
    for path in _py_files("oracle"):
        for mod, _ in _imports(path):
            assert not mod.startswith(PKG) and "tqr" not in mod, (path, mod)


def test_library_never_imports_the_oracle():
    for path in _py_files(PKG):
        for mod, _ in _imports(path):
            assert not mod.split(".")[0] == "oracle", (path, mod)


def test_entry_points_use_the_oracle_only_where_allowed():
    allowed = {"__graft_entry__.py": {"smoke"}, "bench.py": {"oracle_sample"}}
    for name, funcs in allowed.items():
        for mod, func in _imports(os.path.join(ROOT, name)):
            if mod.split(".")[0] == "oracle":
                assert func in funcs, (name, func)


def test_library_sources_do_not_include_oracle_code():
    csrc = os.path.join(ROOT, PKG, "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in text.lower() or f.endswith(".md"), f
