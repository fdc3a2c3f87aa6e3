"""Static checks of the boundaries between the library, the oracle and the
input generators:

* the library (paper_1607_01649_gb300/, Python and CUDA) never imports or
  includes the oracle or the input generators, and its Python binding does
  no linear algebra of its own (no CPU path besides the kernels);
* the oracle imports only numpy, math and its own modules (never the library,
  torch or the generators), so the two sides share no code;
* the generators import neither side;
* bench.py imports the oracle only inside its CPU legs, and
  __graft_entry__.py only inside smoke()."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1607_01649_gb300")


def _py_files(d):
    for dirpath, dirnames, files in os.walk(d):
        dirnames[:] = [x for x in dirnames if not x.startswith(("_build", "__pycache__"))]
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(dirpath, f)


def _imports(path):
    """(top-level module, enclosing function name or None) of every import."""
    tree = ast.parse(open(path).read())
    out = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            name = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else fn
            if isinstance(child, ast.Import):
                out.extend((a.name.split(".")[0], fn) for a in child.names)
            elif isinstance(child, ast.ImportFrom):
                out.append(("." if child.level else (child.module or "").split(".")[0], fn))
            visit(child, name)

    visit(tree, None)
    return out


def test_library_never_reaches_the_oracle_or_the_generators():
    for path in _py_files(PKG):
        mods = {m for m, _ in _imports(path)}
        assert not mods & {"oracle", "workloads", "scipy"}, path
        src = open(path).read()
        assert not re.search(r"linalg|\.svd\(|\.qr\(|cholesky|einsum|torch\.matmul|torch\.mm\b| @ ", src), path
    csrc = os.path.join(PKG, "csrc")
    for f in os.listdir(csrc):
        if f.endswith((".cu", ".cuh", ".h")):
            for inc in re.findall(r'#include\s+[<"]([^>"]+)[>"]', open(os.path.join(csrc, f)).read()):
                assert "oracle" not in inc and "workloads" not in inc, (f, inc)


def test_oracle_imports_only_numpy_math_and_itself():
    odir = os.path.join(ROOT, "oracle")
    for path in _py_files(odir):
        for mod, _ in _imports(path):
            assert mod in {".", "numpy", "math"}, (path, mod)


def test_generators_import_neither_side():
    for path in _py_files(os.path.join(ROOT, "workloads")):
        for mod, _ in _imports(path):
            assert mod not in {"oracle", "paper_1607_01649_gb300"}, (path, mod)


def test_oracle_only_in_cpu_legs_and_smoke():
    allowed = {
        "bench.py": {"oracle_sample", "oracle_full", "run_reference", "controller_oracle_solve", "nystrom_oracle_solve",
                     "batched_oracle_sample"},
        "__graft_entry__.py": {"smoke"},
    }
    for name, fns in allowed.items():
        uses = [fn for mod, fn in _imports(os.path.join(ROOT, name)) if mod == "oracle"]
        assert uses, name
        assert set(uses) <= fns, (name, uses)
