"""The oracle and the CUDA path share no code, and the product path never reaches the oracle.

* Nothing in the package (Python binding, C++ host code, CUDA kernels, headers) imports,
  includes, loads or names the oracle.
* Nothing in the oracle includes the package's sources or the C ABI header, or imports the
  package.
* The seeded input generators (``musr_inputs``), the one module both sides use, import
  neither side.
* ``bench.py`` imports the oracle only inside its CPU-baseline and reference legs (the
  Poisson leg's direct-sum baseline among them) and the precision report, which compares
  the two paths; never at module level.
"""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1509_07685_gb300")
ORACLE = os.path.join(ROOT, "oracle")
SOURCE_EXT = (".py", ".cu", ".cuh", ".cpp", ".h")


def _sources(top):
    for dirpath, dirnames, files in os.walk(top):
        dirnames[:] = [d for d in dirnames if not d.startswith(("_build", "__pycache__"))]
        for f in files:
            if f.endswith(SOURCE_EXT):
                yield os.path.join(dirpath, f)


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            names.add(node.module.split(".")[0])
    return names


def test_package_does_not_reach_the_oracle():
    files = list(_sources(PKG))
    assert any(f.endswith(".cuh") for f in files)
    for f in files:
        text = open(f).read()
        if f.endswith(".py"):
            assert "oracle" not in _imports(f), f
        assert not re.search(r"musr_oracle|_musr_oracle|\boracle/", text), f


def test_oracle_does_not_reach_the_package():
    files = list(_sources(ORACLE))
    assert any(f.endswith(".cpp") for f in files)
    for f in files:
        text = open(f).read()
        if f.endswith(".py"):
            assert "paper_1509_07685_gb300" not in _imports(f), f
        else:
            includes = re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', text)
            assert not [i for i in includes if "musr" in i or "csrc" in i], (f, includes)


def test_input_generators_import_neither_side():
    for f in _sources(os.path.join(ROOT, "musr_inputs")):
        if f.endswith(".py"):
            names = _imports(f)
            assert "oracle" not in names and "paper_1509_07685_gb300" not in names, f


def test_bench_imports_the_oracle_only_inside_its_cpu_legs():
    path = os.path.join(ROOT, "bench.py")
    tree = ast.parse(open(path).read(), path)
    allowed = {"run_reference", "_pool_init", "_oracle_task", "_oracle_worker", "cpu_baseline", "config_sweep",
               "precision_report", "_poisson"}  # _poisson: its direct-sum CPU baseline
    for node in tree.body:  # module level
        if isinstance(node, (ast.Import, ast.ImportFrom)):
            mods = [a.name for a in node.names] if isinstance(node, ast.Import) else [node.module or ""]
            assert not any(m.split(".")[0] == "oracle" for m in mods)
    for fn in [n for n in ast.walk(tree) if isinstance(n, ast.FunctionDef)]:
        for node in ast.walk(fn):
            if isinstance(node, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in node.names):
                assert fn.name in allowed, fn.name
