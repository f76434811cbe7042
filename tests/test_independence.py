"""Static checks that the CUDA path and the FP64 oracle stay apart.

- The package (Python and CUDA sources, and its build) never reaches the
  oracle, so no product call can fall back to it.
- The oracle never reaches the package, so the parity tests compare two
  independent programs.
- The seeded input generators import neither.
- bench.py touches the oracle only in its CPU-baseline legs and in the
  reference arm.
"""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2412_11554_gb300")


def _files(top, exts):
    for d, _, names in os.walk(top):
        for f in sorted(names):
            if f.endswith(exts):
                yield os.path.join(d, f)


def _imported_modules(path, tree=None):
    if tree is None:
        tree = ast.parse(open(path).read(), filename=path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name.split(".")[0], node
        elif isinstance(node, ast.ImportFrom):
            if node.level == 0 and node.module:
                yield node.module.split(".")[0], node


def test_package_never_reaches_the_oracle():
    py = list(_files(PKG, (".py",)))
    assert py
    for path in py:
        mods = {m for m, _ in _imported_modules(path)}
        assert "oracle" not in mods and "synth" not in mods, path
    for path in _files(PKG, (".cu", ".cuh", ".h", ".cpp")):
        src = open(path).read()
        assert not re.search(r'#\s*include\s*[<"][^>"]*oracle', src), path
    # the build compiles the package's own sources only
    build = open(os.path.join(PKG, "build.py")).read()
    assert "oracle" not in build


def test_oracle_never_reaches_the_package():
    for path in _files(os.path.join(ROOT, "oracle"), (".py",)):
        mods = {m for m, _ in _imported_modules(path)}
        assert not mods & {"paper_2412_11554_gb300", "torch", "synth", "bench"}, (path, mods)


def test_generators_hold_no_method_code():
    for path in _files(os.path.join(ROOT, "synth"), (".py",)):
        mods = {m for m, _ in _imported_modules(path)}
        assert not mods & {"oracle", "paper_2412_11554_gb300", "torch"}, (path, mods)


def test_bench_uses_the_oracle_only_for_the_cpu_baseline():
    """Every oracle import in bench.py sits in a CPU-baseline helper, in the
    reference arm, or under the `--no-cpu-baseline` switch's branch."""
    path = os.path.join(ROOT, "bench.py")
    src = open(path).read()
    tree = ast.parse(src)
    allowed_functions = {"oracle_sample", "oracle_trial_seconds", "run_reference"}
    parents = {}
    for node in ast.walk(tree):
        for child in ast.iter_child_nodes(node):
            parents[child] = node
    found = 0
    for mod, node in _imported_modules(path, tree):
        if mod != "oracle":
            continue
        found += 1
        ok = False
        up = parents.get(node)
        while up is not None:
            if isinstance(up, ast.FunctionDef) and up.name in allowed_functions:
                ok = True
            if isinstance(up, ast.If) and "no_cpu_baseline" in ast.get_source_segment(src, up.test):
                ok = True
            up = parents.get(up)
        assert ok, f"bench.py line {node.lineno} imports the oracle outside the CPU baseline"
    assert found >= 1
    # the module itself does not import the oracle at load time
    assert all(not isinstance(parents.get(n), ast.Module) for m, n in _imported_modules(path, tree) if m == "oracle")


def test_smoke_refuses_to_run_without_a_gpu():
    """__graft_entry__.smoke() needs a CUDA device; on a host without one it
    stops before any computation instead of falling back."""
    import sys

    import pytest
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    sys.path.insert(0, ROOT)
    import __graft_entry__ as g
    assert callable(g.build) and callable(g.smoke)
    with pytest.raises(AssertionError, match="CUDA device"):
        g.smoke()
