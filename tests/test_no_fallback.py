"""The product path has no CPU fallback: the binding refuses to run without
the CUDA library, and no module of the package reaches the oracle."""
import ast
import os

import pytest

import paper_2609_03866_b300 as pkg
from paper_2609_03866_b300 import api

PKG_DIR = os.path.dirname(pkg.__file__)


def test_missing_library_raises(monkeypatch):
    monkeypatch.setattr(api, "_lib", None)
    monkeypatch.setattr(api, "LIB_PATH", os.path.join(PKG_DIR, "no_such_libncf.so"))
    with pytest.raises(RuntimeError, match="is missing"):
        api.lib()
    with pytest.raises(RuntimeError, match="is missing"):
        api.corr([0.0, 1.0, 2.0], [1.0, 0.0, 2.0], [1.0])


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            yield from (a.name for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            yield node.module or ""


def test_package_never_imports_the_oracle_or_a_cpu_estimator():
    # only the test suite, the smoke check and the benchmark's CPU legs may use
    # the oracle; the package imports neither it nor a CPU library that could
    # stand in for the CUDA kernels
    banned = ("oracle", "scipy", "numpy.fft", "torch.fft")
    for name in sorted(os.listdir(PKG_DIR)):
        if not name.endswith(".py"):
            continue
        for mod in _imports(os.path.join(PKG_DIR, name)):
            assert not any(mod == b or mod.startswith(b + ".") for b in banned), f"{name} imports {mod}"
