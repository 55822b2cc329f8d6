"""The product path has no CPU fallback: without a GPU or without the CUDA
library every call raises, and no module of the package reaches the oracle."""
import ast
import os

import numpy as np
import pytest
import torch

import paper_1804_02883_gb300 as P
from paper_1804_02883_gb300 import binding
from paper_1804_02883_gb300 import workloads as W

PKG = os.path.dirname(os.path.abspath(P.__file__))


def test_package_never_imports_the_oracle():
    for root, _, files in os.walk(PKG):
        for f in files:
            if not f.endswith(".py"):
                continue
            tree = ast.parse(open(os.path.join(root, f)).read())
            for node in ast.walk(tree):
                if isinstance(node, ast.Import):
                    names = [a.name for a in node.names]
                elif isinstance(node, ast.ImportFrom):
                    names = [node.module or ""] + [a.name for a in node.names]
                else:
                    continue
                assert not any("oracle" in n for n in names), (f, names)


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the host without a GPU")
def test_calls_raise_without_a_gpu():
    small = W.with_(W.plain_small(), nx=16, ny=16, ns=8)
    with pytest.raises(RuntimeError):
        P.EpdLb([small])
    with pytest.raises(RuntimeError):
        P.prop_solve3d(small, np.zeros((3, 8, 16, 16)))


def test_missing_library_raises(monkeypatch):
    def no_library(*a, **k):
        raise FileNotFoundError("libepd_lb.so")

    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding._build, "build", no_library)
    with pytest.raises(FileNotFoundError):
        P.epd_lb_workspace_bytes([W.plain_small()])
    with pytest.raises(FileNotFoundError):
        P.EpdLb([W.plain_small()])
