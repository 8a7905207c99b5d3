"""The product path has no CPU fallback and never touches the oracle: the
binding refuses host tensors before any work, raises when the CUDA library is
missing, and no module of the package imports the oracle."""
import ast
import glob
import os

import pytest
import torch

from paper_1401_2720_gb300 import jsvd as J
from tests.conftest import ROOT


def test_host_tensors_are_refused():
    A = torch.zeros((8, 4), dtype=torch.float64)
    with pytest.raises(ValueError):
        J.svd(A)
    with pytest.raises(ValueError):
        J.hsvd(A, 2)
    with pytest.raises(ValueError):
        J.block_pstep(torch.zeros((4, 4), dtype=torch.float64), None, 2, 0)


def test_missing_library_raises(monkeypatch):
    monkeypatch.setattr(J, "_lib", None)
    monkeypatch.setattr(J, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libjsvd.so"))
    with pytest.raises(RuntimeError):
        J.library()


def test_package_never_imports_the_oracle():
    for path in glob.glob(os.path.join(ROOT, "paper_1401_2720_gb300", "*.py")):
        tree = ast.parse(open(path).read())
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                assert all(not a.name.split(".")[0] == "oracle" for a in node.names), path
            elif isinstance(node, ast.ImportFrom):
                assert (node.module or "").split(".")[0] != "oracle", path
