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


def test_packing_round_trip_and_offsets():
    """The batched ABI's packed layout: A_i column-major back to back at the
    element offsets the binding passes (host-side marshalling only)."""
    import numpy as np

    rng = np.random.default_rng(3)
    shapes = [(5, 3), (1, 1), (7, 7), (9, 2)]
    mats = [rng.standard_normal(s) for s in shapes]
    pk = J.Packing([m for m, _ in shapes], [n for _, n in shapes])
    buf = pk.pack(mats, "cpu")
    assert buf.numel() == pk.mn_total == sum(m * n for m, n in shapes)
    for a, o, (m, n) in zip(mats, pk.mn_off, shapes):
        assert np.array_equal(buf[o:o + m * n].numpy(), a.T.reshape(-1))        # column-major
    for a, back in zip(mats, pk.unpack_mn(buf)):
        assert np.array_equal(back.numpy(), a)
    assert list(pk.n_off) == [0, 3, 4, 11] and pk.n_total == 13
    assert list(pk.nn_off) == [0, 9, 10, 59] and pk.nn_total == 63
    sq = torch.arange(pk.nn_total, dtype=torch.float64)
    assert [tuple(x.shape) for x in pk.unpack_nn(sq)] == [(3, 3), (1, 1), (7, 7), (2, 2)]
    assert pk.unpack_nn(sq)[2][1, 0].item() == 10 + 1                           # (1, 0) of V_2, column-major
