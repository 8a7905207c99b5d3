"""The dynamic block ordering (jsvd_opts.dynamic_order) and the ordering
study's building blocks on the GPU.

* The sweep table the solver uses is computed by one kernel
  (jsvd_sorted_pivot_table): its ranking must be a stable descending sort of
  the given block norms, and feeding that ranking to the oracle's remap of
  the oracle's static table must give the GPU's table bit for bit.
* Solves with the dynamic ordering: the oracle's block method with the same
  ordering (element-wise after one sweep, per column; the rankings of the
  two sides agree because the block norms of the start matrix are far apart),
  and converged singular values (SVD and HSVD) within the parity gates.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import pivots as P
from paper_1401_2720_gb300 import inputs as I
from paper_1401_2720_gb300 import jsvd as J
from tests.test_gpu_svd import _np, _orth, _t, assert_columns_close

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


@pytest.mark.parametrize("name", ["modulus", "rR", "R", "C", "rC"])
@pytest.mark.parametrize("nb", [4, 16, 64, 256])
def test_sorted_table_bit_exact(cuda, name, nb):
    rng = np.random.default_rng(nb)
    norms = rng.integers(0, nb // 2 + 1, size=nb).astype(np.float64)     # with ties
    perm, pairs = J.sorted_pivot_table(name, torch.from_numpy(norms).to(cuda))
    perm = _np(perm).tolist()
    assert perm == P.norm_order(norms)
    ref = P.to_array(P.remap(P.strategy(name, nb), perm))
    assert np.array_equal(_np(pairs), ref)


@pytest.mark.parametrize("contraction", ["split", "fp64"])
def test_dynamic_order_first_sweep_elementwise(cuda, contraction):
    b = 8
    A = I.graded_columns(320, 8 * b, 4.0, seed=5)[:, ::-1].copy(order="F")   # blocks in ascending norm
    r = O.block_svd_dynamic(A, b, strategy="rR", max_sweeps=1)
    U, S, V, info = J.svd(_t(A, cuda), b=b, strategy="rR", max_sweeps=1, sort=False, return_info=True,
                          contraction=contraction, dynamic_order=True)
    G = _np(U) * _np(S)[None, :]
    assert_columns_close(G, r["G"])
    assert np.max(np.abs(_np(V) - r["V"])) <= 1e-12


@pytest.mark.parametrize("shape", [(600, 256), (333, 200)])
def test_dynamic_order_svd(cuda, shape):
    m, n = shape
    A = I.graded_gaussian(m, n, seed=n)
    U, S, V, info = J.svd(_t(A, cuda), b=16, return_info=True, dynamic_order=True)
    assert info["converged"]
    _, So, _, _ = O.svd(A, strategy="modulus")
    S = _np(S)
    assert np.max(np.abs(S - So)) <= 1e-12 * So[0]
    assert _orth(_np(U)) <= 50 * n * EPS and _orth(_np(V)) <= 50 * n * EPS


def test_dynamic_order_hsvd(cuda):
    rng = np.random.default_rng(3)
    m, n, npl = 300, 192, 80
    G = np.asfortranarray(rng.standard_normal((m, n)))
    U, S, V, info = J.hsvd(_t(G, cuda), npl, b=8, return_info=True, dynamic_order=True)
    assert info["converged"]
    _, So, _, _ = O.hsvd(G, npl, strategy="modulus")
    S, V = _np(S), _np(V)
    assert np.max(np.abs(S - So)) / So.max() <= 1e-12
    j = np.where(np.arange(n) < npl, 1.0, -1.0)
    Jm = np.diag(j)
    assert np.abs(V.T @ Jm @ V - Jm).max() <= 50 * n * EPS * np.linalg.norm(V, 2) ** 2
