"""Parity of the block method's edge cases against the oracle's block method
(Sec. 2, Sec. 4): rank-deficient pivot pairs (Cholesky breakdown, Sec. 4.1,
read as "zero the pivot's column of L and count it") and the full row count
of the benchmark's columns.

Gates, per column j of G = U S (oracle column g_j):
  max_i |G_ij - G^o_ij| <= 1e-12 ||g_j||; an exactly zero oracle column must be
  exactly zero; V element-wise <= 1e-12; breakdown counts equal.
The breakdown decision is exact on both sides only where the Gram matrix is:
  * a zero column has an exactly zero Gram row, hence a zero pivot in every
    p-step that holds it;
  * an exact duplicate of a column with 16 entries +-1 at pivot position 0
    gives L(0,0) = 4 exactly and a pivot of exactly 0 for the copy, in the
    first p-step.  Later p-steps see a numerically (not exactly) singular
    Gram; there the iterates are rounding-sensitive, so the duplicate case is
    compared element-wise after its first sweep of one pivot pair only, and on
    the converged singular values.
"""
import numpy as np
import pytest

import oracle as O
from paper_1401_2720_gb300 import inputs as I
from paper_1401_2720_gb300 import jsvd as J
from tests.test_gpu_svd import _np, _orth, _t, assert_columns_close

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


@pytest.mark.parametrize("contraction", ["fp64", "split"])
@pytest.mark.parametrize("b", [8, 16])
@pytest.mark.parametrize("sweeps", [1, 2])
def test_zero_columns_elementwise(cuda, b, sweeps, contraction):
    m, n = 320, 8 * b
    A = I.graded_columns(m, n, 4.0, seed=30 + b)
    zero = [5, n // 2 + 3]
    A[:, zero] = 0.0
    r = O.block_svd(A, b, strategy="rR", max_sweeps=sweeps)
    U, S, V, info = J.svd(_t(A, cuda), b=b, strategy="rR", max_sweeps=sweeps, sort=False, return_info=True,
                          contraction=contraction)
    nb = n // b
    # every p-step holds each zero column in exactly one pivot pair
    assert r["breakdowns"] == len(zero) * (nb - 1) * sweeps
    assert info["breakdowns"] == r["breakdowns"]
    G = _np(U) * _np(S)[None, :]
    assert_columns_close(G, r["G"])
    assert np.max(np.abs(_np(V) - r["V"])) <= 1e-12


@pytest.mark.parametrize("contraction", ["fp64", "split"])
@pytest.mark.parametrize("b", [8, 16])
def test_duplicate_column_breakdown(cuda, b, contraction):
    m, n = 320, 2 * b                      # one pivot pair: a sweep is one p-step
    A = I.duplicated_pm1_column(I.graded_columns(m, n, 4.0, seed=40 + b), 0, 3, seed=41 + b)
    r = O.block_svd(A, b, strategy="rR", max_sweeps=1)
    U, S, V, info = J.svd(_t(A, cuda), b=b, strategy="rR", max_sweeps=1, sort=False, return_info=True,
                          contraction=contraction)
    assert r["breakdowns"] == 1 and info["breakdowns"] == 1
    G = _np(U) * _np(S)[None, :]
    assert_columns_close(G, r["G"])
    assert np.max(np.abs(_np(V) - r["V"])) <= 1e-12
    # converged: one singular value is numerically zero on both sides; the
    # others agree normwise with the oracle's block and pointwise methods
    Uc, Sc, Vc, infc = J.svd(_t(A, cuda), b=b, strategy="rR", return_info=True, contraction=contraction)
    assert infc["converged"]
    rc = O.block_svd(A, b, strategy="rR", max_sweeps=30)
    So_blk = np.sort(O.colnorms(rc["G"]))[::-1]
    _, So, _, _ = O.svd(A)
    Sc = _np(Sc)
    for ref in (So_blk, So):
        assert ref[-1] <= 50 * n * EPS * ref[0]
        assert np.max(np.abs(Sc - ref)) <= 1e-12 * ref[0]
    assert Sc[-1] <= 50 * n * EPS * Sc[0]
    assert _orth(_np(Vc)) <= 50 * n * EPS
    keep = Sc > 1e3 * n * EPS * Sc[0]
    assert _orth(_np(Uc)[:, keep]) <= 50 * n * EPS


_FULL = {}


def _full_rows_oracle(sweeps):
    """The oracle's block method on 8192 x 256 graded columns (b = 32, the
    benchmark's pivot order 64, its 256-row Gram partials and 512-row update
    units over the full column length), cached per sweep count."""
    if sweeps not in _FULL:
        A = I.graded_columns(8192, 256, 4.0, seed=99)
        _FULL[sweeps] = (A, O.block_svd(A, 32, strategy="rR", max_sweeps=sweeps))
    return _FULL[sweeps]


@pytest.mark.parametrize("contraction", ["fp64", "split"])
@pytest.mark.parametrize("sweeps", [1, 2])
def test_full_column_length_elementwise(cuda, sweeps, contraction):
    A, r = _full_rows_oracle(sweeps)
    U, S, V, info = J.svd(_t(A, cuda), b=32, strategy="rR", max_sweeps=sweeps, sort=False, return_info=True,
                          contraction=contraction)
    assert info["sweeps"] == sweeps and info["breakdowns"] == r["breakdowns"] == 0
    G = _np(U) * _np(S)[None, :]
    assert_columns_close(G, r["G"])
    assert np.max(np.abs(_np(V) - r["V"])) <= 1e-12
