"""Parity of the block method's edge cases against the oracle's block method
(Sec. 2, Sec. 4): rank-deficient pivot pairs (Cholesky breakdown, Sec. 4.1,
read as "zero the pivot's column of L and count it"), the full row count
of the benchmark's columns, and the benchmark's own 8192 x 8192 input and
launch configuration, one block p-step at a time.

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
import os

import numpy as np
import pytest
import torch

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


_BENCH = {}


def _bench_oracle():
    """The oracle's first two block p-steps on the 8192 x 8192 graded
    benchmark input (seed 0), b = 32, reversed row-cyclic strategy, and its
    disagreement with itself when the rows are reversed (the same exact
    values, another summation order in every Gram entry and update): per step
    (G, V, stats, floor of G per column relative to ||g_j||, floor of V)."""
    if not _BENCH:
        n, b = 8192, 32
        A = I.graded_gaussian(n, n, seed=0)
        tab = O.strategy_array("rR", n // b)
        inner = O.strategy_array("rR", 2 * b)
        O.set_threads(os.cpu_count() or 1)      # disjoint pairs: bitwise the same as one thread
        try:
            Go, Vo = np.array(A, order="F", copy=True), np.asfortranarray(np.eye(n))   # A stays the input
            Gr, Vr = np.asfortranarray(A[::-1]), np.asfortranarray(np.eye(n))
            for step in (0, 1):
                Go, Vo, r = O.block_pstep(Go, Vo, b, tab[step], inner, inplace=True)
                Gr, Vr, _ = O.block_pstep(Gr, Vr, b, tab[step], inner, inplace=True)
                fg = (np.abs(Go - Gr[::-1]).max(axis=0) / np.linalg.norm(Go, axis=0)).max()
                _BENCH[step] = (Go.copy(order="F"), Vo.copy(order="F"), r, fg, np.abs(Vo - Vr).max())
        finally:
            O.set_threads(1)
        _BENCH["A"] = A
    return _BENCH


@pytest.mark.parametrize("contraction", ["split", "fp64"])
def test_benchmark_input_psteps_elementwise(cuda, contraction):
    """The benchmark's 8192 x 8192 input, b = 32, reversed row-cyclic strategy:
    its first two block p-steps (128 pivot pairs each, every pair updated)
    with the kernels and launch configuration of the benchmark's solve,
    against the oracle's block p-steps, every entry of G and V.  Gates: G per
    column max(1e-12, 10 floor_G) ||g_j||, V element-wise max(1e-12, 10
    floor_V), where the floors are the oracle's own disagreement under row
    reversal (measured: V 2.3e-12 and 1.7e-12 -- rotation angles of pairs whose
    column norms nearly agree are that sensitive to the Gram's rounding)."""
    ref = _bench_oracle()
    n, b = 8192, 32
    G = torch.from_numpy(np.ascontiguousarray(ref["A"].T)).to(cuda).t()
    V = torch.eye(n, dtype=torch.float64, device=cuda).t()     # column-major view
    for step in (0, 1):
        Go, Vo, r, fg, fv = ref[step]
        info = J.block_pstep(G, V, b, step, "rR", contraction)
        assert info["pairs_updated"] == r["updated"] == n // (2 * b)
        assert info["breakdowns"] == r["breakdowns"] == 0
        worst = (np.abs(_np(G) - Go).max(axis=0) / np.linalg.norm(Go, axis=0)).max()
        assert worst <= max(1e-12, 10 * fg), (step, worst, fg)
        dv = np.abs(_np(V) - Vo).max()
        assert dv <= max(1e-12, 10 * fv), (step, dv, fv)
