"""FP64 block contractions on the tensor cores (contraction="split"): the Gram
(Eq. (2.7)) and the block update (Eq. (2.9)) formed from exact bf16 digit
slices.  The same parity gates as the FP64 FMA form, against the oracle."""
import os

import numpy as np
import pytest

import oracle as O
from paper_1401_2720_gb300 import inputs as I
from paper_1401_2720_gb300 import jsvd as J
from tests.test_gpu_svd import _np, _orth, _sigma_gates, _t, assert_columns_close, smoothed_floor

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


@pytest.mark.parametrize("b", [8, 16, 32])
@pytest.mark.parametrize("sweeps", [1, 2])
def test_split_block_sweeps_elementwise(cuda, b, sweeps):
    """After k block sweeps G = U S and V agree element by element with the
    oracle's block method (graded columns, as for the FP64 form).  Covers the
    three pivot orders 2b = 16, 32, 64 of the split Gram and update kernels."""
    m, n = 320, 8 * b
    rng = np.random.default_rng(b)
    A = np.asfortranarray(rng.standard_normal((m, n)) * (10.0 ** (-4.0 * np.arange(n) / (n - 1)))[None, :])
    r = O.block_svd(A, b, strategy="rR", max_sweeps=sweeps)
    U, S, V, info = J.svd(_t(A, cuda), b=b, strategy="rR", max_sweeps=sweeps, sort=False, return_info=True,
                          contraction="split")
    assert info["sweeps"] == sweeps
    G = _np(U) * _np(S)[None, :]
    assert_columns_close(G, r["G"])
    assert np.max(np.abs(_np(V) - r["V"])) <= 1e-12
    assert info["breakdowns"] == r["breakdowns"] == 0


@pytest.mark.parametrize("b", [8, 16, 32])
def test_split_row_count_not_a_multiple_of_the_update_unit(cuda, b):
    """m = 1000 rows: the workspace rows (1024 with the border) end inside an
    update unit of 512 rows, and the Gram has 8 chunks of 128."""
    m, n = 1000, 4 * b
    rng = np.random.default_rng(7 + b)
    A = np.asfortranarray(rng.standard_normal((m, n)) * (10.0 ** (-3.0 * np.arange(n) / (n - 1)))[None, :])
    r = O.block_svd(A, b, strategy="rR", max_sweeps=1)
    U, S, V, info = J.svd(_t(A, cuda), b=b, strategy="rR", max_sweeps=1, sort=False, return_info=True,
                          contraction="split")
    G = _np(U) * _np(S)[None, :]
    assert_columns_close(G, r["G"])
    assert np.max(np.abs(_np(V) - r["V"])) <= 1e-12


@pytest.mark.parametrize("b", [8, 16])
def test_split_small_planted(cuda, b):
    """512 x 256, sigma geometric 1 .. 1e-8, Haar U, V: the FP64 form's gates."""
    A = I.workload_small_planted(seed=0)
    n = A.shape[1]
    U, S, V, info = J.svd(_t(A, cuda), b=b, strategy="modulus", return_info=True, contraction="split")
    assert info["converged"] and info["breakdowns"] == 0
    _, So, _, _ = O.svd(A, strategy="modulus")
    _, So2, _, _ = O.svd(A, strategy="rR")
    S, U, V = _np(S), _np(U), _np(V)
    _sigma_gates(S, So, smoothed_floor(So, So2))
    assert _orth(U) <= 50 * n * EPS and _orth(V) <= 50 * n * EPS
    assert np.linalg.norm(A - (U * S) @ V.T) <= 50 * n * EPS * np.linalg.norm(A)
    s_true = I.geometric(n, 1.0, 1e-8)
    assert np.max(np.abs(S - s_true)) <= 1e-12 * s_true[0]


def test_split_graded_relative_accuracy(cuda):
    """Columns graded over 12 decades (D A with well-conditioned A): one-sided
    Jacobi resolves every sigma to high relative accuracy; the split form must
    keep it (the column scaling D of the update is what protects the small
    columns)."""
    m, n = 400, 128
    rng = np.random.default_rng(3)
    B = np.linalg.qr(rng.standard_normal((m, n)))[0] @ np.diag(1.0 + rng.uniform(0, 1, n))
    A = np.asfortranarray(B * (10.0 ** (-12.0 * rng.uniform(0, 1, n)))[None, :])
    U, S, V, info = J.svd(_t(A, cuda), b=16, return_info=True, contraction="split")
    assert info["converged"]
    _, So, _, _ = O.svd(A)
    S = _np(S)
    assert np.max(np.abs(S - So) / So) <= 1e-12
    assert _orth(_np(V)) <= 50 * n * EPS and _orth(_np(U)) <= 50 * n * EPS


@pytest.mark.parametrize("mn", [(300, 75), (97, 33), (64, 1), (5, 5), (40, 17)])
def test_split_bordered_shapes(cuda, mn):
    m, n = mn
    A = I.gaussian(m, n, seed=m + n) * (10.0 ** np.linspace(0, -3, n))[None, :]
    U, S, V, info = J.svd(_t(A, cuda), b=8, strategy="modulus", return_info=True, contraction="split")
    assert info["converged"]
    _, So, _, _ = O.svd(A, strategy="modulus")
    S, U, V = _np(S), _np(U), _np(V)
    assert np.max(np.abs(S - So)) / So[0] <= 1e-12
    assert _orth(U) <= 50 * max(n, 2) * EPS and _orth(V) <= 50 * max(n, 2) * EPS
    assert np.linalg.norm(A - (U * S) @ V.T) <= 50 * max(n, 2) * EPS * np.linalg.norm(A)


def test_split_hsvd(cuda):
    rng = np.random.default_rng(11)
    m, n, npl = 200, 128, 48
    G = np.asfortranarray(rng.standard_normal((m, n)))
    U, S, V, info = J.hsvd(_t(G, cuda), npl, b=8, return_info=True, contraction="split")
    assert info["converged"]
    _, So, _, _ = O.hsvd(G, npl)
    S, U, V = _np(S), _np(U), _np(V)
    assert np.max(np.abs(S - So)) / So.max() <= 1e-12
    j = np.where(np.arange(n) < npl, 1.0, -1.0)
    Jm = np.diag(j)
    nv = np.linalg.norm(V, 2) ** 2
    assert np.abs(V.T @ Jm @ V - Jm).max() <= 50 * n * EPS * nv
    assert _orth(U) <= 50 * n * EPS
    assert np.linalg.norm(G - (U * S) @ V.T) <= 50 * n * EPS * np.linalg.norm(G) * nv


def test_split_mixed_precision(cuda):
    """FP32 sweeps, then FP64 sweeps whose contractions are split."""
    m, n = 600, 256
    A, s_true = I.workload_mixed(m, n, seed=1)
    U, S, V, info = J.svd(_t(A, cuda), b=16, precision="mixed", return_info=True, contraction="split")
    assert info["converged"] and info["sweeps_low"] >= 1
    S = _np(S)
    s_true = np.sort(s_true)[::-1]
    assert np.max(np.abs(S - s_true)) <= 1e-12 * s_true[0]
    assert _orth(_np(V)) <= 50 * n * EPS


def test_split_agrees_with_fp64_form(cuda):
    """Both contraction forms on a 1024 x 768 graded matrix: the same sigma to
    the FP64 gate, both orthogonal."""
    A = np.asfortranarray(I.graded_gaussian(1024, 768, seed=4))
    _, S0, V0, i0 = J.svd(_t(A, cuda), b=32, return_info=True, contraction="fp64")
    _, S1, V1, i1 = J.svd(_t(A, cuda), b=32, return_info=True, contraction="split")
    assert i0["converged"] and i1["converged"]
    S0, S1 = _np(S0), _np(S1)
    assert np.max(np.abs(S1 - S0)) <= 1e-12 * S0[0]
    assert np.max(np.abs(S1 - S0) / S0) <= 1e-10
    assert _orth(_np(V1)) <= 50 * 768 * EPS


@pytest.mark.parametrize("b", [8, 16, 32])
def test_split_coherent_digits(cuda, b):
    """Columns whose 8-bit digits below the top one are the same in every row
    (up to the row's sign): the digit products add up coherently, so the
    Gram's level sums over a 256-row chunk come close to 2^24, the largest the
    FP32 accumulators hold exactly, and the update's level sums pass 2^22.
    The columns are nearly parallel (a dominant rank-one part), so the first
    sweep's rotation angles are sensitive to the Gram's rounding: after one
    block sweep the split form must be as close to the oracle, column by
    column, as the FP64 FMA form is (within a factor 4, or 1e-12); the
    converged singular values must match LAPACK."""
    m, n = 768, 4 * b
    A = I.coherent_digit_columns(m, n, seed=b)
    r = O.block_svd(A, b, strategy="rR", max_sweeps=1)
    cn = np.linalg.norm(r["G"], axis=0)
    errs = {}
    for form in ("split", "fp64"):
        U, S, V, info = J.svd(_t(A, cuda), b=b, strategy="rR", max_sweeps=1, sort=False, return_info=True,
                              contraction=form)
        G = _np(U) * _np(S)[None, :]
        errs[form] = np.max(np.abs(G - r["G"]), axis=0) / cn
    assert np.all(errs["split"] <= np.maximum(1e-12, 4.0 * errs["fp64"])), (errs["split"].max(), errs["fp64"].max())
    U, S, V, info = J.svd(_t(A, cuda), b=b, return_info=True, contraction="split")
    sl = np.linalg.svd(A, compute_uv=False)
    assert info["converged"] and info["breakdowns"] == 0
    assert np.max(np.abs(_np(S) - sl)) <= 1e-13 * sl[0]
    assert _orth(_np(V)) <= 50 * n * EPS


def test_split_gram_chunk_runs_and_cluster_jacobi(cuda):
    """2048 x 1280, b = 32: 20 pivot pairs x 8 Gram chunks of 256 rows = 160
    units for the GPU's CTAs, so some CTAs hold two consecutive chunks of a
    pair and sum them before writing the pair's partial, and the 20 pairs run
    their Jacobi steps on 2-CTA clusters.  After one block sweep every column
    is within 1e-10 of the oracle's, relative to its norm (a chunk missing from
    a partial would be off by O(1)), and the worst column is as close to the
    oracle as the FP64 FMA form's worst (within 4x, or 1e-12): with 640 pivot
    pairs some pair has nearly equal column norms, whose rotation angle
    amplifies the Gram's rounding (the FP64 form itself is 7e-12 off there).  The
    converged singular values match LAPACK."""
    m, n, b = 2048, 1280, 32
    A = I.graded_gaussian(m, n, seed=11)
    O.set_threads(os.cpu_count() or 1)      # disjoint pairs: bitwise the same as one thread
    try:
        r = O.block_svd(A, b, strategy="rR", max_sweeps=1)
    finally:
        O.set_threads(1)
    cn = np.linalg.norm(r["G"], axis=0)
    errs = {}
    for form in ("split", "fp64"):
        U, S, V, info = J.svd(_t(A, cuda), b=b, strategy="rR", max_sweeps=1, sort=False, return_info=True,
                              contraction=form)
        G = _np(U) * _np(S)[None, :]
        errs[form] = np.max(np.abs(G - r["G"]), axis=0) / cn
    assert errs["split"].max() <= 1e-10
    assert errs["split"].max() <= max(1e-12, 4.0 * errs["fp64"].max()), (errs["split"].max(), errs["fp64"].max())
    U, S, V, info = J.svd(_t(A, cuda), b=b, return_info=True, contraction="split")
    sl = np.linalg.svd(A, compute_uv=False)
    assert info["converged"] and info["breakdowns"] == 0
    assert np.max(np.abs(_np(S) - sl)) <= 1e-13 * sl[0]
