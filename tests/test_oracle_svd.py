"""Pins of the oracle's SVD / HSVD against what mathematics and the paper fix:
planted singular values, LAPACK (numpy) and mpmath SVDs, the invariants
||A - U S V^T||, ||U^T U - I||, ||V^T V - I||, the eigenvalues of G J G^T for
the HSVD (Eq. (2.10), the error metric (6.1)), V^T J V = J, determinism."""
import numpy as np
import pytest

import oracle as O
from paper_1401_2720_gb300 import inputs as I

EPS = 2.0 ** -53


def _orth(X):
    return np.abs(X.T @ X - np.eye(X.shape[1])).max()


@pytest.mark.parametrize("strategy", ["modulus", "rR", "R", "C", "rC"])
def test_planted_sigma(strategy):
    m, n = 96, 48
    s_true = I.geometric(n, 1.0, 1e-6)
    A = I.planted(m, n, s_true, seed=3)
    U, S, V, r = O.svd(A, strategy=strategy)
    assert r["converged"]
    assert np.max(np.abs(S - s_true)) <= 50 * np.sqrt(n) * EPS * s_true[0]
    assert _orth(U) <= 50 * n * EPS and _orth(V) <= 50 * n * EPS
    assert np.linalg.norm(A - (U * S) @ V.T) <= 50 * n * EPS * np.linalg.norm(A)


def test_matches_lapack_and_vectors():
    rng = np.random.default_rng(4)
    A = np.asfortranarray(rng.standard_normal((80, 64)))
    U, S, V, _ = O.svd(A)
    Ul, Sl, Vlt = np.linalg.svd(A, full_matrices=False)
    assert np.max(np.abs(S - Sl)) <= 100 * EPS * Sl[0]
    # singular vectors agree up to sign (well separated spectrum)
    sgn = np.sign(np.sum(U * Ul, axis=0))
    assert np.max(np.abs(U * sgn - Ul)) < 1e-9
    assert np.max(np.abs(V * sgn - Vlt.T)) < 1e-9


def test_matches_mpmath_high_precision():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(5)
    A = np.asfortranarray(rng.standard_normal((7, 4)) * np.array([1.0, 1e-3, 10.0, 1e-5]))
    U, S, V, _ = O.svd(A)
    s_mp = mpmath.svd_r(mpmath.matrix(A.tolist()), compute_uv=False)
    s_ref = np.sort(np.array([float(x) for x in s_mp]))[::-1]
    # one-sided Jacobi is relatively accurate for column-scaled inputs
    assert np.max(np.abs(S - s_ref) / s_ref) <= 1e-13


@pytest.mark.parametrize("nplus", [2, 0])
def test_p2_sort_after_one_rotation(nplus):
    """Sec. 4.3 subphase 5 (reading R1 for the sign of the new diagonal): after
    the rotation of a trigonometric pair its columns are ordered by their new
    norms -- non-increasing in the J+ block, non-decreasing in the J- block --
    so one step on a two-column matrix leaves them in that order."""
    rng = np.random.default_rng(12)
    swaps = 0
    for _ in range(200):
        A = np.asfortranarray(rng.standard_normal((6, 2)) * 10.0 ** rng.uniform(-1, 1, size=2))
        r = O.hestenes(A, nplus=nplus, max_sweeps=1)
        h0, h1 = np.sum(r["G"] ** 2, axis=0)
        if nplus == 2:
            assert h0 >= h1 * (1 - 1e-12)
        else:
            assert h0 <= h1 * (1 + 1e-12)
        swaps += r["swaps"]
    assert 0 < swaps < 200                        # both orders occur before the sort


def test_tiny_bruteforce_2x2():
    A = np.asfortranarray(np.array([[3.0, 1.0], [1.0, 2.0]]))
    U, S, V, _ = O.svd(A)
    ev = np.linalg.eigvalsh(A.T @ A)
    assert np.allclose(np.sort(S ** 2), np.sort(ev), rtol=1e-15, atol=0)


def test_hsvd_eigenvalues_and_j_orthogonality():
    rng = np.random.default_rng(6)
    m, n, npl = 40, 24, 10
    G = np.asfortranarray(rng.standard_normal((m, n)))
    U, S, V, r = O.hsvd(G, npl)
    assert r["converged"]
    j = np.where(np.arange(n) < npl, 1.0, -1.0)
    J = np.diag(j)
    # Eq. (2.10): G = U S V^T with V^T J V = J
    assert np.linalg.norm(G - (U * S) @ V.T) <= 1e3 * EPS * np.linalg.norm(G) * np.linalg.norm(V) ** 2
    assert np.abs(V.T @ J @ V - J).max() <= 1e3 * n * EPS * np.linalg.norm(V, 2) ** 2
    assert _orth(U) <= 50 * n * EPS
    # sigma_i^2 j_i are the non-zero eigenvalues of G J G^T
    lam = np.linalg.eigvalsh(G @ J @ G.T)
    lam = lam[np.argsort(-np.abs(lam))][:n]
    mine = S ** 2 * j
    assert np.allclose(np.sort(mine), np.sort(lam), rtol=0, atol=1e-12 * np.abs(lam).max())
    # sign blocks sorted non-increasingly
    assert np.all(np.diff(S[:npl]) <= 0) and np.all(np.diff(S[npl:]) <= 0)


def test_hsvd_with_identity_j_is_svd():
    rng = np.random.default_rng(7)
    G = np.asfortranarray(rng.standard_normal((30, 20)))
    a = O.svd(G)
    b = O.hsvd(G, 20)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)


def test_deterministic():
    A = I.planted(64, 32, I.geometric(32, 1, 1e-4), seed=8)
    a = O.svd(A)
    b = O.svd(A)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("b", [2, 4, 8])
def test_block_method_agrees_with_pointwise(b):
    m, n = 72, 48
    s_true = I.geometric(n, 1.0, 1e-5)
    A = I.planted(m, n, s_true, seed=9)
    r = O.block_svd(A, b, strategy="rR")
    assert r["converged"] and r["breakdowns"] == 0
    U, S, V = O.finish(r["G"], r["V"])
    U2, S2, V2, _ = O.svd(A)
    assert np.max(np.abs(S - s_true)) <= 50 * np.sqrt(n) * EPS * s_true[0]
    assert np.max(np.abs(S - S2)) <= 50 * np.sqrt(n) * EPS * s_true[0]
    assert _orth(U) <= 50 * n * EPS and _orth(V) <= 50 * n * EPS
    # G = A V holds throughout (Eq. (2.5))
    assert np.linalg.norm(r["G"] - A @ r["V"]) <= 50 * n * EPS * np.linalg.norm(A)


def test_block_pstep_invariants():
    """One p-step: G' = A V', V' orthogonal, and the pair of block-columns it
    touched became (relatively) closer to orthogonal."""
    from oracle import pivots as P

    m, n, b = 64, 32, 4
    A = I.planted(m, n, I.geometric(n, 1, 1e-3), seed=10)
    tab = P.strategy("rR", n // b)
    inner = P.to_array(P.strategy("rR", 2 * b))
    G, V, st = O.block_pstep(A, np.eye(n), b, tab[0], inner)
    assert st["updated"] == len(tab[0]) and st["breakdowns"] == 0
    assert _orth(V) <= 50 * n * EPS
    assert np.linalg.norm(G - A @ V) <= 50 * n * EPS * np.linalg.norm(A)

    def off(X, P_, Q_):
        cols = list(range(P_ * b, P_ * b + b)) + list(range(Q_ * b, Q_ * b + b))
        Y = X[:, cols]
        H = Y.T @ Y
        d = np.sqrt(np.diag(H))
        Hn = H / np.outer(d, d)
        return np.linalg.norm(Hn - np.eye(2 * b))

    for P_, Q_ in tab[0]:
        assert off(G, P_, Q_) < off(A, P_, Q_)


@pytest.mark.parametrize("mn", [(2, 2), (5, 5), (40, 17), (97, 33), (300, 75), (64, 1)])
def test_block_method_with_identity_border(mn):
    """Identity bordering to a multiple of 2b (border columns static): the
    matrix columns' sigma equal LAPACK's, and the border rows of the matrix
    columns stay exactly zero."""
    m, n = mn
    A = I.gaussian(m, n, seed=m + n) * (10.0 ** np.linspace(0, -3, n))[None, :]
    B, bd, _ = O.bordered(A, 8)
    r = O.block_svd(B, 8, strategy="modulus", border=bd)
    assert r["converged"]
    keep = np.ones(B.shape[1], bool)
    keep[bd[0]:bd[1]] = False
    s = np.sort(np.sqrt((r["G"][:, keep] ** 2).sum(0)))[::-1]
    sl = np.linalg.svd(A, compute_uv=False)
    assert np.max(np.abs(s - sl)) <= 50 * np.sqrt(max(n, 2)) * EPS * sl[0]
    # the method's fixed point: the columns of the bordered G, border ones
    # included, are mutually orthogonal, and the matrix columns keep exactly
    # zero border rows
    Gc = r["G"][:, np.linalg.norm(r["G"], axis=0) > 0]
    H = Gc.T @ Gc
    d = np.sqrt(np.diag(H))
    assert np.abs(H / np.outer(d, d) - np.eye(H.shape[0])).max() <= 50 * np.sqrt(B.shape[0]) * EPS
    assert not np.any(r["G"][m:, keep])


@pytest.mark.parametrize("mnp", [(30, 13, 5), (41, 22, 0), (25, 10, 10), (36, 19, 18)])
def test_hsvd_block_method_with_identity_border(mnp):
    """HSVD of a bordered input (the border goes in at the J boundary): the
    matrix columns' signed squared norms are the non-zero eigenvalues of
    G J G^T (Eq. (2.10)), and the border columns leave as unit columns."""
    m, n, npl = mnp
    rng = np.random.default_rng(m + n + npl)
    G = np.asfortranarray(rng.standard_normal((m, n)))
    B, bd, npl_w = O.bordered(G, 4, npl)
    r = O.block_svd(B, 4, strategy="modulus", nplus=npl_w, border=bd)
    assert r["converged"]
    keep = np.ones(B.shape[1], bool)
    keep[bd[0]:bd[1]] = False
    sign = np.where(np.arange(B.shape[1]) < npl_w, 1.0, -1.0)
    mine = np.sort(((r["G"] ** 2).sum(0) * sign)[keep])
    j = np.where(np.arange(n) < npl, 1.0, -1.0)
    lam = np.linalg.eigvalsh(G @ np.diag(j) @ G.T)
    lam = np.sort(lam[np.argsort(-np.abs(lam))][:n])
    assert np.max(np.abs(mine - lam)) <= 1e-12 * np.abs(lam).max()
    assert np.allclose(np.linalg.norm(r["G"][:, bd[0]:bd[1]], axis=0), 1.0, rtol=0, atol=4 * EPS)
    assert np.all(r["G"][m:, keep] == 0.0)
    assert np.array_equal(r["G"][:, ~keep], B[:, ~keep])     # the border never moves


@pytest.mark.parametrize("b", [4, 8])
def test_block_method_zero_column_breaks_down_every_pstep(b):
    """Sec. 4.1 with a singular pivot Gram: a zero column has a zero Gram row,
    so its Cholesky pivot is exactly 0 in every p-step (one pivot pair per
    p-step holds it); it stays exactly zero and its singular value is 0."""
    m, n = 96, 8 * b
    A = I.graded_columns(m, n, 3.0, seed=b)
    A[:, 3] = 0.0
    for sweeps in (1, 2):
        r = O.block_svd(A, b, strategy="rR", max_sweeps=sweeps)
        assert r["breakdowns"] == (n // b - 1) * sweeps
        assert np.all(r["G"][:, np.linalg.norm(r["G"], axis=0) == 0.0] == 0.0)
    r = O.block_svd(A, b, strategy="rR", max_sweeps=30)
    assert r["converged"]
    s = np.sort(O.colnorms(r["G"]))[::-1]
    assert s[-1] == 0.0
    sl = np.linalg.svd(A, compute_uv=False)
    assert np.max(np.abs(s - sl)) <= 100 * np.sqrt(n) * EPS * sl[0]
    assert _orth(r["V"]) <= 50 * n * EPS


@pytest.mark.parametrize("b", [4, 8])
def test_block_method_duplicate_column_exact_breakdown(b):
    """An exact duplicate of a column with 16 entries +-1 at pivot position 0:
    L(0,0) = sqrt(16) = 4 and every multiplier of the copy is exact, so its
    pivot is exactly 16 - 4^2 = 0 (one breakdown in the first p-step).  The
    converged result has a numerically zero singular value and otherwise
    matches LAPACK normwise; the pointwise method agrees."""
    m, n = 96, 2 * b
    A = I.duplicated_pm1_column(I.graded_columns(m, n, 3.0, seed=10 + b), 0, 3, seed=b)
    r1 = O.block_svd(A, b, strategy="rR", max_sweeps=1)
    assert r1["breakdowns"] == 1
    r = O.block_svd(A, b, strategy="rR", max_sweeps=30)
    assert r["converged"]
    s = np.sort(O.colnorms(r["G"]))[::-1]
    sl = np.linalg.svd(A, compute_uv=False)
    assert s[-1] <= 50 * n * EPS * s[0]
    assert np.max(np.abs(s - sl)) <= 100 * np.sqrt(n) * EPS * sl[0]
    _, sp, _, _ = O.svd(A)
    assert sp[-1] <= 50 * n * EPS * sp[0]
    assert np.max(np.abs(sp - sl)) <= 100 * np.sqrt(n) * EPS * sl[0]


@pytest.mark.parametrize("mn", [(200, 40), (96, 48), (501, 17)])
def test_qr_preprocessing(mn):
    """Sec. 2, Eqs. (2.1)-(2.2): A P = Q [R; 0] with Q orthogonal, R upper
    triangular with non-increasing diagonal magnitudes (column pivoting), and
    the SVD through R^T equals LAPACK's; on a graded tall matrix the method on
    R^T needs fewer sweeps than on A."""
    m, n = mn
    A = I.graded_columns(m, n, 4.0, seed=m)[:, np.random.default_rng(n).permutation(n)].copy(order="F")
    W, tau, piv = O.qrcp(A)
    R = np.triu(W[:n, :])
    Q = O.apply_q(W, tau, np.eye(m))
    assert _orth(Q) <= 20 * m * EPS
    assert np.linalg.norm(Q[:, :n] @ R - A[:, piv]) <= 20 * m * EPS * np.linalg.norm(A)
    d = np.abs(np.diag(R))
    assert np.all(d[:-1] >= d[1:] * (1 - 1e-12))
    U, S, V, r = O.svd_qr(A)
    sl = np.linalg.svd(A, compute_uv=False)
    assert np.max(np.abs(S - sl)) <= 100 * np.sqrt(n) * EPS * sl[0]
    assert _orth(U) <= 50 * n * EPS and _orth(V) <= 50 * n * EPS
    assert np.linalg.norm(A - (U * S) @ V.T) <= 50 * n * EPS * np.linalg.norm(A)
    _, _, _, r0 = O.svd(A, strategy="modulus")
    assert r["sweeps"] < r0["sweeps"]
