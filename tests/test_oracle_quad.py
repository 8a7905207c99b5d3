"""Pins of the oracle's binary128 build and of its threading.

The binary128 build runs the same pointwise method (Sec. 2, Sec. 4.3) with
eps = 2^-113; it is the ground truth for small sizes and for finite
differences of the SVD.  Pinned against: mpmath at 40 digits (its singular
values rounded to double must be within one ulp), the closed form
dL/dA = U diag(w) V^T of L = sum w_i s_i (a central difference in binary128
must reproduce it), and the FP64 oracle's adjoint at a well separated
spectrum.  Threading over the disjoint pairs of a p-step must not change a
single bit of the FP64 oracle's results."""
import numpy as np
import pytest

import oracle as O
from paper_1401_2720_gb300 import inputs as I

EPS = 2.0 ** -53


def test_q_svd_matches_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(8)
    A = np.asfortranarray(rng.standard_normal((9, 6)) * np.array([1.0, 1e-3, 10.0, 1e-5, 3.0, 1e-8]))
    U, S, V, ok = O.q_svd(A)
    assert ok
    s_mp = mpmath.svd_r(mpmath.matrix(A.tolist()), compute_uv=False)
    s_ref = np.sort(np.array([float(x) for x in s_mp]))[::-1]
    assert np.all(np.abs(S - s_ref) <= 2 * EPS * s_ref)
    assert np.abs(U.T @ U - np.eye(6)).max() <= 4 * EPS
    assert np.abs(V.T @ V - np.eye(6)).max() <= 4 * EPS
    assert np.linalg.norm(A - (U * S) @ V.T) <= 8 * EPS * np.linalg.norm(A)


def test_q_svd_agrees_with_fp64_oracle():
    A = I.planted(64, 40, I.geometric(40, 1.0, 1e-6), seed=12)
    _, S, _, _ = O.svd(A)
    _, Sq, _, ok = O.q_svd(A, with_vectors=False)
    assert ok
    assert np.max(np.abs(S - Sq)) <= 50 * np.sqrt(40) * EPS * Sq[0]


def test_q_loss_fd_reproduces_the_closed_form_derivative():
    """L = sum w_i s_i has dL/dA = U diag(w) V^T (C = 0)."""
    rng = np.random.default_rng(9)
    m, n = 12, 7
    A = I.planted(m, n, np.linspace(3.0, 0.5, n), rng)
    w = rng.standard_normal(n)
    C = np.zeros((m, n))
    U, S, V, _ = O.q_svd(A)
    grad = (U * w) @ V.T
    for _ in range(3):
        E = rng.standard_normal((m, n))
        fd = O.q_loss_fd(A, E, 2.0 ** -40, w, C)
        assert fd == pytest.approx(float(np.sum(grad * E)), rel=1e-13, abs=1e-13)


def test_q_loss_fd_matches_fp64_adjoint_well_separated():
    rng = np.random.default_rng(10)
    m, n = 15, 9
    A = I.planted(m, n, np.linspace(2.0, 0.4, n), rng)
    w = rng.standard_normal(n)
    C = np.asfortranarray(rng.standard_normal((m, n)))
    U, S, V, _ = O.svd(A)
    dA = O.svd_adjoint(U, S, V, C @ V, w, C.T @ U)
    for _ in range(3):
        E = rng.standard_normal((m, n))
        fd = O.q_loss_fd(A, E, 2.0 ** -40, w, C)
        assert fd == pytest.approx(float(np.sum(dA * E)), rel=1e-10, abs=1e-12)


def test_threads_do_not_change_a_bit():
    A = I.graded_columns(200, 96, 3.0, seed=4)
    res = []
    for t in (1, 3, 8):
        O.set_threads(t)
        rb = O.block_svd(A, 8, strategy="rR", max_sweeps=3)
        rp = O.hestenes(A, strategy="rR", max_sweeps=3)
        res.append((rb["G"], rb["V"], rb["proper"], rp["G"], rp["V"], rp["rotations"]))
    O.set_threads(1)
    for r in res[1:]:
        for x, y in zip(res[0], r):
            assert np.array_equal(np.asarray(x), np.asarray(y))
