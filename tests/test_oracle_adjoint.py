"""Pins of the oracle's SVD adjoint: central finite differences of
L(A) = sum_i w_i s_i + <C, U V^T> evaluated with LAPACK (numpy) SVDs."""
import numpy as np
import pytest

import oracle as O
from paper_1401_2720_gb300 import inputs as I


def _loss(A, w, C):
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    return float(w @ s + np.sum(C * (U @ Vt)))


@pytest.mark.parametrize("mn", [(12, 8), (20, 20), (33, 9)])
def test_adjoint_finite_differences(mn):
    m, n = mn
    rng = np.random.default_rng(m * 100 + n)
    s = np.linspace(2.0, 1.0, n)                       # gaps >= 1/(n-1)
    A = I.planted(m, n, s, rng)
    w = rng.standard_normal(n)
    C = rng.standard_normal((m, n))
    U, S, V, _ = O.svd(A)
    dA = O.svd_adjoint(U, S, V, C @ V, w, C.T @ U)
    h = 1e-6
    for _ in range(6):
        E = rng.standard_normal((m, n))
        fd = (_loss(A + h * E, w, C) - _loss(A - h * E, w, C)) / (2 * h)
        an = float(np.sum(dA * E))
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-7)


def test_adjoint_sigma_only_is_u_v_outer():
    """With only dS: dA = U diag(dS) V^T exactly (closed form)."""
    rng = np.random.default_rng(1)
    m, n = 10, 6
    A = I.planted(m, n, np.linspace(3, 1, n), rng)
    U, S, V, _ = O.svd(A)
    w = rng.standard_normal(n)
    dA = O.svd_adjoint(U, S, V, np.zeros((m, n)), w, np.zeros((n, n)))
    assert np.allclose(dA, (U * w) @ V.T, atol=1e-14)
