"""GPU parity on the degenerate cases of the one-sided Jacobi method (Sec. 2,
Sec. 4), through the C ABI, against the oracle and against what the input fixes.

Where the singular vectors are not unique (equal or clustered singular values,
zero singular values) only what is unique is compared -- the singular values,
the orthogonal projectors onto the invariant subspaces of a cluster, the rank-one
part u_1 s_1 v_1^T -- and the rest is checked for validity (orthogonality of V,
A = U S V^T).  Tolerances:
  * a permuted diagonal input needs no rotation: the Gram off-diagonals are
    exactly zero (Sec. 4.3: h_pq = 0 is relatively orthogonal), the P2 sorting
    only permutes columns, and the update by a permutation is exact in both
    contraction forms, so V is the oracle's permutation exactly and S, U agree
    to the rounding of the final column norm (4 eps relative);
  * clusters: per cluster, the projector and the relative singular-value error
    within 30x the oracle's own error against the planted factors (floor 1e-13
    and 1e-12), i.e. the same perturbation bound the oracle meets;
  * orthogonal input: all singular values 1 to 1e-14;
  * rank one: s_1 to 1e-14 relative, the other singular values below 1e-13 s_1,
    u_1 s_1 v_1^T = A to 1e-13 relative, V orthogonal to 50 n 2^-53.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1401_2720_gb300 import inputs as I
from paper_1401_2720_gb300 import jsvd as J

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


def _t(A, dev):
    return torch.from_numpy(np.ascontiguousarray(A)).to(dev)


def _np(x):
    return x.detach().cpu().numpy()


def _orth(X):
    return np.abs(X.T @ X - np.eye(X.shape[1])).max()


@pytest.mark.parametrize("contraction", ["split", "fp64"])
def test_permuted_diagonal_is_only_sorted(cuda, contraction):
    rng = np.random.default_rng(5)
    m, n = 48, 32
    d = (10.0 ** rng.uniform(-6, 0, n)) * rng.choice([-1.0, 1.0], n)
    A = np.zeros((m, n))
    A[np.arange(n), rng.permutation(n)] = d
    U, S, V, info = J.svd(_t(A, cuda), b=8, contraction=contraction, return_info=True)
    assert info["converged"] and info["proper_rotations"] == 0 and info["breakdowns"] == 0
    Uo, So, Vo, _ = O.svd(A)
    S, U, V = _np(S), _np(U), _np(V)
    assert np.array_equal(So, np.sort(np.abs(d))[::-1])
    assert np.all(np.abs(S - So) <= 4 * EPS * So)
    assert np.array_equal(V, Vo)                       # a permutation, exactly
    assert np.abs(U - Uo).max() <= 4 * EPS


def test_orthogonal_input_all_singular_values_one(cuda):
    Q = I.haar_thin(160, 96, seed=3)
    U, S, V, info = J.svd(_t(Q, cuda), b=8, return_info=True)
    assert info["converged"]
    _, So, _, _ = O.svd(Q)
    S, U, V = _np(S), _np(U), _np(V)
    assert np.abs(So - 1.0).max() <= 1e-14 and np.abs(S - 1.0).max() <= 1e-14
    n = Q.shape[1]
    assert _orth(U) <= 50 * n * EPS and _orth(V) <= 50 * n * EPS
    assert np.abs(Q - (U * S) @ V.T).max() <= 50 * n * EPS


def test_clustered_singular_values_subspaces(cuda):
    m, n, k = 200, 64, 16
    s = np.repeat([1.0, 1e-2, 1e-4, 1e-6], k)
    Uh = I.haar_thin(m, n, seed=7)
    Vh = I.haar(n, seed=8)
    A = (Uh * s) @ Vh.T
    U, S, V, info = J.svd(_t(A, cuda), b=8, return_info=True)
    assert info["converged"]
    Uo, So, Vo, _ = O.svd(A)
    S, U, V = _np(S), _np(U), _np(V)
    assert np.max(np.abs(S - s)) <= 1e-12
    assert _orth(V) <= 50 * n * EPS
    for c in range(4):
        sl = slice(k * c, k * (c + 1))
        pu, pv = Uh[:, sl] @ Uh[:, sl].T, Vh[:, sl] @ Vh[:, sl].T
        for X, Xo, P in ((U, Uo, pu), (V, Vo, pv)):
            err_o = np.abs(Xo[:, sl] @ Xo[:, sl].T - P).max()
            err = np.abs(X[:, sl] @ X[:, sl].T - P).max()
            assert err <= max(30 * err_o, 1e-13), (c, err, err_o)
        rel_o = np.max(np.abs(So[sl] - s[sl]) / s[sl])
        rel = np.max(np.abs(S[sl] - s[sl]) / s[sl])
        assert rel <= max(30 * rel_o, 1e-12), (c, rel, rel_o)


@pytest.mark.parametrize("contraction", ["split", "fp64"])
def test_rank_one(cuda, contraction):
    rng = np.random.default_rng(6)
    x = rng.standard_normal(120)
    y = rng.standard_normal(48) * 10.0 ** rng.uniform(-3, 0, 48)
    A = np.outer(x, y)
    U, S, V, info = J.svd(_t(A, cuda), b=8, contraction=contraction, return_info=True)
    assert info["converged"]
    _, So, _, _ = O.svd(A)
    S, U, V = _np(S), _np(U), _np(V)
    s1 = np.linalg.norm(x) * np.linalg.norm(y)
    assert abs(So[0] - s1) <= 1e-14 * s1 and abs(S[0] - s1) <= 1e-14 * s1
    assert S[1:].max() <= 1e-13 * s1
    assert np.abs(np.outer(U[:, 0] * S[0], V[:, 0]) - A).max() <= 1e-13 * np.abs(A).max()
    assert _orth(V) <= 50 * A.shape[1] * EPS
