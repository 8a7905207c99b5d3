"""GPU parity of the FP64 block-oriented SVD / HSVD against the oracle.

Tolerances (readings of the accuracy targets):
  * rotation parameters: bit-identical (same correctly rounded formulas);
  * one block sweep: element-wise agreement of G = U S and V with the
    oracle's block-oriented run, up to rounding of the Gram summation order;
  * converged results: normwise max |s - s_oracle| / s_1 <= 1e-12, relative
    |s - s_oracle| / s <= max(1e-12, 10 * floor) where floor is the oracle's
    own disagreement between two pivot orderings; orthogonality of U and V
    <= 50 n 2^-53 (max-abs of U^T U - I, V^T V - I).
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
    X = np.asarray(X)
    return np.abs(X.T @ X - np.eye(X.shape[1])).max()


def test_rotation_params_bitwise(cuda):
    rng = np.random.default_rng(0)
    n = 20000
    g = rng.standard_normal((n, 2, 5)) * 10.0 ** rng.uniform(-4, 4, size=(n, 2, 1))
    hpp = np.einsum("ij,ij->i", g[:, 0], g[:, 0])
    hqq = np.einsum("ij,ij->i", g[:, 1], g[:, 1])
    hpq = np.einsum("ij,ij->i", g[:, 0], g[:, 1])
    # add the branch cases: huge |ct2|, tiny |ct2|, ct2 = +-0, hyperbolic 5/4
    extra = np.array([[0.0, 2.0 ** 29, 1.0], [1.0, 1.0 + 2e-9, 1.0], [3.0, 3.0, 0.5],
                      [3.0, 3.0, -0.5], [1.0, 1.0, -1.0], [1.0, 1.0, 1.0]])
    hpp = np.concatenate([hpp, extra[:, 0]])
    hqq = np.concatenate([hqq, extra[:, 1]])
    hpq = np.concatenate([hpq, extra[:, 2]])
    for hyp in (False, True):
        cs_o, tn_o, pr_o = O.rotation(hpp, hqq, hpq, hyperbolic=hyp)
        cs, tn, pr = J.rotation_params(_t(hpp, cuda), _t(hqq, cuda), _t(hpq, cuda),
                                       torch.full((hpp.size,), int(hyp), dtype=torch.int32))
        assert np.array_equal(_np(cs).view(np.int64), cs_o.view(np.int64))
        assert np.array_equal(_np(tn).view(np.int64), tn_o.view(np.int64))
        assert np.array_equal(_np(pr), pr_o)


@pytest.mark.parametrize("contraction", ["fp64", "split"])
@pytest.mark.parametrize("b", [8, 16, 32])
@pytest.mark.parametrize("sweeps", [1, 2])
def test_block_sweeps_elementwise(cuda, b, sweeps, contraction):
    """After k block sweeps (no sorting of the output), G = U S and V agree
    element by element with the oracle's block-oriented method.  The columns
    are graded (norms 1 .. 1e-4) so that no two column norms nearly tie: a
    rotation angle's sensitivity to the Gram's rounding grows like
    eps / (relative gap of h_pp and h_qq), and the Gram summation orders of
    the two sides differ."""
    m, n = 320, 8 * b
    rng = np.random.default_rng(b)
    A = np.asfortranarray(rng.standard_normal((m, n)) * (10.0 ** (-4.0 * np.arange(n) / (n - 1)))[None, :])
    r = O.block_svd(A, b, strategy="rR", max_sweeps=sweeps)
    U, S, V, info = J.svd(_t(A, cuda), b=b, strategy="rR", max_sweeps=sweeps, sort=False,
                          return_info=True, contraction=contraction)
    assert info["sweeps"] == sweeps
    G = _np(U) * _np(S)[None, :]
    assert_columns_close(G, r["G"])
    assert np.max(np.abs(_np(V) - r["V"])) <= 1e-12
    assert info["breakdowns"] == r["breakdowns"] == 0


def assert_columns_close(G, Go, rtol=1e-12, zero_tol=None):
    """Per column: max_i |G_ij - Go_ij| <= rtol ||go_j||.  A column the
    oracle leaves numerically zero (||go_j|| <= zero_tol, if given) must be
    numerically zero on the GPU too; an exactly zero oracle column must be
    exactly zero."""
    cn = np.linalg.norm(Go, axis=0)
    for j in range(Go.shape[1]):
        d = np.max(np.abs(G[:, j] - Go[:, j]))
        if cn[j] == 0.0:
            assert d == 0.0, f"column {j}: oracle column is zero, GPU differs by {d:.3e}"
        elif zero_tol is not None and cn[j] <= zero_tol:
            assert np.linalg.norm(G[:, j]) <= zero_tol, f"column {j}: not numerically zero"
        else:
            assert d <= rtol * cn[j], f"column {j}: |dG| = {d:.3e} > {rtol:.0e} * {cn[j]:.3e}"


def smoothed_floor(So, So2, decades=0.5):
    """The oracle's disagreement with itself under a second ordering, as a
    per-sigma error level: the maximum over all sigma_j within `decades`
    decades of sigma_i (one pair of runs estimates the level only noisily)."""
    d = np.abs(So - So2) / So
    lg = np.log10(So)
    return np.array([d[np.abs(lg - lg[i]) <= decades].max() for i in range(len(So))])


def _sigma_gates(S, So, floor):
    assert np.max(np.abs(S - So)) / So[0] <= 1e-12
    rel = np.abs(S - So) / So
    assert np.all(rel <= np.maximum(1e-12, 10 * floor))


@pytest.mark.parametrize("b", [8, 16])
def test_svd_small_planted(cuda, b):
    """512 x 256, sigma geometric 1 .. 1e-8, Haar U and V (modulus ordering).
    kappa = 1e8 with Haar factors: no FP64 method resolves the small sigma
    to 1e-12 relative, so their gate is the smoothed oracle floor."""
    A = I.workload_small_planted(seed=0)
    n = A.shape[1]
    U, S, V, info = J.svd(_t(A, cuda), b=b, strategy="modulus", return_info=True)
    assert info["converged"] and info["breakdowns"] == 0
    Uo, So, Vo, _ = O.svd(A, strategy="modulus")
    _, So2, _, _ = O.svd(A, strategy="rR")
    floor = smoothed_floor(So, So2)
    S, U, V = _np(S), _np(U), _np(V)
    _sigma_gates(S, So, floor)
    assert _orth(U) <= 50 * n * EPS and _orth(V) <= 50 * n * EPS
    assert np.linalg.norm(A - (U * S) @ V.T) <= 50 * n * EPS * np.linalg.norm(A)
    s_true = I.geometric(n, 1.0, 1e-8)
    assert np.max(np.abs(S - s_true)) <= 1e-12 * s_true[0]


@pytest.mark.parametrize("strategy", ["modulus", "R", "C", "rR", "rC"])
def test_svd_strategies(cuda, strategy):
    A = I.gaussian(200, 128, seed=5)
    U, S, V, info = J.svd(_t(A, cuda), b=8, strategy=strategy, return_info=True)
    assert info["converged"]
    _, So, _, _ = O.svd(A)
    S = _np(S)
    assert np.max(np.abs(S - So)) / So[0] <= 1e-12
    assert _orth(_np(V)) <= 50 * 128 * EPS


@pytest.mark.parametrize("mn", [(300, 75), (97, 33), (64, 1), (5, 5), (2, 2), (40, 17)])
def test_svd_bordered_shapes(cuda, mn):
    """n not a multiple of 2b: identity bordering inside the library."""
    m, n = mn
    A = I.gaussian(m, n, seed=m + n) * (10.0 ** np.linspace(0, -3, n))[None, :]
    U, S, V, info = J.svd(_t(A, cuda), b=8, strategy="modulus", return_info=True)
    assert info["converged"]
    _, So, _, _ = O.svd(A, strategy="modulus")
    S, U, V = _np(S), _np(U), _np(V)
    assert np.max(np.abs(S - So)) / So[0] <= 1e-12
    assert _orth(U) <= 50 * max(n, 2) * EPS and _orth(V) <= 50 * max(n, 2) * EPS
    assert np.linalg.norm(A - (U * S) @ V.T) <= 50 * max(n, 2) * EPS * np.linalg.norm(A)


def test_hsvd(cuda):
    rng = np.random.default_rng(11)
    m, n, npl = 200, 128, 48
    G = np.asfortranarray(rng.standard_normal((m, n)))
    U, S, V, info = J.hsvd(_t(G, cuda), npl, b=8, return_info=True)
    assert info["converged"]
    Uo, So, Vo, _ = O.hsvd(G, npl)
    S, U, V = _np(S), _np(U), _np(V)
    assert np.max(np.abs(S - So)) / So.max() <= 1e-12
    j = np.where(np.arange(n) < npl, 1.0, -1.0)
    Jm = np.diag(j)
    nv = np.linalg.norm(V, 2) ** 2
    assert np.abs(V.T @ Jm @ V - Jm).max() <= 50 * n * EPS * nv
    assert _orth(U) <= 50 * n * EPS
    assert np.linalg.norm(G - (U * S) @ V.T) <= 50 * n * EPS * np.linalg.norm(G) * nv
    # eigenvalues of G J G^T, the error metric (6.1) of the paper
    lam = np.linalg.eigvalsh(G @ Jm @ G.T)
    lam = np.sort(lam[np.argsort(-np.abs(lam))][:n])
    assert np.max(np.abs(np.sort(S ** 2 * j) - lam)) <= 1e-12 * np.abs(lam).max()


def test_hsvd_identity_j_equals_svd(cuda):
    A = I.gaussian(96, 64, seed=2)
    a = J.svd(_t(A, cuda), b=8)
    b = J.hsvd(_t(A, cuda), 64, b=8)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_deterministic(cuda):
    A = I.planted(256, 128, I.geometric(128, 1, 1e-6), seed=4)
    a = J.svd(_t(A, cuda), b=16)
    b = J.svd(_t(A, cuda), b=16)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_nonfinite_rejected(cuda):
    A = I.gaussian(40, 16, seed=1)
    A[3, 5] = np.nan
    with pytest.raises(J.JsvdError) as e:
        J.svd(_t(A, cuda), b=8)
    assert e.value.status == 2


def test_zero_matrix(cuda):
    A = np.zeros((32, 16))
    U, S, V = J.svd(_t(A, cuda), b=8)
    assert torch.all(S == 0) and torch.all(U == 0)
    assert _orth(_np(V)) == 0.0


@pytest.mark.parametrize("mn_plus", [(150, 100, 37), (90, 61, 0), (70, 45, 45), (64, 33, 1)])
def test_hsvd_bordered(cuda, mn_plus):
    """HSVD with n not a multiple of 2b: the border goes in at the J boundary."""
    m, n, npl = mn_plus
    rng = np.random.default_rng(m + n + npl)
    G = np.asfortranarray(rng.standard_normal((m, n)))
    U, S, V, info = J.hsvd(_t(G, cuda), npl, b=8, return_info=True)
    assert info["converged"]
    _, So, _, _ = O.hsvd(G, npl, strategy="modulus")
    S, U, V = _np(S), _np(U), _np(V)
    assert np.max(np.abs(S - So)) / So.max() <= 1e-12
    j = np.where(np.arange(n) < npl, 1.0, -1.0)
    Jm = np.diag(j)
    nv = np.linalg.norm(V, 2) ** 2
    assert np.abs(V.T @ Jm @ V - Jm).max() <= 50 * n * EPS * nv
    assert np.linalg.norm(G - (U * S) @ V.T) <= 50 * n * EPS * np.linalg.norm(G) * nv
