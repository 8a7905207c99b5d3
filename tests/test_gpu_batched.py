"""Batched forward (one graph launch over matrices of uneven sizes) and the SVD
adjoint, against the oracle and against the single-matrix path.

Gates: sigma normwise <= 1e-12 against the oracle, orthogonality <= 50 n
2^-53, the batched result bit-identical to the single-matrix path (same
arithmetic: zero padding rows add exact zeros), the adjoint within 1e-10
(relative, Frobenius) of the oracle's adjoint on the same U, S, V and within
1e-6 of central finite differences of L(A) = sum w_i s_i + <C, U V^T>.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1401_2720_gb300 import inputs as I
from paper_1401_2720_gb300 import jsvd as J
from tests.test_gpu_svd import _np, _orth, _t

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


def _batch(count, seed, m_hi=160):
    mats, sig, ws, Cs = I.workload_batch(count, seed=seed, m_hi=m_hi)
    return mats, sig, ws, Cs


@pytest.mark.parametrize("b", [None, 8, 16])
def test_batched_against_oracle(cuda, b):
    mats, sig, _, _ = _batch(40, seed=1)
    pk = J.Packing([a.shape[0] for a in mats], [a.shape[1] for a in mats])
    A = pk.pack(mats, cuda)
    U, S, V, infos, rc = J.svd_batched_packed(pk, A, b=b, return_info=True)
    assert rc == 0 and all(i["converged"] for i in infos)
    for a, s_true, u, s, v in zip(mats, sig, pk.unpack_mn(U), pk.unpack_n(S), pk.unpack_nn(V)):
        n = a.shape[1]
        s, u, v = _np(s), _np(u), _np(v)
        _, So, _, _ = O.svd(a, strategy="modulus")
        assert np.max(np.abs(s - So)) / So[0] <= 1e-12
        assert np.max(np.abs(s - s_true)) / s_true[0] <= 1e-12
        assert _orth(u) <= 50 * max(n, 2) * EPS and _orth(v) <= 50 * max(n, 2) * EPS
        assert np.linalg.norm(a - (u * s) @ v.T) <= 50 * max(n, 2) * EPS * np.linalg.norm(a)


@pytest.mark.parametrize("contraction", ["fp64", "split_sync"])
@pytest.mark.parametrize("b", [8, 16, 32])
def test_batched_equals_single_path(cuda, contraction, b):
    """Same block width, ordering and contraction form: the batched solver
    performs the single path's arithmetic (extra zero rows only add exact
    zeros; the split Gram's 256-row partials start at the same rows), bit for
    bit.  Row counts that end inside a split update block are included.  The
    batched solver's split form is the mma.sync one (both split modes), so it
    is compared with the single path's split_sync mode."""
    mats, _, _, _ = _batch(12, seed=2 + b)
    pk = J.Packing([a.shape[0] for a in mats], [a.shape[1] for a in mats])
    U, S, V = J.svd_batched_packed(pk, pk.pack(mats, cuda), b=b, contraction=contraction)
    for a, u, s, v in zip(mats, pk.unpack_mn(U), pk.unpack_n(S), pk.unpack_nn(V)):
        u1, s1, v1 = J.svd(_t(a, cuda), b=b, contraction=contraction)
        assert torch.equal(s, s1) and torch.equal(u, u1) and torch.equal(v, v1)


def test_batched_edge_shapes(cuda):
    rng = np.random.default_rng(3)
    shapes = [(1, 1), (2, 1), (2, 2), (16, 8), (17, 17), (33, 5), (64, 64), (100, 1)]
    mats = [np.asfortranarray(rng.standard_normal(s)) for s in shapes]
    pk = J.Packing([s[0] for s in shapes], [s[1] for s in shapes])
    U, S, V, infos, rc = J.svd_batched_packed(pk, pk.pack(mats, cuda), return_info=True)
    assert rc == 0
    for a, u, s, v in zip(mats, pk.unpack_mn(U), pk.unpack_n(S), pk.unpack_nn(V)):
        sl = np.linalg.svd(a, compute_uv=False)
        s = _np(s)
        assert np.max(np.abs(s - sl)) <= 1e-13 * max(sl[0], 1e-300)
        assert np.linalg.norm(a - (_np(u) * s) @ _np(v).T) <= 1e-13 * np.linalg.norm(a)


def test_batched_single_matrix_and_no_v(cuda):
    a = I.gaussian(70, 40, seed=4)
    pk = J.Packing([70], [40])
    U, S, V = J.svd_batched_packed(pk, pk.pack([a], cuda), with_v=False)
    assert V is None
    assert np.max(np.abs(_np(S) - np.linalg.svd(a, compute_uv=False))) <= 1e-13 * np.linalg.norm(a, 2)


def test_adjoint_matches_oracle(cuda):
    mats, sig, ws, Cs = _batch(16, seed=5, m_hi=96)
    pk = J.Packing([a.shape[0] for a in mats], [a.shape[1] for a in mats])
    U, S, V = J.svd_batched_packed(pk, pk.pack(mats, cuda))
    Us, Ss, Vs = pk.unpack_mn(U), pk.unpack_n(S), pk.unpack_nn(V)
    dU = torch.cat([torch.from_numpy(C).to(cuda).mm(v).t().reshape(-1) for C, v in zip(Cs, Vs)])
    dV = torch.cat([torch.from_numpy(C).to(cuda).t().mm(u).t().reshape(-1) for C, u in zip(Cs, Us)])
    dS = torch.cat([torch.from_numpy(w).to(cuda) for w in ws])
    dA = J.svd_backward_packed(pk, U, S, V, dU, dS, dV)
    for k, g in enumerate(pk.unpack_mn(dA)):
        u, s, v = _np(Us[k]), _np(Ss[k]), _np(Vs[k])
        C, w = Cs[k], ws[k]
        ref = O.svd_adjoint(u, s, v, C @ v, w, C.T @ u)
        assert np.linalg.norm(_np(g) - ref) <= 1e-10 * np.linalg.norm(ref)


def _loss(a, w, C, cuda):
    u, s, v = J.svd(_t(a, cuda), b=8)
    return float((torch.from_numpy(w).to(cuda) * s).sum() + (torch.from_numpy(C).to(cuda) * (u @ v.T)).sum())


@pytest.mark.parametrize("mn", [(24, 16), (40, 40), (60, 9)])
def test_adjoint_finite_differences(cuda, mn):
    """Well separated spectrum (gaps >= 0.1) so that FP64 central differences
    with h = 1e-6 resolve the derivative to ~1e-8."""
    m, n = mn
    rng = np.random.default_rng(m + n)
    a = I.planted(m, n, np.linspace(2.0, 0.5, n) if n > 1 else [1.0], rng)
    w = rng.standard_normal(n)
    C = rng.standard_normal((m, n))
    A = _t(a, cuda).requires_grad_(True)
    u, s, v = J.svd_autograd(A, b=8)
    L = (torch.from_numpy(w).to(cuda) * s).sum() + (torch.from_numpy(C).to(cuda) * (u @ v.T)).sum()
    L.backward()
    g = _np(A.grad)
    h = 1e-6
    for _ in range(4):
        E = rng.standard_normal((m, n))
        fd = (_loss(a + h * E, w, C, cuda) - _loss(a - h * E, w, C, cuda)) / (2 * h)
        assert float(np.sum(g * E)) == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_batched_autograd_matches_direct(cuda):
    mats, sig, ws, Cs = _batch(6, seed=6, m_hi=64)
    X = [_t(a, cuda).requires_grad_(True) for a in mats]
    Us, Ss, Vs = J.svd_batched(X)
    L = sum((torch.from_numpy(w).to(cuda) * s).sum() + (torch.from_numpy(C).to(cuda) * (u @ v.T)).sum()
            for u, s, v, w, C in zip(Us, Ss, Vs, ws, Cs))
    L.backward()
    for x, a, w, C in zip(X, mats, ws, Cs):
        u, s, v = J.svd(_t(a, cuda), b=8)
        un, sn, vn = _np(u), _np(s), _np(v)
        ref = O.svd_adjoint(un, sn, vn, C @ vn, w, C.T @ un)
        assert np.linalg.norm(_np(x.grad) - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("strategy", ["modulus", "R", "C", "rC"])
def test_batched_other_orderings(cuda, strategy):
    mats, sig, _, _ = _batch(10, seed=30, m_hi=120)
    pk = J.Packing([a.shape[0] for a in mats], [a.shape[1] for a in mats])
    U, S, V, infos, rc = J.svd_batched_packed(pk, pk.pack(mats, cuda), b=8, strategy=strategy,
                                              return_info=True)
    assert rc == 0
    for a, s_true, s, v in zip(mats, sig, pk.unpack_n(S), pk.unpack_nn(V)):
        assert np.max(np.abs(_np(s) - s_true)) / s_true[0] <= 1e-12
        assert _orth(_np(v)) <= 50 * max(a.shape[1], 2) * EPS
