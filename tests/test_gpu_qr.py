"""The batched solver's QR preprocessing (Sec. 2, Eqs. (2.1)-(2.2)):
matrices with m >= 2n are factored A P = Q [R; 0] (Householder, column
pivoting) and the method runs on R^T; the others pass through unchanged.
Gates: singular values normwise <= 1e-12 against the oracle's preprocessed
SVD and LAPACK, orthogonality and reconstruction <= 50 n 2^-53; the
pass-through matrices are bit-identical to a run without preprocessing;
graded tall matrices need fewer sweeps."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1401_2720_gb300 import inputs as I
from paper_1401_2720_gb300 import jsvd as J
from tests.test_gpu_svd import _np, _orth

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


def _mats():
    rng = np.random.default_rng(21)
    shapes = [(200, 40), (96, 48), (501, 17), (120, 100), (64, 64), (300, 9), (33, 16), (128, 70)]
    mats = []
    for k, (m, n) in enumerate(shapes):
        a = I.graded_columns(m, n, 4.0, seed=k)[:, rng.permutation(n)]
        mats.append(np.asfortranarray(a))
    return mats


@pytest.mark.parametrize("b", [8, 16])
def test_batched_qr_preprocessing(cuda, b):
    mats = _mats()
    pk = J.Packing([a.shape[0] for a in mats], [a.shape[1] for a in mats])
    A = pk.pack(mats, cuda)
    U, S, V, infos, rc = J.svd_batched_packed(pk, A, b=b, return_info=True, preprocess=True)
    assert rc == 0
    U0, S0, V0, infos0, rc0 = J.svd_batched_packed(pk, A, b=b, return_info=True)
    for k, (a, u, s, v) in enumerate(zip(mats, pk.unpack_mn(U), pk.unpack_n(S), pk.unpack_nn(V))):
        m, n = a.shape
        u, s, v = _np(u), _np(s), _np(v)
        sl = np.linalg.svd(a, compute_uv=False)
        _, sq, _, _ = O.svd_qr(a)
        assert np.max(np.abs(s - sl)) <= 1e-12 * sl[0]
        assert np.max(np.abs(s - sq)) <= 1e-12 * sq[0]
        assert _orth(u) <= 50 * n * EPS and _orth(v) <= 50 * n * EPS
        assert np.linalg.norm(a - (u * s) @ v.T) <= 50 * n * EPS * np.linalg.norm(a)
        if m < 2 * n:    # passed through: the same computation bit for bit
            assert torch.equal(pk.unpack_n(S)[k], pk.unpack_n(S0)[k])
            assert torch.equal(pk.unpack_mn(U)[k], pk.unpack_mn(U0)[k])
        else:            # the method on R^T converges in fewer sweeps here
            assert infos[k]["sweeps"] <= infos0[k]["sweeps"]
