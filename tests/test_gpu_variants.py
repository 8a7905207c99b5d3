"""Full-block variant (M_s > 1 inner sweeps, Sec. 4.3), the sweep-limit status
and argument validation through the C ABI."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_1401_2720_gb300 import inputs as I
from paper_1401_2720_gb300 import jsvd as J
from tests.test_gpu_svd import _np, _orth, _t

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


@pytest.mark.parametrize("inner", [2, 30])
def test_full_block_variant_elementwise(cuda, inner):
    """M_s inner sweeps per pivot pair: after one block sweep G = U S and V
    agree element by element with the oracle's block method with the same M_s
    (graded columns, as in the block-oriented element-wise test)."""
    m, n, b = 256, 64, 8
    rng = np.random.default_rng(inner)
    A = np.asfortranarray(rng.standard_normal((m, n)) * (10.0 ** (-4.0 * np.arange(n) / (n - 1)))[None, :])
    r = O.block_svd(A, b, strategy="rR", inner_sweeps=inner, max_sweeps=1)
    U, S, V, info = J.svd(_t(A, cuda), b=b, strategy="rR", inner_sweeps=inner, max_sweeps=1, sort=False,
                          return_info=True)
    G = _np(U) * _np(S)[None, :]
    assert np.max(np.abs(G - r["G"])) <= 1e-12 * np.linalg.norm(A, 2)
    assert np.max(np.abs(_np(V) - r["V"])) <= 1e-12


def test_full_block_variant_converges(cuda):
    A = I.planted(300, 128, I.geometric(128, 1.0, 1e-6), seed=3)
    _, S1, _, i1 = J.svd(_t(A, cuda), b=16, return_info=True)
    U, S, V, i30 = J.svd(_t(A, cuda), b=16, inner_sweeps=30, return_info=True)
    assert i30["converged"] and i30["sweeps"] <= i1["sweeps"]
    assert float((S - S1).abs().max()) <= 1e-12 * float(S1[0])
    assert _orth(_np(V)) <= 50 * 128 * EPS


def test_sweep_limit_status_and_partial_result(cuda):
    """The sweep limit returns JSVD_NOT_CONVERGED with the last iterate: V is
    still orthogonal and U S V^T reproduces A."""
    A = I.planted(200, 96, I.geometric(96, 1.0, 1e-8), seed=5)
    U, S, V, info = J.svd(_t(A, cuda), b=8, max_sweeps=2, return_info=True)
    assert info["status"] == 1 and not info["converged"] and info["sweeps"] == 2
    V, S, U = _np(V), _np(S), _np(U)
    assert _orth(V) <= 50 * 96 * EPS
    assert np.linalg.norm(A - (U * S) @ V.T) <= 1e-12 * np.linalg.norm(A)


def test_argument_validation(cuda):
    lib = J.library()
    h = J.context()
    buf = torch.zeros(64 * 64, dtype=torch.float64, device=cuda)
    p = buf.data_ptr()
    # m < n, n < 1, null A, lda < m, null S, ldu < m
    assert lib.jsvd_dgesvj(h, 10, 20, p, 10, p, p, 10, p, 20, None, None) == -2
    assert lib.jsvd_dgesvj(h, 10, 0, p, 10, p, p, 10, p, 10, None, None) == -3
    assert lib.jsvd_dgesvj(h, 10, 5, None, 10, p, p, 10, p, 5, None, None) == -4
    assert lib.jsvd_dgesvj(h, 10, 5, p, 9, p, p, 10, p, 5, None, None) == -5
    assert lib.jsvd_dgesvj(h, 10, 5, p, 10, None, p, 10, p, 5, None, None) == -6
    assert lib.jsvd_dgesvj(h, 10, 5, p, 10, p, p, 9, p, 5, None, None) == -8
    assert lib.jsvd_dhsvj(h, 10, 5, 6, p, 10, p, p, 10, p, 5, None, None) == -4
    assert lib.jsvd_dgesvj(None, 10, 5, p, 10, p, p, 10, p, 5, None, None) == -1
    # an unsupported block width is reported, not run
    o = J.make_opts(b=12)
    assert lib.jsvd_dgesvj(h, 32, 16, p, 32, p, p, 32, p, 16, ctypes.byref(o), None) == 5
