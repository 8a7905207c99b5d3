"""Mixed precision (FP32 block sweeps, FP64 re-orthonormalization of V by the
polar series, FP64 block sweeps to convergence) against the FP64 oracle.

Same gates as the FP64 path: normwise |s - s_oracle| / s_1 <= 1e-12,
per-sigma relative error within 10x the oracle's own (smoothed)
disagreement between two orderings, orthogonality <= 50 n 2^-53.
"""
import numpy as np
import pytest

import oracle as O
from paper_1401_2720_gb300 import inputs as I
from paper_1401_2720_gb300 import jsvd as J
from tests.test_gpu_svd import _np, _orth, _t, smoothed_floor

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


@pytest.mark.parametrize("b", [8, 16])
def test_mixed_loguniform_spectrum(cuda, b):
    """A small copy of the mixed workload: s_i = 10^(-12 x_i), x_i ~ U(0,1)."""
    A, s_true = I.workload_mixed(384, 192, seed=3)
    U, S, V, info = J.svd(_t(A, cuda), b=b, precision="mixed", return_info=True)
    assert info["converged"] and info["sweeps_low"] >= 1
    _, So, _, _ = O.svd(A, strategy="rR")
    _, So2, _, _ = O.svd(A, strategy="modulus")
    floor = smoothed_floor(So, So2)
    S, U, V = _np(S), _np(U), _np(V)
    n = A.shape[1]
    assert np.max(np.abs(S - So)) / So[0] <= 1e-12
    assert np.all(np.abs(S - So) / So <= np.maximum(1e-12, 10 * floor))
    assert _orth(V) <= 50 * n * EPS
    assert np.linalg.norm(A - (U * S) @ V.T) <= 50 * n * EPS * np.linalg.norm(A)
    # U is orthonormal only as far as the tiny sigma are resolved in FP64;
    # the columns with s_i >= 1e-4 s_1 are checked to the orthogonality bound
    big = S >= 1e-4 * S[0]
    assert _orth(U[:, big]) <= 50 * n * EPS


def test_mixed_needs_fewer_fp64_sweeps(cuda):
    A = I.graded_gaussian(512, 256, seed=7)
    _, S64, _, i64 = J.svd(_t(A, cuda), b=16, return_info=True)
    _, Smx, _, imx = J.svd(_t(A, cuda), b=16, precision="mixed", return_info=True)
    assert imx["sweeps"] < i64["sweeps"]
    S64, Smx = _np(S64), _np(Smx)
    assert np.max(np.abs(S64 - Smx)) / S64[0] <= 1e-12


def test_mixed_hsvd(cuda):
    rng = np.random.default_rng(12)
    G = np.asfortranarray(rng.standard_normal((160, 128)))
    U, S, V, info = J.hsvd(_t(G, cuda), 64, b=8, precision="mixed", return_info=True)
    assert info["converged"]
    _, So, _, _ = O.hsvd(G, 64)
    assert np.max(np.abs(_np(S) - So)) / So.max() <= 1e-12


def test_mixed_bordered_shape(cuda):
    A, s_true = I.workload_mixed(210, 83, seed=9)
    U, S, V, info = J.svd(_t(A, cuda), b=16, precision="mixed", return_info=True)
    assert info["converged"]
    assert np.max(np.abs(_np(S) - s_true)) <= 1e-12 * s_true[0]
    assert _orth(_np(V)) <= 50 * 83 * EPS
