"""The robust path (App. A) on the GPU: DRDSSQ column norms and the initial
power-of-two scaling of the solvers.

* jsvd_column_sumsq against the oracle's DRDSSQ column by column (values
  within m 2^-53 relative), on columns far outside the range where a plain
  sum of squares survives.
* A power-of-two scaling of the input commutes with every floating-point
  operation of the method (the split contractions' exponent bounds shift
  with it), so the solve of 2^s A equals the solve of A with S scaled by 2^s
  bit for bit -- also for s = +-700, where the Gram matrices of the unscaled
  input would overflow or underflow and only the initial scaling keeps them
  in range.
* Columns of norms 1e-150 .. 1e+150 with disjoint supports (exactly
  orthogonal): the singular values are the column norms, against binary128.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_1401_2720_gb300 import inputs as I
from paper_1401_2720_gb300 import jsvd as J
from tests.test_gpu_svd import _np, _t

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


def test_column_sumsq_against_oracle(cuda):
    rng = np.random.default_rng(4)
    m = 333
    cols = [rng.standard_normal(m) * s for s in (1.0, 1e200, 1e-200, 1e300, 1e-300, 1e-310)]
    mixed = rng.standard_normal(m)
    mixed[::3] *= 1e250
    mixed[1::3] *= 1e-250
    cols += [mixed, np.zeros(m)]
    A = np.asfortranarray(np.stack(cols, axis=1))
    e, f = J.column_sumsq(_t(A, cuda))
    e, f = _np(e), _np(f)
    for j in range(A.shape[1]):
        eo, fo = O.drdssq(A[:, j])
        if fo == 0.0:
            assert f[j] == 0.0
            continue
        assert e[j] % 2 == 0 and 0.5 <= f[j] < 2.0
        assert abs(math.ldexp(f[j], int(e[j]) - eo) / fo - 1.0) <= m * EPS


@pytest.mark.parametrize("s", [700, -700, 500, -450])
@pytest.mark.parametrize("contraction", ["split", "fp64"])
def test_power_of_two_scaling_is_exact(cuda, s, contraction):
    A = I.graded_gaussian(300, 160, seed=9)
    U0, S0, V0 = J.svd(_t(A, cuda), b=16, contraction=contraction)
    U1, S1, V1 = J.svd(_t(np.ldexp(A, s), cuda), b=16, contraction=contraction)
    assert torch.equal(S1, torch.ldexp(S0, torch.tensor(s, device=cuda)))
    assert torch.equal(U1, U0) and torch.equal(V1, V0)


def test_power_of_two_scaling_hsvd_and_mixed(cuda):
    G = I.gaussian(200, 96, seed=7)
    a = J.hsvd(_t(G, cuda), 40, b=8)
    b = J.hsvd(_t(np.ldexp(G, -640), cuda), 40, b=8)
    assert torch.equal(b[1], torch.ldexp(a[1], torch.tensor(-640, device=cuda)))
    A = I.workload_mixed(256, 128, seed=3)[0]
    c = J.svd(_t(A, cuda), b=8, precision="mixed")
    d = J.svd(_t(np.ldexp(A, 120), cuda), b=8, precision="mixed")    # FP32 copies would overflow unscaled
    assert torch.equal(d[1], torch.ldexp(c[1], torch.tensor(120, device=cuda)))


def test_orthogonal_columns_spanning_300_decades(cuda):
    rng = np.random.default_rng(6)
    m, n = 256, 32
    A = np.zeros((m, n))
    for j in range(n):
        A[8 * j:8 * j + 8, j] = rng.standard_normal(8) * 10.0 ** (150 - 300 * j / (n - 1))
    A = np.asfortranarray(A)
    U, S, V = J.svd(_t(A, cuda), b=8)
    S = _np(S)
    ref = []
    for j in range(n):
        e, f = O.q_sumsq(A[:, j])
        ref.append(math.sqrt(f) * 2.0 ** (e / 2) if e % 2 == 0 else math.sqrt(2 * f) * 2.0 ** ((e - 1) / 2))
    ref = np.sort(np.array(ref))[::-1]
    assert np.all(np.abs(S - ref) <= 4 * EPS * ref)
