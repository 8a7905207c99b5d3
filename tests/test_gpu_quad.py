"""The GPU path against the oracle's binary128 build (the exact answer for
these inputs, to far below FP64 rounding).

* The 512 x 256 planted matrix (sigma geometric 1 .. 1e-8, Haar U, V, b = 16,
  modulus ordering): normwise |s - s_q| / s_1 <= 1e-12, and per sigma the
  GPU is as accurate as the FP64 oracle: |s - s_q| / s_q <= max(1e-12,
  10 x the FP64 oracle's own relative error against s_q, smoothed over
  +-0.5 decades).
* The adjoint of the batched workload's loss L = sum w_i s_i + <C, U V^T> at
  its spectra (log-uniform on [1e-6, 1], relative gaps >= 1e-3) against
  binary128 central differences, <dA, E> within 1e-6 relative, on a seeded
  sample of 16 matrices with m <= 64 (FP64 differences cannot resolve
  absolute gaps of 1e-9).
"""
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_1401_2720_gb300 import inputs as I
from paper_1401_2720_gb300 import jsvd as J
from tests.test_gpu_svd import _np, _t, smoothed_floor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def threads():
    O.set_threads(os.cpu_count() or 1)
    yield
    O.set_threads(1)


@pytest.mark.parametrize("contraction", ["split", "fp64"])
def test_small_planted_against_binary128(cuda, contraction):
    A = I.workload_small_planted(seed=0)
    _, Sq, _, ok = O.q_svd(A, strategy="modulus", with_vectors=False)
    assert ok
    U, S, V, info = J.svd(_t(A, cuda), b=16, strategy="modulus", return_info=True, contraction=contraction)
    assert info["converged"]
    S = _np(S)
    _, So, _, _ = O.svd(A, strategy="modulus")
    assert np.max(np.abs(S - Sq)) <= 1e-12 * Sq[0]
    floor = smoothed_floor(Sq, So)          # the FP64 oracle's relative error against the exact values
    assert np.all(np.abs(S - Sq) / Sq <= np.maximum(1e-12, 10 * floor))


def test_adjoint_against_binary128_differences_at_batch_gaps(cuda):
    mats, sig, ws, Cs = I.workload_batch(16, seed=77, m_hi=64)
    pk = J.Packing([a.shape[0] for a in mats], [a.shape[1] for a in mats])
    U, S, V = J.svd_batched_packed(pk, pk.pack(mats, cuda))
    Us, Vs = pk.unpack_mn(U), pk.unpack_nn(V)
    dU = torch.cat([torch.from_numpy(C).to(cuda).mm(v).t().reshape(-1) for C, v in zip(Cs, Vs)])
    dV = torch.cat([torch.from_numpy(C).to(cuda).t().mm(u).t().reshape(-1) for C, u in zip(Cs, Us)])
    dS = torch.cat([torch.from_numpy(w).to(cuda) for w in ws])
    dA = pk.unpack_mn(J.svd_backward_packed(pk, U, S, V, dU, dS, dV))
    # absolute gaps down to ~2e-8 s_1 (relative 1e-3 near s = 1e-6) are present
    assert min(np.min(s[:-1] - s[1:]) / s[0] for s in sig) < 1e-7
    rng = np.random.default_rng(78)
    worst = 0.0
    for a, w, C, g, s in zip(mats, ws, Cs, dA, sig):
        g = _np(g)
        for _ in range(2):
            E = rng.standard_normal(a.shape)
            fd = O.q_loss_fd(a, E, 2.0 ** -44, w, C, strategy="modulus")
            rel = abs(float(np.sum(g * E)) - fd) / max(abs(fd), 1e-300)
            worst = max(worst, rel)
    assert worst <= 1e-6, worst
