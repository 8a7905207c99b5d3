"""Full-size GPU checks at the benchmark's workloads and launch configuration.

The oracle cannot run at these sizes, so these tests use properties that hold
at any size (with the gates of the smaller parity tests):
  * reconstruction ||A - U S V^T||_F / ||A||_F and orthogonality of U, V
    (HSVD: V^T J V = J) within 50 n 2^-53 (max-abs entries);
  * residuals ||A v_i - s_i u_i|| and ||A^T u_i - s_i v_i|| for sampled i
    (HSVD: ||G v_i - s_i u_i||, the right vectors are J-orthogonal);
  * sigma^2 against the eigenvalues of A^T A (HSVD: s_i^2 j_i against those of
    G J G^T) from a library eigensolver (cuSOLVER through torch), normwise;
  * mixed precision: sigma within 1e-12 (normwise) of the planted values.
"""
import numpy as np
import pytest
import torch

from paper_1401_2720_gb300 import inputs as I
from paper_1401_2720_gb300 import jsvd as J

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


def _dev(A, cuda):
    return torch.from_numpy(np.ascontiguousarray(A.T)).to(cuda).t()


def _checks(A, U, S, V, n):
    eye = torch.eye(n, dtype=torch.float64, device=A.device)
    assert float((U.t() @ U - eye).abs().max()) <= 50 * n * EPS
    assert float((V.t() @ V - eye).abs().max()) <= 50 * n * EPS
    R = A - (U * S) @ V.t()
    assert float(torch.linalg.norm(R) / torch.linalg.norm(A)) <= 50 * n * EPS
    idx = torch.linspace(0, n - 1, 64, device=A.device).long()
    r1 = torch.linalg.norm(A @ V[:, idx] - U[:, idx] * S[idx], dim=0)
    r2 = torch.linalg.norm(A.t() @ U[:, idx] - V[:, idx] * S[idx], dim=0)
    assert float(torch.max(r1.max(), r2.max())) <= 50 * n * EPS * float(S[0])
    assert bool(torch.all(S[:-1] >= S[1:]))


def test_graded_8192_bench_configuration(cuda):
    """The benchmark's workload and launch configuration (b = 32, reverse R||)."""
    n = 8192
    A = _dev(I.workload_graded_square(n, seed=0), cuda)
    U, S, V, info = J.svd(A, b=32, strategy="rR", return_info=True)
    assert info["converged"] and info["breakdowns"] == 0
    _checks(A, U, S, V, n)
    lam = torch.linalg.eigvalsh(A.t() @ A).flip(0)
    assert float((S * S - lam).abs().max()) <= 1e-12 * float(lam[0])


def test_hsvd_4096_configuration(cuda):
    n = 4096
    G0, npl = I.workload_hsvd_square(n, seed=0)
    G = _dev(G0, cuda)
    U, S, V, info = J.hsvd(G, npl, b=32, return_info=True)
    assert info["converged"]
    j = torch.where(torch.arange(n, device=cuda) < npl, 1.0, -1.0).to(torch.float64)
    Jm = torch.diag(j)
    nv = float(torch.linalg.matrix_norm(V, ord=2)) ** 2
    assert float((V.t() @ Jm @ V - Jm).abs().max()) <= 50 * n * EPS * nv
    eye = torch.eye(n, dtype=torch.float64, device=cuda)
    assert float((U.t() @ U - eye).abs().max()) <= 50 * n * EPS
    R = G - (U * S) @ V.t()
    assert float(torch.linalg.norm(R) / torch.linalg.norm(G)) <= 50 * n * EPS * nv
    # s_i^2 j_i are the eigenvalues of G J G^T (square G: all n of them)
    lam = torch.linalg.eigvalsh(G @ Jm @ G.t())
    mine = torch.sort(S * S * j).values
    assert float((mine - lam).abs().max()) <= 1e-11 * float(lam.abs().max())


def test_mixed_8192x4096_configuration(cuda):
    m, n = 8192, 4096
    A0, s_true = I.workload_mixed(m, n, seed=0)
    A = _dev(A0, cuda)
    U, S, V, info = J.svd(A, b=32, precision="mixed", return_info=True)
    assert info["converged"] and info["sweeps_low"] >= 1
    _checks(A, U, S, V, n)
    s_true = torch.from_numpy(np.sort(s_true)[::-1].copy()).to(cuda)
    assert float((S - s_true).abs().max()) <= 1e-12 * float(s_true[0])
