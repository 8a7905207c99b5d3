"""The no-allocation entry point (jsvd_dgesvj_noalloc) against the regular
allocating one (jsvd_dgesvj), through the C ABI, on two calls in a row.

This file is collected last on purpose: it exercises a library-wide static
device array that every call shares, so a run that stops at the first failure
has already run every other test.  It must pass alone in a fresh process too.
Tolerances are those of the FP64 parity tests: normwise sigma <= 1e-12,
orthogonality <= 50 n 2^-53; the two entry points run the same kernels on the
same inputs, so U, S, V are also compared element by element (<= 1e-12).
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1401_2720_gb300 import build_ext
from paper_1401_2720_gb300 import inputs as I
from paper_1401_2720_gb300 import jsvd as J

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


@pytest.fixture(scope="module")
def lib(cuda):
    build_ext.build()
    return J.library()


def _noalloc(lib, A, b, want_v=True, want_info=True, S=None):
    """Call jsvd_dgesvj_noalloc through ctypes on torch-owned buffers, on
    torch's current stream."""
    m, n = A.shape
    Ac = A.t().contiguous()                              # column-major m x n, ld = m
    U = torch.empty((n, m), dtype=torch.float64, device=A.device)
    if S is None:
        S = torch.empty(n, dtype=torch.float64, device=A.device)
    V = torch.empty((n, n), dtype=torch.float64, device=A.device) if want_v else None
    opts = J.make_opts(b=b)
    info = J.Info()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.jsvd_dgesvj_noalloc(m, n, Ac.data_ptr(), m, S.data_ptr(), U.data_ptr(), m,
                                 V.data_ptr() if want_v else None, n, ctypes.byref(opts),
                                 ctypes.byref(info) if want_info else None, stream)
    torch.cuda.current_stream().synchronize()
    return rc, U.t(), S, (V.t() if want_v else None), info


def test_no_alloc_matches_regular_entry_point_twice(lib, cuda):
    # two calls in a row, different shapes: the second finds the first's
    # contents in the shared array and must not depend on them
    for call, (m, n, b) in enumerate([(400, 272, 16), (300, 200, 8)]):
        A = torch.from_numpy(np.ascontiguousarray(I.graded_gaussian(m, n, seed=10 + call))).to(cuda)
        rc, U, S, V, info = _noalloc(lib, A, b)
        assert rc == 0 and info.converged
        U1, S1, V1 = J.svd(A, b=b)
        assert float((S - S1).abs().max()) <= 1e-12 * float(S1[0])
        assert float((U - U1).abs().max()) <= 1e-12
        assert float((V - V1).abs().max()) <= 1e-12
        eye = torch.eye(n, dtype=torch.float64, device=cuda)
        assert float((U.t() @ U - eye).abs().max()) <= 50 * n * EPS
        assert float((V.t() @ V - eye).abs().max()) <= 50 * n * EPS


def test_no_alloc_partial_svd_on_a_side_stream(lib, cuda):
    """V = NULL (no right vectors: no V workspace is carved, so the scratch
    layout differs) and info = NULL, issued on a non-default stream."""
    m, n, b = 360, 240, 16
    A = torch.from_numpy(np.ascontiguousarray(I.graded_gaussian(m, n, seed=21))).to(cuda)
    U1, S1, V1 = J.svd(A, b=b)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        rc, U, S, V, _ = _noalloc(lib, A, b, want_v=False, want_info=False)
    assert rc == 0 and V is None
    assert float((S - S1).abs().max()) <= 1e-12 * float(S1[0])
    assert float((U - U1).abs().max()) <= 1e-12


def test_no_alloc_rejects_a_problem_beyond_its_scratch(lib, cuda):
    A = torch.zeros((2048, 2048), dtype=torch.float64, device=cuda)
    S = torch.full((2048,), -7.25, dtype=torch.float64, device=cuda)     # sentinel
    rc, U, S, V, info = _noalloc(lib, A, 16, S=S)
    assert rc == 7                                        # JSVD_ERR_TOO_LARGE
    assert lib.jsvd_status_string(rc)
    assert bool(torch.all(S == -7.25))                    # outputs untouched
