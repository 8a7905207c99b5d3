"""The block-width autotuner returns a valid width per populated bucket, and
the batched solve with the tuned per-matrix widths matches LAPACK."""
import numpy as np
import pytest

from paper_1401_2720_gb300 import autotune
from paper_1401_2720_gb300 import inputs as I
from paper_1401_2720_gb300 import jsvd as J
from tests.test_gpu_svd import _np

pytestmark = pytest.mark.gpu


def test_autotune_table_and_tuned_solve(cuda):
    mats, _, _, _ = I.workload_batch(48, seed=21, m_hi=200)
    table = autotune.tune(mats, sample=12, repeats=1)
    populated = {autotune.bucket_of(a.shape[1]) for a in mats}
    assert set(table) >= populated and all(v in (8, 16, 32) for v in table.values())
    pk = J.Packing([a.shape[0] for a in mats], [a.shape[1] for a in mats])
    b = autotune.block_widths(pk.n, table)
    U, S, V, infos, rc = J.svd_batched_packed(pk, pk.pack(mats, cuda), b=b, return_info=True)
    assert rc == 0 and [i["b"] for i in infos] == list(b)
    for a, s in zip(mats, pk.unpack_n(S)):
        sl = np.linalg.svd(a, compute_uv=False)
        assert np.max(np.abs(_np(s) - sl)) <= 1e-12 * sl[0]


def test_autotune_strategy(cuda):
    mats, _, _, _ = I.workload_batch(40, seed=23, m_hi=160)
    table = autotune.tune(mats, sample=10, repeats=1)
    best, times = autotune.tune_strategy(mats, table, sample=20, repeats=1)
    assert best in ("rR", "rC", "modulus") and set(times) == {"rR", "rC", "modulus"}
    assert times[best] == min(times.values())
    pk = J.Packing([a.shape[0] for a in mats], [a.shape[1] for a in mats])
    U, S, V, infos, rc = J.svd_batched_packed(pk, pk.pack(mats, cuda), b=autotune.block_widths(pk.n, table),
                                              strategy=best, return_info=True)
    assert rc == 0
    for a, s in zip(mats, pk.unpack_n(S)):
        sl = np.linalg.svd(a, compute_uv=False)
        assert np.max(np.abs(_np(s) - sl)) <= 1e-12 * sl[0]
