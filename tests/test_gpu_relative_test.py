"""The relative orthogonality test of Sec. 4.3 as the sweep kernels evaluate it
(squares compared first, square roots only inside a guard band) gives the
same decision, bit for bit, as the correctly rounded definition
|h_pq| >= c(eps) * (sqrt(h_pp) * sqrt(h_qq)) evaluated on the CPU."""
import numpy as np
import pytest
import torch

from paper_1401_2720_gb300 import jsvd as J

pytestmark = pytest.mark.gpu


def _cpu(hpp, hqq, hpq, c):
    a = np.abs(hpq)
    return (a != 0.0) & ~(a < c * (np.sqrt(hpp) * np.sqrt(hqq)))


@pytest.mark.parametrize("bb", [16, 32, 64])
def test_relative_test_matches_definition(cuda, bb):
    c = 2.0 ** -53 * np.sqrt(float(bb))
    rng = np.random.default_rng(bb)
    n = 200_000
    hpp = 10.0 ** rng.uniform(-30, 30, n)
    hqq = 10.0 ** rng.uniform(-30, 30, n)
    thr = c * (np.sqrt(hpp) * np.sqrt(hqq))
    # a third random, a third at the threshold within a few ulps, a third scaled
    # by factors across the guard band (1 +- 2^-48)
    k = rng.integers(-40, 41, n).astype(np.float64)
    near = thr * (1.0 + k * 2.0 ** -53)
    band = thr * (1.0 + rng.uniform(-2.0 ** -46, 2.0 ** -46, n))
    pick = rng.integers(0, 3, n)
    hpq = np.where(pick == 0, thr * 10.0 ** rng.uniform(-3, 3, n), np.where(pick == 1, near, band))
    hpq *= rng.choice([-1.0, 1.0], n)
    # exact threshold values, zeros, and exponents outside the fast range
    hpq[:1000] = thr[:1000]
    hpq[1000:1100] = 0.0
    hpp[1100:1200] = 10.0 ** rng.uniform(130, 150, 100)
    hqq[1200:1300] = 10.0 ** rng.uniform(-150, -130, 100)
    hpp[1300:1310] = 0.0
    hpq[1100:1300] = c * (np.sqrt(hpp[1100:1300]) * np.sqrt(hqq[1100:1300])) * (1 + rng.integers(-3, 4, 200) * 2.0 ** -52)
    want = _cpu(hpp, hqq, hpq, c)
    t = lambda x: torch.from_numpy(x).to(cuda)
    got = J.relative_test(t(hpp), t(hqq), t(hpq), c).cpu().numpy()
    assert np.array_equal(got, want), int(np.sum(got != want))
    # both outcomes occur near the threshold
    assert want[pick == 1].any() and (~want[pick == 1]).any()
