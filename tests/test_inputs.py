"""The seeded workload generators produce the structure their recipes state
(sizes, distributions, planted spectra, gaps), deterministically per seed."""
import numpy as np

from paper_1401_2720_gb300 import inputs as I

EPS = 2.0 ** -53


def test_haar_factors_are_orthogonal_and_seeded():
    Q = I.haar_thin(50, 20, seed=1)
    assert np.abs(Q.T @ Q - np.eye(20)).max() <= 50 * EPS * 20
    assert np.array_equal(Q, I.haar_thin(50, 20, seed=1)) and not np.array_equal(Q, I.haar_thin(50, 20, seed=2))
    assert Q.flags.f_contiguous


def test_planted_spectrum():
    s = I.geometric(24, 1.0, 1e-6)
    assert s[0] == 1.0 and abs(s[-1] - 1e-6) <= 1e-20 and np.all(np.diff(s) < 0)
    A = I.planted(60, 24, s, seed=4)
    sl = np.linalg.svd(A, compute_uv=False)
    assert np.max(np.abs(sl - s)) <= 100 * EPS


def test_graded_columns_span_the_stated_decades():
    A = I.graded_gaussian(4000, 64, seed=0)
    # column RMS = 10^u_j (up to sampling noise), u_j in [-4, 0)
    u = np.log10(np.sqrt((A ** 2).mean(axis=0)))
    assert u.min() > -4.2 and u.max() < 0.1 and u.max() - u.min() > 2.5


def test_mixed_spectrum_range():
    A, s = I.workload_mixed(300, 40, seed=5)
    assert np.all(np.diff(s) <= 0) and s[0] <= 1.0 and s[-1] >= 1e-12
    sl = np.linalg.svd(A, compute_uv=False)
    assert np.max(np.abs(sl - s)) <= 100 * EPS


def test_batch_shapes_and_gaps():
    mats, sig, ws, Cs = I.workload_batch(40, seed=7, m_hi=120)
    for A, s, w, C in zip(mats, sig, ws, Cs):
        m, n = A.shape
        assert 16 <= m <= 120 and 8 <= n <= m
        assert s[0] <= 1.0 and s[-1] >= 1e-6 and np.all((s[:-1] - s[1:]) / s[:-1] >= 1e-3 * (1 - 1e-12))
        assert w.shape == (n,) and C.shape == (m, n)
        assert np.max(np.abs(np.linalg.svd(A, compute_uv=False) - s)) <= 100 * EPS
