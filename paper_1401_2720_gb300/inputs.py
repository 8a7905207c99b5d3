"""Seeded synthetic inputs shaped like the workloads the benchmark and tests use.

This module holds none of the method's arithmetic; both the CUDA path's tests
and the oracle's tests draw their matrices from here.  All generators take a
``numpy.random.Generator`` (or a seed) and return column-major (Fortran-order)
float64 arrays.

Recipes:
  haar(n)            Haar-distributed orthogonal n x n: QR of an N(0,1) matrix
                     with the signs of diag(R) folded into Q (Mezzadri 2007).
  haar_thin(m, n)    the same for an m x n Gaussian (orthonormal columns).
  planted(m, n, s)   U diag(s) V^T with Haar U (thin) and V.
  geometric(n, hi, lo)        s_i = hi * (lo/hi)^((i-1)/(n-1)).
  graded_gaussian(m, n)       N(0,1) entries, column j scaled by 10^u_j,
                              u_j ~ U(-4, 0).
  loguniform_sorted(n, lo, hi, min_gap)  log-uniform values sorted
                              non-increasingly with relative gaps >= min_gap.
  batch_shapes(count)         m ~ U{16..512}, n ~ U{8..m}.
  graded_columns(m, n, decades)  N(0,1) entries, column j scaled by
                              10^(-decades j/(n-1)) (no two norms nearly tie).
  duplicated_pm1_column(A, j0, j1, count)  column j0 := `count` entries +-1
                              (the rest 0), column j1 := column j0.
"""

from __future__ import annotations

import numpy as np


def rng_of(seed) -> np.random.Generator:
    return seed if isinstance(seed, np.random.Generator) else np.random.default_rng(seed)


def haar_thin(m: int, n: int, seed=0) -> np.ndarray:
    rng = rng_of(seed)
    Z = rng.standard_normal((m, n))
    Q, R = np.linalg.qr(Z)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return np.asfortranarray(Q * d[None, :])


def haar(n: int, seed=0) -> np.ndarray:
    return haar_thin(n, n, seed)


def geometric(n: int, hi: float = 1.0, lo: float = 1e-8) -> np.ndarray:
    if n == 1:
        return np.array([hi])
    return hi * (lo / hi) ** (np.arange(n) / (n - 1))


def planted(m: int, n: int, sigma, seed=0) -> np.ndarray:
    """A = U diag(sigma) V^T, U m x n with orthonormal columns, V n x n orthogonal."""
    rng = rng_of(seed)
    U = haar_thin(m, n, rng)
    V = haar(n, rng)
    return np.asfortranarray((U * np.asarray(sigma)[None, :]) @ V.T)


def gaussian(m: int, n: int, seed=0) -> np.ndarray:
    return np.asfortranarray(rng_of(seed).standard_normal((m, n)))


def graded_gaussian(m: int, n: int, seed=0, lo: float = -4.0, hi: float = 0.0) -> np.ndarray:
    rng = rng_of(seed)
    Z = rng.standard_normal((m, n))
    u = rng.uniform(lo, hi, size=n)
    return np.asfortranarray(Z * (10.0 ** u)[None, :])


def loguniform_sorted(n: int, lo: float, hi: float, seed=0, min_gap: float = 0.0) -> np.ndarray:
    """Log-uniform values on [lo, hi], sorted non-increasingly, then pushed
    down so that (s_i - s_{i+1}) / s_i >= min_gap; a draw whose tail falls
    below lo is redrawn."""
    rng = rng_of(seed)
    for _ in range(1000):
        s = np.sort(10.0 ** rng.uniform(np.log10(lo), np.log10(hi), size=n))[::-1].copy()
        for i in range(1, n):
            s[i] = min(s[i], s[i - 1] * (1.0 - min_gap))
        if s[-1] >= lo:
            return s
    raise RuntimeError("could not draw a spectrum with the requested gaps")


def batch_shapes(count: int, seed=0, m_lo: int = 16, m_hi: int = 512, n_lo: int = 8):
    rng = rng_of(seed)
    ms = rng.integers(m_lo, m_hi + 1, size=count)
    ns = np.array([rng.integers(n_lo, m + 1) for m in ms])
    return ms.astype(np.int64), ns.astype(np.int64)


# --- the named workloads --------------------------------------------------
def workload_small_planted(seed=0):
    """512 x 256, s geometric from 1 to 1e-8, Haar U and V."""
    return planted(512, 256, geometric(256, 1.0, 1e-8), seed)


def workload_graded_square(n: int = 8192, seed=0):
    """n x n N(0,1), column j scaled by 10^u_j, u_j ~ U(-4, 0)."""
    return graded_gaussian(n, n, seed)


def workload_hsvd_square(n: int = 4096, seed=0):
    """n x n N(0,1) with J = diag(+1 x n/2, -1 x n/2): returns (G, n_plus)."""
    return gaussian(n, n, seed), n // 2


def workload_mixed(m: int = 8192, n: int = 4096, seed=0):
    """m x n, s_i = 10^(-12 x_i) with x_i ~ U(0,1) sorted, Haar U and V."""
    rng = rng_of(seed)
    x = np.sort(rng.uniform(0.0, 1.0, size=n))
    s = 10.0 ** (-12.0 * x)
    return planted(m, n, s, rng), s


def workload_batch(count: int = 4096, seed=0, m_hi: int = 512):
    """count matrices, m ~ U{16..m_hi}, n ~ U{8..m}, s log-uniform on
    [1e-6, 1] with relative gaps >= 1e-3, Haar U and V; plus the loss data
    w ~ N(0,1) (length n) and C ~ N(0,1) (m x n) of each matrix."""
    rng = rng_of(seed)
    ms, ns = batch_shapes(count, rng, m_hi=m_hi)
    mats, sig, ws, Cs = [], [], [], []
    for m, n in zip(ms, ns):
        s = loguniform_sorted(int(n), 1e-6, 1.0, rng, min_gap=1e-3)
        mats.append(planted(int(m), int(n), s, rng))
        sig.append(s)
        ws.append(rng.standard_normal(int(n)))
        Cs.append(np.asfortranarray(rng.standard_normal((int(m), int(n)))))
    return mats, sig, ws, Cs


def graded_columns(m: int, n: int, decades: float = 4.0, seed=0) -> np.ndarray:
    rng = rng_of(seed)
    scale = 10.0 ** (-decades * np.arange(n) / max(n - 1, 1))
    return np.asfortranarray(rng.standard_normal((m, n)) * scale[None, :])


def duplicated_pm1_column(A, j0: int, j1: int, count: int = 16, seed=0) -> np.ndarray:
    """A copy of A whose column j0 holds `count` entries +-1 at random rows
    (zeros elsewhere) and whose column j1 is an exact copy of column j0."""
    rng = rng_of(seed)
    B = np.array(A, dtype=np.float64, order="F", copy=True)
    B[:, j0] = 0.0
    rows = rng.choice(B.shape[0], count, replace=False)
    B[rows, j0] = rng.choice([-1.0, 1.0], count)
    B[:, j1] = B[:, j0]
    return np.asfortranarray(B)


def coherent_digit_columns(m: int, n: int, seed=0) -> np.ndarray:
    """A_kj = s_k y_j + M_kj / 16 with signs s_k = +-1, integers M_kj in
    [-3, 3] and y_j = t_j 2^-62, t_j = 0x207F7F7F7F7F7C00 + 2^50 j (exact
    doubles in [0.5, 0.6)).  Every entry's fixed-point value trunc(x 2^62)
    shares the bytes 0x7F of t_j below the top one, with the row's sign, so
    products of the 8-bit digits add up coherently over the rows: level sums of
    a 256-row contraction reach ~2^24, the largest the digit form must carry
    exactly.  The random integer part (top digit only) keeps the matrix well
    conditioned."""
    rng = rng_of(seed)
    t = np.array([0x207F7F7F7F7F7C00 + (j << 50) for j in range(n)], dtype=np.float64)
    y = np.ldexp(t, -62)
    s = rng.choice([-1.0, 1.0], m)
    M = rng.integers(-3, 4, size=(m, n)).astype(np.float64)
    return np.asfortranarray(s[:, None] * y[None, :] + M / 16.0)
