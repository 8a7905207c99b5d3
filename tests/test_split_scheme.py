"""The arithmetic of the split-digit contractions, modelled exactly on the CPU.

The tensor-core Gram forms each FP64 product from 9 balanced 7-bit digits of
power-of-two scaled fixed-point operands and accumulates the 45 digit
products with i + l <= 8 per level in FP32; the tcgen05 update uses 8
balanced 8-bit digits and the 36 products with i + l <= 7 (8 level
accumulators of 64 columns fill the 512 TMEM columns).  Both recombine the
levels into one FP64 number (see the device headers that implement them).  This model uses Python
integers for the exact parts, so it checks the scheme's claims independently
of the GPU code: the digit bias and ranges, that every level sum is an integer
small enough for exact FP32 accumulation, and that the result is at least as
accurate, column by column, as an FP64 dot product of the same length.
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

S = 9                                   # digits of the 7-bit scheme
BIAS = sum(64 * 128 ** k for k in range(S))
S8 = 8                                  # digits of the 8-bit scheme
BIAS8 = sum(128 * 256 ** k for k in range(S8))


def fixed(x: float, E: int) -> int:
    """trunc(x 2^(62 - E)) for |x| < 2^E."""
    return int(Fraction(x) * Fraction(2) ** (62 - E))


def digits(Y: int) -> list[int]:
    Z = Y + BIAS
    assert 0 <= Z < 2 ** 64
    top = (Z >> 56) - 64
    rest = [((Z >> (56 - 7 * i)) & 127) - 64 for i in range(1, S)]
    return [top] + rest


def digits8(Y: int) -> list[int]:
    Z = Y + BIAS8
    assert 0 <= Z < 2 ** 64
    return [((Z >> (56 - 8 * i)) & 255) - 128 for i in range(S8)]


def exp_bound(v) -> int:
    m = float(np.max(np.abs(v)))
    return int(np.frexp(m)[1]) if m > 0 else 0


def split_product(A: np.ndarray, B: np.ndarray, dscale: bool = True, eight_bit: bool = False):
    """A @ B by the scheme (7-bit digits, 9 slices; or 8-bit digits, 8
    slices); returns (result, max |level sum|)."""
    m, K = A.shape
    N = B.shape[1]
    nd, base, dig = (S8, 256, digits8) if eight_bit else (S, 128, digits)
    if dscale:
        cn = np.sqrt((A * A).sum(0))
        dexp = np.where(cn > 0, np.round(np.log2(np.where(cn > 0, cn, 1))), 0).astype(int)
    else:
        dexp = np.zeros(K, int)
    A1 = A / 2.0 ** dexp[None, :]
    B1 = B * 2.0 ** dexp[:, None]
    Er = [exp_bound(A1[r]) for r in range(m)]
    Fk = [exp_bound(B1[:, k]) for k in range(N)]
    ad = [[dig(fixed(A1[r, j], Er[r])) for j in range(K)] for r in range(m)]
    bd = [[dig(fixed(B1[j, k], Fk[k])) for k in range(N)] for j in range(K)]
    out = np.zeros((m, N))
    lmax = 0
    for r in range(m):
        for k in range(N):
            lev = [sum(ad[r][j][i] * bd[j][k][L - i] for j in range(K) for i in range(L + 1)) for L in range(nd)]
            lmax = max(lmax, max(abs(v) for v in lev))
            T = sum(lev[L] * base ** (nd - 1 - L) for L in range(nd))          # exact
            # the top digit has weight 2^56 in both schemes:
            # 2^(E + F - 124) * 2^56 * T, rounded once
            out[r, k] = float(Fraction(T) * Fraction(2) ** (Er[r] + Fk[k] - 124 + 56))
    return out, lmax


def test_bias_and_digit_ranges():
    assert BIAS == 0x4081020408102040
    for Y in (0, 1, -1, 2 ** 62 - 1, -(2 ** 62 - 1), 123456789123456789, -987654321987654321):
        d = digits(Y)
        assert sum(di * 128 ** (S - 1 - i) for i, di in enumerate(d)) == Y
        assert -64 <= d[0] <= 64 and all(-64 <= di <= 63 for di in d[1:])


def test_bias_and_digit_ranges_8bit():
    assert BIAS8 == 0x8080808080808080
    for Y in (0, 1, -1, 2 ** 62 - 1, -(2 ** 62 - 1), 123456789123456789, -987654321987654321):
        d = digits8(Y)
        assert sum(di * 256 ** (S8 - 1 - i) for i, di in enumerate(d)) == Y
        assert -64 <= d[0] <= 64 and all(-128 <= di <= 127 for di in d[1:])


def test_level_sums_fit_fp32_8bit_update():
    # worst case: every digit product 128 * 128, 8 terms per level, K = 64
    assert 8 * 64 * 128 * 128 <= 2 ** 23
    rng = np.random.default_rng(1)
    A = rng.standard_normal((2, 64))
    B = np.linalg.qr(rng.standard_normal((64, 64)))[0][:, :2]
    _, lmax = split_product(A, B, eight_bit=True)
    assert lmax < 2 ** 23


def test_level_sums_fit_fp32_for_256_rows():
    # worst case: every digit product 64 * 64, 9 terms per level, 256 rows
    assert 9 * 256 * 64 * 64 < 2 ** 24
    rng = np.random.default_rng(0)
    A = rng.standard_normal((2, 256))
    _, lmax = split_product(A, A.T.copy(), dscale=False)
    assert lmax < 2 ** 24


@pytest.mark.parametrize("eight_bit", [False, True])
@pytest.mark.parametrize("kind", ["gaussian", "graded", "near_identity"])
def test_columnwise_error_at_most_fp64_dot(kind, eight_bit):
    """Against exact rational products: the scheme's worst column error (relative
    to the column norm) is below 1 ulp and no larger than that of FP64 products
    of the same operands (which reach 2.6-4.1 ulp on these inputs)."""
    rng = np.random.default_rng({"gaussian": 1, "graded": 2, "near_identity": 3}[kind])
    m, K = 12, 64
    A = rng.standard_normal((m, K))
    if kind != "gaussian":
        A *= 10.0 ** rng.uniform(-4, 0, K)[None, :]
    B = np.linalg.qr(rng.standard_normal((K, K)))[0][:, :8]
    if kind == "near_identity":
        B = (np.eye(K) + 1e-3 * rng.standard_normal((K, K)))[:, :8]
    exact = np.array([[float(sum(Fraction(A[r, j]) * Fraction(B[j, k]) for j in range(K)))
                       for k in range(B.shape[1])] for r in range(m)])
    got, _ = split_product(A, B, eight_bit=eight_bit)
    f64 = A @ B
    eps = 2.0 ** -53
    cn = np.linalg.norm(exact, axis=0)
    err_split = (np.linalg.norm(got - exact, axis=0) / cn).max() / eps
    err_f64 = (np.linalg.norm(f64 - exact, axis=0) / cn).max() / eps
    assert err_split <= 1.0
    assert err_split <= err_f64


def _stacked_gram_levels(Dg: np.ndarray, BB: int):
    """The tcgen05 Gram's accumulators for one 256-row chunk, modelled with
    integers: Dg[i, k, c] = digit i of row k, column c.  The A operand stacks
    SF = 128 / BB slices (slice g SF + s in rows s BB .. s BB + BB - 1), the
    B operand holds slices 0 .. 7 - g SF, and MMA g adds its products at
    column block g SF, so lane s BB + c, block j accumulates
    sum_{g SF <= j} sum_k d_{g SF + s}(k, c) d_{j - g SF}(k, n).  Returns the
    per-column sums [lane, block, n] and the levels assembled from them."""
    SF = 128 // BB
    acc = np.zeros((128, 8, BB), dtype=object)
    for g in range(8 // SF):
        for s in range(SF):
            for j in range(g * SF, 8):
                for c in range(BB):
                    acc[s * BB + c, j, :] += [int(Dg[g * SF + s, :, c] @ Dg[j - g * SF, :, n]) for n in range(BB)]
    lev = np.zeros((BB, BB, 8), dtype=object)
    for L in range(8):
        for s in range(SF):
            if L - s >= 0:
                lev[:, :, L] += acc[s * BB:(s + 1) * BB, L - s, :]
    return acc, lev


@pytest.mark.parametrize("BB", [16, 64])
@pytest.mark.parametrize("kind", ["coherent", "extreme"])
def test_stacked_gram_column_sums_exact_and_levels(BB, kind):
    """Every tensor-memory column of the stacked tcgen05 Gram sums at most
    8 / SF digit products over 256 rows, so it stays within 2^24 (exact in
    FP32) even for inputs whose digits add coherently (the assembled level
    sums then pass 2^24), and the assembled levels are the level sums
    sum_{i+l=L} sum_k d_i d_l."""
    from paper_1401_2720_gb300 import inputs as I
    if kind == "coherent":
        A = I.coherent_digit_columns(256, BB, seed=BB)
        Dg = np.array([[digits8(fixed(A[k, c], 0)) for k in range(256)] for c in range(BB)]).transpose(2, 1, 0)
    else:
        # the most negative digits (Y = -63 2^56 - sum_{i>0} 128 256^(7-i) > -2^62) in
        # every row and column: all products positive, the largest level sums
        Dg = np.full((8, 256, BB), -128)
        Dg[0] = -63
    Dg = Dg.astype(np.int64)
    acc, lev = _stacked_gram_levels(Dg, BB)
    assert max(abs(int(v)) for v in acc.flat) <= 2 ** 24
    for c in range(0, BB, 7):
        for n in range(0, BB, 5):
            for L in range(8):
                assert lev[c, n, L] == sum(int(Dg[i, :, c] @ Dg[L - i, :, n]) for i in range(L + 1))
    if kind == "extreme":
        assert max(abs(int(v)) for v in lev.flat) > 2 ** 24
    # the epilogue adds the level sums of up to 32 consecutive chunks of a pair
    # as int32 and recombines them with combine_levels (|lev| < 2^30): one
    # chunk's levels stay within 7 2^22 (only 6 of a level's 8 digit products
    # reach 2^14 per row, the other two hold d_0, |d_0| <= 64)
    assert max(abs(int(v)) for v in lev.flat) <= 7 * 2 ** 22
    assert 32 * max(abs(int(v)) for v in lev.flat) < 2 ** 30


def _combine_by_conversion(l, e):
    """The steps of split8::combine_levels: T = H 2^32 + R0 from the two
    half sums, |T| = M 2^32 + R, a right shift by k in {0, 8, 16, 24} to below
    2^64 with the discarded bits ORed into the last bit, one correctly rounded
    conversion to FP64 (Python's int -> float rounds to nearest, ties to even)
    and an exact power-of-two scale."""
    hi = l[0] * 2 ** 24 + l[1] * 2 ** 16 + l[2] * 2 ** 8 + l[3]
    lo = l[4] * 2 ** 24 + l[5] * 2 ** 16 + l[6] * 2 ** 8 + l[7]
    H, R0 = hi + (lo >> 32), lo & 0xFFFFFFFF
    neg = H < 0
    M = (~H if R0 else -H) if neg else H
    R = (-R0) & 0xFFFFFFFF if neg else R0
    assert 0 <= M < 2 ** 56
    k = ((M >> 32).bit_length() + 7) & ~7
    X = (M << (32 - k)) | (R >> k)
    assert X < 2 ** 64 and (k == 0 or X >= 2 ** 56)
    if R & ((1 << k) - 1):
        X |= 1
    r = math.ldexp(float(X), k + e - 68)
    return -r if neg else r


def test_combine_by_conversion_rounds_once():
    """The level recombination (rounding to odd at >= 57 bits, then one
    round-to-nearest conversion) equals T 2^(e-68) rounded once, ties to even:
    random levels up to the 2^30 bound, sparse levels, and constructed exact
    ties and near-ties of every magnitude up to 2^86, both signs."""
    rng = random.Random(7)

    def exact(l, e):
        T = sum(l[L] * 256 ** (7 - L) for L in range(8))
        return float(Fraction(T) * Fraction(2) ** (e - 68)) if T else 0.0

    cases = []
    for it in range(4000):
        bound = [2 ** 23, 2 ** 30 - 1, 300][it % 3]
        cases.append([rng.randint(-bound, bound) for _ in range(8)])
    for it in range(4000):
        bits = rng.randint(54, 86)
        s = bits - 53
        T = ((rng.getrandbits(52) | 2 ** 52) << s) + rng.choice([2 ** (s - 1), 2 ** (s - 1) - 1, 2 ** (s - 1) + 1])
        T = -T if it % 2 else T
        l = [0] * 8
        for L in range(7, 0, -1):
            l[L], T = T & 255, T >> 8
        l[0] = T
        cases.append(l)
    for l in cases:
        e = rng.randint(-150, 150)
        assert _combine_by_conversion(l, e) == exact(l, e), (l, e)
