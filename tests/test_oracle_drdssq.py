"""Pins of the oracle's DRDSSQ (App. A): the scaled sum of squares
||x||^2 = f 2^e (e even, 0.5 <= f < 2).  Where nothing over- or underflows
it equals the plain sum of squares to rounding; where the plain sum
overflows or underflows it equals the binary128 sum (exact range) to a few
units of 2^-53; partial sums of very different magnitudes (entries near
1e+-200 in one vector) are combined correctly."""
import math

import numpy as np
import pytest

import oracle as O

EPS = 2.0 ** -53


def _val_ratio(e1, f1, e2, f2):
    return math.ldexp(f1, e1 - e2) / f2


def test_common_form_and_plain_range():
    rng = np.random.default_rng(1)
    for n in (1, 7, 100, 1000):
        x = rng.standard_normal(n)
        e, f = O.drdssq(x)
        assert e % 2 == 0 and 0.5 <= f < 2.0
        plain = float(np.sum(x * x))
        assert math.ldexp(f, e) == pytest.approx(plain, rel=n * EPS)


def test_zero_vector():
    assert O.drdssq(np.zeros(5)) == (0, 0.0)


@pytest.mark.parametrize("scale", [1e154, 1e200, 1e300, 1e-154, 1e-200, 1e-300, 1e-315])
def test_beyond_the_plain_range_against_binary128(scale):
    rng = np.random.default_rng(2)
    x = rng.standard_normal(500) * scale
    e, f = O.drdssq(x)
    eq, fq = O.q_sumsq(x)
    assert abs(_val_ratio(e, f, eq, fq) - 1.0) <= 8 * 500 * EPS
    with np.errstate(over="ignore", under="ignore"):
        plain = float(np.sum(x * x))
    if scale >= 1e200:
        assert math.isinf(plain)           # the plain sum overflows here


def test_mixed_magnitudes_against_binary128():
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(300) * 1e200, rng.standard_normal(300),
                        rng.standard_normal(300) * 1e-200])
    rng.shuffle(x)
    e, f = O.drdssq(x)
    eq, fq = O.q_sumsq(x)
    assert abs(_val_ratio(e, f, eq, fq) - 1.0) <= 8 * 900 * EPS
