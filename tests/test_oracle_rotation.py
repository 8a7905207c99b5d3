"""Pins of the oracle's rotation formulas, Eqs. (4.3)-(4.6) of the paper."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from tests.conftest import GOLDEN

EPS = 2.0 ** -53


def _rng(seed=0):
    return np.random.default_rng(seed)


def _spd2(rng, n):
    """Random 2x2 Gram data (hpp, hqq, hpq) of random column pairs."""
    g = rng.standard_normal((n, 2, 7)) * 10.0 ** rng.uniform(-3, 3, size=(n, 2, 1))
    hpp = np.einsum("ij,ij->i", g[:, 0], g[:, 0])
    hqq = np.einsum("ij,ij->i", g[:, 1], g[:, 1])
    hpq = np.einsum("ij,ij->i", g[:, 0], g[:, 1])
    return hpp, hqq, hpq


def test_trig_diagonalises_2x2():
    """V^T H V is diagonal and its diagonal is the pair of eigenvalues of H
    (numpy.linalg.eigvalsh); cos^2 (1 + tan^2) = 1."""
    rng = _rng(1)
    hpp, hqq, hpq = _spd2(rng, 2000)
    cs, tn, _ = O.rotation(hpp, hqq, hpq, hyperbolic=False)
    for a, d, c, C, T in zip(hpp, hqq, hpq, cs, tn):
        H = np.array([[a, c], [c, d]])
        Vr = C * np.array([[1.0, T], [-T, 1.0]])          # Eq. (4.1)
        D = Vr.T @ H @ Vr
        scale = np.linalg.norm(H)
        assert abs(D[0, 1]) <= 64 * EPS * scale
        ev = np.sort(np.linalg.eigvalsh(H))
        assert np.allclose(np.sort(np.diag(D)), ev, rtol=0, atol=64 * EPS * scale)
        # diagonal update used by the sort (reading: hpp - tan*hpq, hqq + tan*hpq)
        assert abs((a - T * c) - D[0, 0]) <= 64 * EPS * scale
        assert abs((d + T * c) - D[1, 1]) <= 64 * EPS * scale
        assert abs(C * C * (1 + T * T) - 1) <= 8 * EPS
        assert abs(T) <= 1.0


def test_hyperbolic_diagonalises_and_is_j_orthogonal():
    """Eq. (4.2): V^T H V diagonal, V^T J V = J, cosh^2 (1 - tanh^2) = 1."""
    rng = _rng(2)
    hpp, hqq, hpq = _spd2(rng, 2000)
    cs, tn, _ = O.rotation(hpp, hqq, hpq, hyperbolic=True)
    J = np.diag([1.0, -1.0])
    for a, d, c, C, T in zip(hpp, hqq, hpq, cs, tn):
        H = np.array([[a, c], [c, d]])
        Vh = C * np.array([[1.0, T], [T, 1.0]])
        ct2 = -(a + d) / (2 * c)
        if abs(ct2) <= 1.0 + 1e-12:
            continue                       # the 5/4 substitution, tested below
        D = Vh.T @ H @ Vh
        cond = np.linalg.norm(Vh) ** 2
        assert abs(D[0, 1]) <= 256 * EPS * cond * np.linalg.norm(H)
        assert np.allclose(Vh.T @ J @ Vh, J, rtol=0, atol=64 * EPS * cond)
        assert abs(C * C * (1 - T * T) - 1) <= 64 * EPS * C * C
        assert abs(T) < 1.0


def test_shortcut_branches():
    # |cot 2phi| >= sqrt(2/eps) = 2^27: |cot phi| = 2|cot 2phi|, cos = 1
    cs, tn, pr = O.rotation(0.0, 2.0 ** 29, 1.0)          # ct2 = 2^28
    assert cs[0] == 1.0 and tn[0] == 1.0 / 2.0 ** 29 and not pr[0]
    # |cot 2phi| < sqrt(eps), trigonometric: |cot phi| = |cot 2phi| + 1
    ct2 = 1e-9
    cs, tn, pr = O.rotation(1.0, 1.0 + 2 * ct2, 1.0)
    h = (1.0 + 2 * ct2) - 1.0
    assert tn[0] == 1.0 / (abs(h / 2.0) + 1.0) and pr[0]
    # ct2 = 0 (equal diagonal): phi = pi/4, tan = sgn(hpq) (copysign reading)
    cs, tn, _ = O.rotation(3.0, 3.0, 0.5)
    assert tn[0] == 1.0 and cs[0] == 1.0 / np.sqrt(2.0)
    cs, tn, _ = O.rotation(3.0, 3.0, -0.5)
    assert tn[0] == -1.0
    # hyperbolic |coth 2phi| <= 1 -> 5/4: |coth phi| = 5/4 + 3/4 = 2
    cs, tn, _ = O.rotation(1.0, 1.0, -1.0, hyperbolic=True)
    assert tn[0] == 0.5 and cs[0] == 2.0 / np.sqrt(3.0)


def _departure_mean(t, cs_form, exps, per, seed):
    rng = np.random.default_rng(seed)
    tot, cnt = Fraction(0), 0
    for e in exps:
        mant = rng.integers(0, 2 ** 52, size=per, dtype=np.int64)
        ct2 = np.array([np.ldexp(1.0 + float(x) / 2 ** 52, int(e)) for x in mant])
        # choose hpp = 0, hqq = ct2 and hpq = t/2 so that (4.3) gives exactly ct2
        cs, tn, _ = O.rotation(np.zeros_like(ct2), ct2, np.full_like(ct2, 0.5 * t),
                               hyperbolic=(t < 0), cs_form=cs_form)
        for c, s in zip(cs, tn):
            c, s = Fraction(c), Fraction(s)
            d = c * c * (1 + s * s) - 1 if t > 0 else c * c * (1 - s * s) - 1
            tot += abs(d)
            cnt += 1
    return float(tot / cnt)


def test_table_b1_departures():
    """App. B, Table B.1, on a smaller sample, in exact rational arithmetic.
    Reading: the hyperbolic sample uses the exponents 0..53 (|coth 2phi| >= 1)."""
    g = json.load(open(os.path.join(GOLDEN, "table_b1.json")))
    dt1 = _departure_mean(1, 1, range(-53, 54), 192, 11)
    dt2 = _departure_mean(1, 2, range(-53, 54), 192, 12)
    dh1 = _departure_mean(-1, 1, range(0, 54), 192, 13)
    dh2 = _departure_mean(-1, 2, range(0, 54), 192, 14)
    assert dt1 == pytest.approx(g["d_t_cos1"], rel=0.08)
    assert dt2 == pytest.approx(g["d_t_cos2"], rel=0.05)
    assert dh1 == pytest.approx(g["d_h_cosh1"], rel=0.08)
    assert dh2 == pytest.approx(g["d_h_cosh2"], rel=0.05)
    assert dh2 < dh1                    # cosh_2 is the more J-orthogonal form
