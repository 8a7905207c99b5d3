"""Pins of the oracle's pivot strategies (Sec. 3 of the paper)."""
import json
import os

import pytest

from oracle import pivots as P
from tests.conftest import GOLDEN


def _one_based(s):
    return [[[i + 1, j + 1] for i, j in step] for step in s]


def test_order4_tables_golden():
    g = json.load(open(os.path.join(GOLDEN, "pstrategy_order4.json")))
    assert _one_based(P.closest_pstrategy("R", 4)) == g["R"]
    assert _one_based(P.closest_pstrategy("C", 4)) == g["C"]
    assert _one_based(P.strategy("rR", 4)) == g["rR"]
    assert _one_based(P.modulus(4)) == g["modulus_order4_reading"]


@pytest.mark.parametrize("n", [2, 4, 6, 8, 10, 12, 14, 16, 18, 20])
@pytest.mark.parametrize("kind", ["R", "C"])
def test_lemma_3_2_first_step(n, kind):
    s = P.closest_pstrategy(kind, n)
    assert s[0] == [(2 * k, 2 * k + 1) for k in range(n // 2)]
    assert P.is_pstrategy(s, n)


@pytest.mark.parametrize("n", [4, 8, 12, 16, 20, 24])
@pytest.mark.parametrize("kind", ["R", "C"])
def test_alg_3_1_equals_alg_3_2(n, kind):
    """Sec. 3: the expansion of O_{n/2} equals the closest p-strategy O_n
    (the paper verified it for orders up to 36)."""
    assert P.expand(P.closest_pstrategy(kind, n // 2), kind) == P.closest_pstrategy(kind, n)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_power_of_two_r_c_step_equivalent(k):
    """Sec. 3: for orders 2^k, R and C are step-equivalent (same p-steps as sets)."""
    n = 2 ** k
    r = P.closest_pstrategy("R", n)
    c = P.closest_pstrategy("C", n)
    assert [sorted(x) for x in r] == [sorted(x) for x in c]


@pytest.mark.parametrize("n", [2, 4, 6, 16, 30, 64, 96, 256, 512])
@pytest.mark.parametrize("name", ["modulus", "R", "C", "rR", "rC"])
def test_one_factorisation(n, name):
    if name != "modulus" and n == 30:
        pytest.skip("order 30 needs the DFS at order 30, outside the budget")
    s = P.strategy(name, n)
    assert P.is_pstrategy(s, n)


def test_reverse_is_literal():
    s = P.closest_pstrategy("R", 8)
    flat = [p for step in s for p in step]
    rflat = [p for step in P.reverse(s) for p in step]
    assert rflat == flat[::-1]
    assert P.reverse(s)[-1] == list(reversed(s[0]))   # ends with S^(1) reversed


def test_invariant_detects_broken_tables():
    s = P.modulus(8)
    bad = [list(x) for x in s]
    bad[1][0], bad[2][0] = bad[2][0], bad[1][0]        # duplicate / collision
    assert not P.is_pstrategy(bad, 8)
