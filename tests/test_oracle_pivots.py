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


# ---------------------------------------------------------------------------
# dynamic block ordering: a remapped parallel strategy is still a parallel
# strategy (Def. 3.1: every p-step a set of disjoint pairs, every pair once
# per sweep), and the ranking is a stable descending sort
@pytest.mark.parametrize("name", ["modulus", "rR", "C"])
@pytest.mark.parametrize("nb", [4, 10, 16, 48])
def test_remapped_table_is_a_parallel_strategy(name, nb):
    import random

    rnd = random.Random(nb)
    perm = list(range(nb))
    rnd.shuffle(perm)
    tab = P.remap(P.strategy(name, nb), perm)
    seen = set()
    for step in tab:
        cols = [c for pq in step for c in pq]
        assert sorted(cols) == list(range(nb))
        for p, q in step:
            assert p < q and (p, q) not in seen
            seen.add((p, q))
    assert len(seen) == nb * (nb - 1) // 2
    # the identity ranking gives the static table back
    assert P.remap(P.strategy(name, nb), list(range(nb))) == P.strategy(name, nb)


def test_norm_order_is_a_stable_descending_sort():
    norms = [3.0, 1.0, 3.0, 7.0, 1.0, 0.0]
    assert P.norm_order(norms) == [3, 0, 2, 1, 4, 5]


@pytest.mark.parametrize("b", [4, 8])
def test_block_method_with_dynamic_order(b):
    """The dynamic ordering changes only which block pairs meet when: the
    method converges to the same singular values (LAPACK, normwise) and
    G = A V keeps holding; the first ranking is that of the input's blocks."""
    import numpy as np

    import oracle as O
    from paper_1401_2720_gb300 import inputs as I

    A = I.graded_columns(120, 8 * b, 3.0, seed=b)[:, ::-1].copy(order="F")   # ascending column norms
    r = O.block_svd_dynamic(A, b, strategy="rR")
    assert r["converged"]
    assert r["perms"][0] == P.norm_order(O.block_norms(A, b))
    assert r["perms"][0][0] == 8 - 1        # the largest block comes first
    s = np.sort(O.colnorms(r["G"]))[::-1]
    sl = np.linalg.svd(A, compute_uv=False)
    assert np.max(np.abs(s - sl)) <= 100 * np.sqrt(8 * b) * 2.0 ** -53 * sl[0]
    assert np.linalg.norm(A @ r["V"] - r["G"]) <= 1e-13 * np.linalg.norm(A)
