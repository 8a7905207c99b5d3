"""Pivot strategies of the oracle -- TEST INFRASTRUCTURE ONLY.

Independent of the product's pivot generator: this file and the product share
no code or table.  Everything here is 0-based; a p-strategy of even order n is
a list of n-1 p-steps, each a list of n/2 pairs (i, j) with i < j.

Paper (Novakovic, hierarchically blocked Jacobi SVD), Sec. 3:
  row_cyclic / col_cyclic  the sequential strategies R_n and C_n
  closest_pstrategy        Alg. 3.1: the p-strategy closest to R_n or C_n in
                           the lexicographic order of Def. 3.1, found by
                           enumerating perfect matchings (maximal independent
                           sets of the collision graph with n/2 vertices) in
                           lexicographic order, with backtracking
  expand                   Alg. 3.2: O_n -> O~_2n
  reverse                  the reverse strategy (the sweep read backwards)
  modulus                  the modulus strategy (reading below)

Reading (modulus): the paper only cites the (modified) modulus strategy.  The
oracle takes Sameh's odd-order modulus ordering completed to even order:
with N = n - 1 (odd), p-step s in 0..N-1 is
  {(i, j) : 0 <= i < j < N, (i + j) mod N = s}  U  {(i*, N)},  2 i* = s mod N,
with pairs listed by ascending first index.
"""

from __future__ import annotations

import itertools

Pair = tuple[int, int]
Strategy = list[list[Pair]]


def row_cyclic(n: int) -> list[Pair]:
    """R_n: (0,1), (0,2), ..., (0,n-1), (1,2), ... (Sec. 3)."""
    return [(i, j) for i in range(n) for j in range(i + 1, n)]


def col_cyclic(n: int) -> list[Pair]:
    """C_n: (0,1), (0,2), (1,2), (0,3), (1,3), (2,3), ... (Sec. 3)."""
    return [(i, j) for j in range(n) for i in range(j)]


def _sequential(kind: str, n: int) -> list[Pair]:
    if kind == "R":
        return row_cyclic(n)
    if kind == "C":
        return col_cyclic(n)
    raise ValueError(kind)


def closest_pstrategy(kind: str, n: int, node_limit: int = 2_000_000) -> Strategy:
    """Alg. 3.1: the p-strategy closest (Def. 3.1) to R_n (kind 'R') or C_n ('C').

    The vertices of the collision graph are the positions 0..tau-1 of the pairs
    in the sequential strategy.  A p-step is a set of n/2 mutually disjoint
    remaining pairs; candidates are generated in lexicographic order of their
    ascending position lists, and the recursion backtracks when the remaining
    graph has no admissible p-step.  Within a p-step pairs are listed by
    ascending position, as Sec. 3 allows (step-equivalence)."""
    if n % 2 or n < 2:
        raise ValueError("order must be even and >= 2")
    seq = _sequential(kind, n)
    t = n // 2
    used = [False] * len(seq)
    result: list[list[int]] = []
    nodes = [0]

    def next_lex(remaining: list[int]):
        """Yield admissible p-steps (position lists) of the remaining graph,
        lexicographically (positions ascending inside each candidate)."""
        covered = [False] * n
        chosen: list[int] = []

        def rec(start: int):
            nodes[0] += 1
            if nodes[0] > node_limit:
                raise RuntimeError("search budget exhausted")
            if len(chosen) == t:
                yield list(chosen)
                return
            # prune: every uncovered index must still be coverable by a later
            # remaining pair whose other end is uncovered too
            for idx in range(start, len(remaining)):
                pos = remaining[idx]
                i, j = seq[pos]
                if covered[i] or covered[j]:
                    continue
                covered[i] = covered[j] = True
                chosen.append(pos)
                if _coverable(remaining, idx + 1, covered):
                    yield from rec(idx + 1)
                chosen.pop()
                covered[i] = covered[j] = False

        yield from rec(0)

    def _coverable(remaining, start, covered):
        need = [k for k in range(n) if not covered[k]]
        if not need:
            return True
        ok = [False] * n
        for idx in range(start, len(remaining)):
            i, j = seq[remaining[idx]]
            if not covered[i] and not covered[j]:
                ok[i] = ok[j] = True
        return all(ok[k] for k in need)

    def gen_strat() -> bool:
        remaining = [p for p in range(len(seq)) if not used[p]]
        if not remaining:
            return True
        for S in next_lex(remaining):
            result.append(S)
            for p in S:
                used[p] = True
            if gen_strat():
                return True
            for p in S:
                used[p] = False
            result.pop()
        return False

    if not gen_strat():
        raise RuntimeError("no p-strategy found")
    return [[seq[p] for p in step] for step in result]


def expand(strategy: Strategy, kind: str) -> Strategy:
    """Alg. 3.2, 0-based: a p-strategy of order n -> one of order 2n.

    1-based indices 2p-1 and 2p become 0-based 2p and 2p+1.  Output step 1
    is ((0,1), (2,3), ...); output step i >= 2 (1-based) expands input step
    floor(i/2): for even i each (p, q) gives NW = (2p, 2q) and SE = (2p+1, 2q+1);
    for odd i it gives NE = (2p, 2q+1) and SW = (2p+1, 2q), appended as
    (NE, SW) for R_n and (SW, NE) for C_n."""
    n = len(strategy) + 1                       # order of the input strategy
    out: Strategy = [[(2 * k, 2 * k + 1) for k in range(n)]]
    for i in range(2, 2 * n):
        src = strategy[i // 2 - 1]
        step: list[Pair] = []
        for p, q in src:
            if i % 2 == 0:
                step += [(2 * p, 2 * q), (2 * p + 1, 2 * q + 1)]
            else:
                ne, sw = (2 * p, 2 * q + 1), (2 * p + 1, 2 * q)
                step += [ne, sw] if kind == "R" else [sw, ne]
        out.append(step)
    return out


def reverse(strategy: Strategy) -> Strategy:
    """The reverse strategy: the sweep's pair sequence read backwards (Sec. 3),
    so both the p-step order and the pair order inside each p-step flip."""
    return [list(reversed(step)) for step in reversed(strategy)]


def modulus(n: int) -> Strategy:
    """Modulus p-strategy of even order n (reading in the module docstring)."""
    if n % 2 or n < 2:
        raise ValueError("order must be even and >= 2")
    N = n - 1
    out: Strategy = []
    for s in range(N):
        step = [(i, j) for i in range(N) for j in range(i + 1, N) if (i + j) % N == s]
        istar = next(i for i in range(N) if (2 * i) % N == s)
        step.append((istar, N))
        step.sort()
        out.append(step)
    return out


def by_expansion(kind: str, n: int) -> Strategy:
    """O~_n for n = 2^k * o (o odd): Alg. 3.1 at order 2o, then Alg. 3.2
    repeated k-1 times (the construction Sec. 3 proposes)."""
    if n % 2:
        raise ValueError("order must be even")
    o, k = n, 0
    while o % 2 == 0:
        o //= 2
        k += 1
    s = closest_pstrategy(kind, 2 * o)
    for _ in range(k - 1):
        s = expand(s, kind)
    return s


def strategy(name: str, n: int) -> Strategy:
    """Named strategies: 'modulus', 'R', 'C', 'rR' (reverse of R), 'rC'."""
    if name == "modulus":
        return modulus(n)
    if name in ("R", "C"):
        return by_expansion(name, n)
    if name in ("rR", "rC"):
        return reverse(by_expansion(name[1], n))
    raise ValueError(name)


def is_pstrategy(s: Strategy, n: int) -> bool:
    """1-factorisation invariant (Eq. (3.1)): n-1 p-steps of n/2 disjoint
    pairs, every pair of P_n exactly once per sweep."""
    if len(s) != n - 1:
        return False
    seen = set()
    for step in s:
        if len(step) != n // 2:
            return False
        idx = list(itertools.chain.from_iterable(step))
        if sorted(idx) != list(range(n)):
            return False
        for i, j in step:
            if not (0 <= i < j < n) or (i, j) in seen:
                return False
            seen.add((i, j))
    return len(seen) == n * (n - 1) // 2


def to_array(s: Strategy):
    """Flatten to a (steps, pairs, 2) int32 numpy array."""
    import numpy as np

    return np.asarray(s, dtype=np.int32).reshape(len(s), len(s[0]) if s else 0, 2)


# ---------------------------------------------------------------------------
# Dynamic block ordering (a reading of the "column-norm-sorted" orderings;
# the paper's strategies are static, Sec. 3): before a sweep the block-columns
# are ranked by descending norm, ties by index, and the static table is
# applied to that ranking; each pair is kept as (lower, higher) block index.
def norm_order(block_norms) -> list[int]:
    """perm[i] = the block of rank i (descending norm, stable)."""
    idx = list(range(len(block_norms)))
    return sorted(idx, key=lambda B: (-float(block_norms[B]), B))


def remap(table, perm):
    """The table with every pair (p, q) replaced by (min, max)(perm[p], perm[q])."""
    return [[(min(perm[p], perm[q]), max(perm[p], perm[q])) for (p, q) in step] for step in table]
