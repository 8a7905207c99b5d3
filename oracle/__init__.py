"""Oracle for the block-oriented one-sided Jacobi (H)SVD -- TEST INFRASTRUCTURE.

A plain, slow, obviously correct CPU implementation of what the CUDA path
computes, written from the paper (Novakovic, "A hierarchically blocked Jacobi
SVD algorithm for single and multiple graphics processing units") and
independent of the CUDA path: the two share no code, header, table or
generator.  Only tests/, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline / reference legs may import this package.  The product path
never does.

Numerics are plain C (``jacobi_oracle.c``, compiled with
``-ffp-contract=off``), written once over a scalar type and built twice: FP64
(the parity reference and the timed CPU baseline) and IEEE binary128
(``q_svd``, ``q_loss_fd``: ground truth for small sizes and finite
differences of the SVD).  The pairs of one p-step are disjoint, so the C code
may run them on several threads (``set_threads``); results are bitwise
identical for any thread count.  Pivot strategies are plain Python
(``pivots.py``).

Pins (tests/test_oracle_*.py): closed-form 2x2 rotations, Table B.1 of the
paper (statistical, exact rational arithmetic), Lemma 3.2 and the n = 4
tables, Alg. 3.1 == Alg. 3.2 for small orders, the 1-factorisation
invariant, planted singular values, LAPACK (numpy) and mpmath SVDs, the
reconstruction / orthogonality invariants, eigenvalues of G J G^T for the
HSVD, and central finite differences for the adjoint.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

if os.environ.get("JO_PIVOTS_SRC"):
    # the mutation tests' hook for a planted-mistake copy of pivots.py
    import importlib.util
    import sys

    _spec = importlib.util.spec_from_file_location(__name__ + ".pivots", os.environ["JO_PIVOTS_SRC"])
    pivots = importlib.util.module_from_spec(_spec)
    sys.modules[__name__ + ".pivots"] = pivots
    _spec.loader.exec_module(pivots)
else:
    from . import pivots

_HERE = os.path.dirname(os.path.abspath(__file__))
# JO_ORACLE_SRC / JO_ORACLE_BUILD: a hook for the mutation tests, which build a
# copy of the C file with one planted mistake into a directory of their own
# and check that the pins catch it; unset, the oracle is this directory's C.
_SRC = os.environ.get("JO_ORACLE_SRC") or os.path.join(_HERE, "jacobi_oracle.c")
_BUILD = os.environ.get("JO_ORACLE_BUILD") or os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libjacobi_oracle.so")
_SO_Q = os.path.join(_BUILD, "libjacobi_oracle_q.so")
_lock = threading.Lock()
_lib = None
_lib_q = None

EPS = 2.0 ** -53


def build(force: bool = False) -> str:
    """Compile the oracle's C file with gcc (plain C, no fused multiply-add
    contraction) into oracle/_build/: the FP64 library and the binary128 one."""
    os.makedirs(_BUILD, exist_ok=True)
    for so, extra in ((_SO, []), (_SO_Q, ["-DJO_QUAD"])):
        if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
            tmp = so + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", *extra,
                                   "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
            os.replace(tmp, so)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            lib.jo_rot.argtypes = [D, D, D, I, I, P, P]
            lib.jo_rot.restype = I
            lib.jo_rot_batch.argtypes = [I, P, P, P, P, I, P, P, P]
            lib.jo_hestenes.argtypes = [I, I, I, P, I, P, I, P, I, I, I, D, P, P]
            lib.jo_block_pstep.argtypes = [I, I, I, I, P, I, P, I, P, I, P, I, I, I, P]
            lib.jo_block_svd.argtypes = [I, I, I, I, P, I, P, I, P, I, I, P, I, I, I, I, P, P]
            lib.jo_colnorms.argtypes = [I, I, P, I, P]
            lib.jo_svd_adjoint.argtypes = [I, I, P, P, P, P, P, P, P]
            lib.jo_set_threads.argtypes = [I]
            lib.jo_qrcp.argtypes = [I, I, P, I, P, P]
            lib.jo_drdssq.argtypes = [I, P, I, P, P]
            lib.jo_apply_q.argtypes = [I, I, P, I, P, I, P, I]
            _lib = lib
    return _lib


def _load_q():
    global _lib_q
    _load()
    with _lock:
        if _lib_q is None:
            lib = ctypes.CDLL(_SO_Q)
            P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            lib.jo_q_set_threads.argtypes = [I]
            lib.jo_q_svd.argtypes = [I, I, P, I, P, I, I, I, P, P, P, P]
            lib.jo_q_loss_fd.argtypes = [I, I, P, P, D, P, P, P, I, I, I, P]
            lib.jo_q_loss_fd.restype = D
            lib.jo_q_sumsq.argtypes = [I, P, P, P]
            _lib_q = lib
    return _lib_q


def set_threads(threads: int) -> None:
    """Worker threads over the disjoint pairs of a p-step (both builds)."""
    _load().jo_set_threads(int(threads))
    _load_q().jo_q_set_threads(int(threads))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _fortran(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


# ---------------------------------------------------------------------------
def rotation(hpp, hqq, hpq, hyperbolic=False, cs_form=2):
    """Eqs. (4.3)-(4.6): (cs, tn, proper) for arrays of 2x2 pivot data."""
    hpp = np.ascontiguousarray(np.atleast_1d(hpp), dtype=np.float64)
    hqq = np.ascontiguousarray(np.broadcast_to(hqq, hpp.shape), dtype=np.float64)
    hpq = np.ascontiguousarray(np.broadcast_to(hpq, hpp.shape), dtype=np.float64)
    t = np.ascontiguousarray(np.broadcast_to(np.where(hyperbolic, -1, 1), hpp.shape), dtype=np.int32)
    n = hpp.size
    cs = np.empty(n)
    tn = np.empty(n)
    pr = np.empty(n, dtype=np.int32)
    _load().jo_rot_batch(n, _ptr(hpp), _ptr(hqq), _ptr(hpq), _ptr(t), cs_form, _ptr(cs), _ptr(tn), _ptr(pr))
    return cs, tn, pr.astype(bool)


def strategy_array(name: str, n: int) -> np.ndarray:
    return pivots.to_array(pivots.strategy(name, n))


def hestenes(A, strategy: str = "rR", nplus: int | None = None, max_sweeps: int = 100,
             with_v: bool = True, nhat: float | None = None):
    """Pointwise one-sided Jacobi on A (m x n, m >= n, n even); returns the raw
    results: G = A V (unsorted), V (or W = V^{-T} for the HSVD), statistics."""
    G = _fortran(A).copy(order="F")
    m, n = G.shape
    nplus = n if nplus is None else nplus
    V = np.asfortranarray(np.eye(n)) if with_v else None
    if n % 2:
        # odd n (Eq. (3.1): n p-steps of (n-1)/2 pairs): the strategy of order
        # n+1 with every pair that holds the phantom index n left out
        full = pivots.strategy(strategy, n + 1)
        tab = np.ascontiguousarray(pivots.to_array([[p for p in st if p[1] < n] for st in full]))
    else:
        tab = np.ascontiguousarray(strategy_array(strategy, n))
    stats = np.zeros(5, dtype=np.int64)
    per = np.zeros(max_sweeps, dtype=np.int64)
    _load().jo_hestenes(m, n, nplus, _ptr(G), m, _ptr(V) if V is not None else None, n,
                        _ptr(tab), tab.shape[0], tab.shape[1], max_sweeps,
                        float(m if nhat is None else nhat), _ptr(stats), _ptr(per))
    return dict(G=G, V=V, sweeps=int(stats[0]), converged=bool(stats[1]),
                rotations=int(stats[2]), proper=int(stats[3]), swaps=int(stats[4]),
                rotations_per_sweep=per[: stats[0]].copy())


def _pointwise_table(strategy: str, n: int) -> np.ndarray:
    """The p-strategy table of order n for the pointwise method; odd n uses
    the order-(n+1) table without the pairs that hold the phantom index n."""
    if n % 2:
        full = pivots.strategy(strategy, n + 1)
        return np.ascontiguousarray(pivots.to_array([[p for p in st if p[1] < n] for st in full]))
    return np.ascontiguousarray(strategy_array(strategy, n))


def q_svd(A, strategy: str = "rR", max_sweeps: int = 100, with_vectors: bool = True):
    """The pointwise one-sided Jacobi SVD in binary128 (eps = 2^-113), sorted;
    returns (U, S, V, converged) rounded to double (U, V None unless asked)."""
    A = _fortran(A)
    m, n = A.shape
    tab = _pointwise_table(strategy, n)
    S = np.empty(n)
    U = np.asfortranarray(np.empty((m, n))) if with_vectors else None
    V = np.asfortranarray(np.empty((n, n))) if with_vectors else None
    st = np.zeros(2, dtype=np.int64)
    _load_q().jo_q_svd(m, n, _ptr(A), m, _ptr(tab), tab.shape[0], tab.shape[1], max_sweeps, _ptr(S),
                       _ptr(U) if U is not None else None, _ptr(V) if V is not None else None, _ptr(st))
    return U, S, V, bool(st[1])


def q_loss_fd(A, E, h: float, w, C, strategy: str = "rR", max_sweeps: int = 100) -> float:
    """Central difference (L(A + hE) - L(A - hE)) / 2h in binary128 of
    L = sum_i w_i s_i + <C, U V^T> (the loss of the batched adjoint check)."""
    A, E, C = _fortran(A), _fortran(E), _fortran(C)
    m, n = A.shape
    w = np.ascontiguousarray(w, dtype=np.float64)
    tab = _pointwise_table(strategy, n)
    ok = ctypes.c_int(0)
    v = _load_q().jo_q_loss_fd(m, n, _ptr(A), _ptr(E), float(h), _ptr(w), _ptr(C), _ptr(tab), tab.shape[0],
                               tab.shape[1], max_sweeps, ctypes.byref(ok))
    if not ok.value:
        raise RuntimeError("binary128 SVD hit the sweep limit")
    return v


def colnorms(G) -> np.ndarray:
    G = _fortran(G)
    m, n = G.shape
    s = np.empty(n)
    _load().jo_colnorms(m, n, _ptr(G), m, _ptr(s))
    return s


def finish(G, V, nplus: int | None = None, hyperbolic_w: bool = False):
    """Sigma extraction and the final order: sigma_i = ||g_i||, u_i = g_i/sigma_i,
    stable sort descending (within the J+ and J- blocks for the HSVD);
    for the HSVD the accumulated W is turned into V = J W J."""
    G = _fortran(G)
    m, n = G.shape
    nplus = n if nplus is None else nplus
    s = colnorms(G)
    if nplus == n:
        order = np.argsort(-s, kind="stable")
    else:
        order = np.concatenate([np.argsort(-s[:nplus], kind="stable"),
                                nplus + np.argsort(-s[nplus:], kind="stable")])
    with np.errstate(divide="ignore", invalid="ignore"):
        U = np.where(s[order] > 0, G[:, order] / s[order], 0.0)
    Vout = None
    if V is not None:
        W = np.asarray(V)
        if hyperbolic_w:
            j = np.where(np.arange(n) < nplus, 1.0, -1.0)
            W = j[:, None] * W * j[None, :]
        Vout = W[:, order]
    return U, s[order], Vout


def svd(A, strategy: str = "rR", max_sweeps: int = 100):
    """Full oracle SVD A = U diag(S) V^T (pointwise Hestenes + finish)."""
    r = hestenes(A, strategy=strategy, max_sweeps=max_sweeps)
    U, S, V = finish(r["G"], r["V"])
    return U, S, V, r


def hsvd(G, nplus: int, strategy: str = "rR", max_sweeps: int = 100):
    """Oracle HSVD G = U diag(S) V^T with V^T J V = J, J = diag(I_nplus, -I)."""
    r = hestenes(G, strategy=strategy, nplus=nplus, max_sweeps=max_sweeps)
    U, S, V = finish(r["G"], r["V"], nplus=nplus, hyperbolic_w=True)
    return U, S, V, r


def block_pstep(G, V, b: int, step_pairs, inner_table, nplus: int | None = None,
                inner_sweeps: int = 1, border: tuple[int, int] = (0, 0), inplace: bool = False):
    """One p-step of the block-oriented method on copies of G and V (or, with
    inplace, on G and V themselves when they are Fortran-ordered float64)."""
    if not (inplace and G.flags.f_contiguous and V.flags.f_contiguous and G.dtype == np.float64
            and V.dtype == np.float64):
        G = _fortran(G).copy(order="F")
        V = _fortran(V).copy(order="F")
    m, n = G.shape
    nplus = n if nplus is None else nplus
    sp = np.ascontiguousarray(np.asarray(step_pairs, dtype=np.int32).reshape(-1, 2))
    it = np.ascontiguousarray(np.asarray(inner_table, dtype=np.int32))
    stats = np.zeros(4, dtype=np.int64)
    _load().jo_block_pstep(m, n, nplus, b, _ptr(G), m, _ptr(V), n, _ptr(sp), sp.shape[0],
                           _ptr(it), inner_sweeps, border[0], border[1], _ptr(stats))
    return G, V, dict(rotations=int(stats[0]), proper=int(stats[1]),
                      updated=int(stats[2]), breakdowns=int(stats[3]))


def bordered(A, b: int, nplus: int | None = None):
    """Identity bordering [[G, 0], [0, I_k]] up to the next multiple of 2b
    columns (for the HSVD the border columns are inserted at the J boundary):
    returns (the bordered matrix, (first, last+1) border column, n_plus of it)."""
    A = _fortran(A)
    m, n = A.shape
    nplus = n if nplus is None else nplus
    n_pad = max(2 * b, -(-n // (2 * b)) * 2 * b)
    k = n_pad - n
    B = np.zeros((m + k, n_pad))
    B[:m, :nplus] = A[:, :nplus]
    B[:m, nplus + k:] = A[:, nplus:]
    B[m:, nplus:nplus + k] = np.eye(k)
    return np.asfortranarray(B), (nplus, nplus + k), nplus + k


def block_svd(A, b: int, strategy: str = "rR", inner_strategy: str | None = None,
              nplus: int | None = None, inner_sweeps: int = 1, max_sweeps: int = 30,
              border: tuple[int, int] = (0, 0)):
    """The block-oriented method (Sec. 2, 4) on CPU: raw G, V and statistics."""
    G = _fortran(A).copy(order="F")
    m, n = G.shape
    if n % (2 * b):
        raise ValueError("n must be a multiple of 2b (see bordered())")
    nb = n // b
    nplus = n if nplus is None else nplus
    V = np.asfortranarray(np.eye(n))
    tab = np.ascontiguousarray(strategy_array(strategy, nb))
    it = np.ascontiguousarray(strategy_array(inner_strategy or strategy, 2 * b))
    stats = np.zeros(6, dtype=np.int64)
    per = np.zeros(max_sweeps, dtype=np.int64)
    _load().jo_block_svd(m, n, nplus, b, _ptr(G), m, _ptr(V), n, _ptr(tab), tab.shape[0],
                         tab.shape[1], _ptr(it), inner_sweeps, max_sweeps, border[0], border[1],
                         _ptr(stats), _ptr(per))
    return dict(G=G, V=V, sweeps=int(stats[0]), converged=bool(stats[1]), rotations=int(stats[2]),
                proper=int(stats[3]), updated=int(stats[4]), breakdowns=int(stats[5]),
                proper_per_sweep=per[: stats[0]].copy())


def drdssq(x) -> tuple[int, float]:
    """App. A: ||x||^2 = f 2^e, e even, 0.5 <= f < 2, without overflow or
    underflow; returns (e, f)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    e = ctypes.c_int(0)
    f = ctypes.c_double(0.0)
    _load().jo_drdssq(x.size, _ptr(x), 1, ctypes.byref(e), ctypes.byref(f))
    return e.value, f.value


def q_sumsq(x) -> tuple[int, float]:
    """||x||^2 in binary128 as f 2^e, 0.5 <= f < 1 (f rounded to double)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    e = ctypes.c_int(0)
    f = ctypes.c_double(0.0)
    _load_q().jo_q_sumsq(x.size, _ptr(x), ctypes.byref(e), ctypes.byref(f))
    return e.value, f.value


def qrcp(A):
    """A P = Q [R; 0] by Householder with column pivoting (Sec. 2, Eq. (2.1)):
    returns (the factored array: R above, reflectors below the diagonal), tau,
    piv (piv[j] = original column at position j)."""
    W = _fortran(A).copy(order="F")
    m, n = W.shape
    tau = np.empty(n)
    piv = np.empty(n, dtype=np.int32)
    _load().jo_qrcp(m, n, _ptr(W), m, _ptr(tau), _ptr(piv))
    return W, tau, piv


def apply_q(W, tau, X):
    """Q X for the Q of qrcp()."""
    W = _fortran(W)
    X = _fortran(X).copy(order="F")
    m, n = W.shape
    _load().jo_apply_q(m, n, _ptr(W), m, _ptr(np.ascontiguousarray(tau)), X.shape[1], _ptr(X), m)
    return X


def svd_qr(A, strategy: str = "modulus", max_sweeps: int = 100):
    """The SVD with the QR preprocessing: A P = Q [R; 0], the pointwise method
    on R^T = X S Y^T, then U = Q [Y; 0], V = P X.  Returns (U, S, V, raw)."""
    W, tau, piv = qrcp(A)
    m, n = W.shape
    RT = np.asfortranarray(np.triu(W[:n, :]).T)
    X, S, Y, r = svd(RT, strategy=strategy, max_sweeps=max_sweeps)
    U = apply_q(W, tau, np.vstack([Y, np.zeros((m - n, n))]))
    V = np.empty_like(X)
    V[piv, :] = X
    return U, S, V, r


def block_norms(G, b: int) -> np.ndarray:
    """Squared Frobenius norm of every block-column of width b (plain sums of
    squares, column by column, in the oracle's column-norm routine)."""
    s = colnorms(G)
    return (s * s).reshape(-1, b).sum(axis=1)


def block_svd_dynamic(A, b: int, strategy: str = "rR", nplus: int | None = None, max_sweeps: int = 30):
    """The block-oriented method with the dynamic block ordering: before each
    sweep the block-columns are ranked by descending norm and the static table
    of `strategy` is applied to that ranking (pivots.norm_order, pivots.remap).
    Returns raw G, V and statistics like block_svd."""
    G = _fortran(A).copy(order="F")
    m, n = G.shape
    if n % (2 * b):
        raise ValueError("n must be a multiple of 2b (see bordered())")
    nb = n // b
    V = np.asfortranarray(np.eye(n))
    static = pivots.strategy(strategy, nb)
    inner = strategy_array(strategy, 2 * b)
    tot = dict(rotations=0, proper=0, updated=0, breakdowns=0)
    per, perms = [], []
    converged = False
    for _ in range(max_sweeps):
        perm = pivots.norm_order(block_norms(G, b))
        perms.append(perm)
        tab = pivots.to_array(pivots.remap(static, perm))
        before = tot["proper"]
        for step in tab:
            G, V, st = block_pstep(G, V, b, step, inner, nplus=nplus, inplace=True)
            for k in tot:
                tot[k] += st[k]
        per.append(tot["proper"] - before)
        if per[-1] == 0:
            converged = True
            break
    return dict(G=G, V=V, sweeps=len(per), converged=converged, proper_per_sweep=np.array(per), perms=perms, **tot)


def svd_adjoint(U, S, V, dU, dS, dV) -> np.ndarray:
    """Reverse-mode derivative dA of A = U diag(S) V^T (published formula)."""
    U, V, dU, dV = (_fortran(x) for x in (U, V, dU, dV))
    S = np.ascontiguousarray(S, dtype=np.float64)
    dS = np.ascontiguousarray(dS, dtype=np.float64)
    m, n = U.shape
    dA = np.asfortranarray(np.empty((m, n)))
    _load().jo_svd_adjoint(m, n, _ptr(U), _ptr(S), _ptr(V), _ptr(dU), _ptr(dS), _ptr(dV), _ptr(dA))
    return dA
