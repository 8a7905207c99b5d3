"""The oracle's pins are sensitive: each case plants one plausible mistake in a
copy of the oracle's C file -- a wrong sign, a dropped factor or term, a
transposed operand, a wrong index, a skipped step -- builds that copy into a
directory of its own (JO_ORACLE_SRC / JO_ORACLE_BUILD) and runs the oracle's
pin tests against it in a subprocess.  Every planted mistake must make at
least one pin fail, and the unmodified copy must pass them all.  CPU only; the
planted mistakes live only in temporary copies.

Cases, by the passage each one breaks:
  Eqs. (4.3)-(4.6)  the rotation: signs of h, ct2 and tan, the factor 2, the
                    cs_2 form of the hyperbolic cosh, the small-angle shortcut;
  Eqs. (4.1)/(4.2)  its application: the FMA signs, the multiply by cs;
  Sec. 4.3          the relative test (|h_pq|), the P2 sort's direction in
                    either J block, V's rotation and swap, the hyperbolic
                    type at the J boundary;
  Eq. (2.7), 4.1    the Gram entry's operands, the Cholesky update and pivot;
  Eq. (2.9)         the update's right factor transposed;
  Sec. 4 (Sigma)    the column norm's square root;
  App. A            DRDSSQ's large-entry scale and its even exponent;
  Sec. 4.5          the stop rules of the pointwise and the block method;
  readings R5, R7   a zero Cholesky pivot not counted, border columns rotated;
  Eq. (2.1)         the QR preprocessing's pivot choice, reflector and tau, and
                    the order in which Q is applied;
  the SVD adjoint   the sign of F, the V term, the projector term.
The same is done for the oracle's pivot generator (pivots.py, JO_PIVOTS_SRC),
against its pins and the bit-exact comparison with the library's tables:
  Sec. 3            R_n enumerated as C_n, the order of Alg. 3.2's NE/SW and
                    NW/SE pairs, the reverse without the in-step reversal, the
                    modulus strategy's idle index, the dynamic ordering's tie
                    break and its (lower, higher) pairs.
And for the oracle's Python layer (oracle/__init__.py, run on a copy of the
tree): the final sort's direction in either J block, u_i = g_i / sigma_i, the
HSVD's V = J W J, the identity border's rows and the columns after it, the QR
preprocessing's R^T and its permutation of V, and the dynamic ordering's
per-sweep ranking.
Not a case: the sign of tan*h_pq in the P2 sort's new diagonal (reading R1).
The annihilating rotation (|phi| <= pi/4) never reverses the order of h_pp and
h_qq, and both new diagonal entries move by the same tan*h_pq, so comparing the
old entries, or entries shifted either way, takes the same decision up to
rounding ties: no outcome can tell the two signs apart (the 2x2 closed-form
pin checks that formula of the new diagonal against the rotated matrix).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

from tests.conftest import ROOT

SRC = os.path.join(ROOT, "oracle", "jacobi_oracle.c")
PINS = ["tests/test_oracle_rotation.py", "tests/test_oracle_svd.py", "tests/test_oracle_adjoint.py",
        "tests/test_oracle_drdssq.py", "tests/test_oracle_quad.py"]

# name: (exact text in the oracle's C file, the planted mistake)
MUTATIONS = {
    "h sign (4.3)": ("real h = hqq - tt * hpp;", "real h = hqq + tt * hpp;"),
    "ct2 sign (4.3)": ("real ct2 = tt * (h / (2.0 * hpq));", "real ct2 = -tt * (h / (2.0 * hpq));"),
    "factor 2 dropped (4.3)": ("real ct2 = tt * (h / (2.0 * hpq));", "real ct2 = tt * (h / hpq);"),
    "small-angle shortcut bound (4.4)": ("else if (t > 0 && act2 < R_SQRT(JO_EPS))",
                                         "else if (t > 0 && act2 < 1.0)"),
    "tan sign (4.5)": ("real tnv = R_COPYSIGN(1.0 / act, ct2);", "real tnv = R_COPYSIGN(1.0 / act, -ct2);"),
    "cs_2 with t = +1 for cosh (4.6)": ("csv = act / R_SQRT(R_FMA(act, act, tt));",
                                       "csv = act / R_SQRT(R_FMA(act, act, 1.0));"),
    "trigonometric FMA sign (4.1)": ("xn = R_FMA(-tn, yi, xi);", "xn = R_FMA(tn, yi, xi);"),
    "hyperbolic FMA sign (4.2)": ("xn = R_FMA(tn, yi, xi);", "xn = R_FMA(-tn, yi, xi);"),
    "cs multiply dropped on one column": ("if (cs != 1.0) { xn = cs * xn; yn = cs * yn; }",
                                          "if (cs != 1.0) { xn = cs * xn; }"),
    "relative test without |h_pq|": ("R_FABS(hpq) < c_eps", "hpq < c_eps"),
    "P2 sort direction, J+ block": ("if (l < nplus && npp < nqq) swap = 1;", "if (l < nplus && npp > nqq) swap = 1;"),
    "P2 sort direction, J- block": ("if (k >= nplus && npp > nqq) swap = 1;", "if (k >= nplus && npp < nqq) swap = 1;"),
    "V not rotated": ("if (nv) apply_rot(nv, vp, vq, t, cs, tn);", "if (0) apply_rot(nv, vp, vq, t, cs, tn);"),
    "V not swapped": ("if (nv) swap_cols(nv, vp, vq);", "if (0) swap_cols(nv, vp, vq);"),
    "Gram operand index (2.7)": ("H[i + j * bb] = dot(m, X + (size_t)i * m, X + (size_t)j * m);",
                                 "H[i + j * bb] = dot(m, X + (size_t)i * m, X + (size_t)i * m);"),
    "Cholesky update sign (4.1)": ("d = R_FMA(-L[k + j * bb], L[k + j * bb], d);",
                                   "d = R_FMA(L[k + j * bb], L[k + j * bb], d);"),
    "Cholesky division dropped (4.1)": ("L[i + k * bb] = s / lkk;", "L[i + k * bb] = s;"),
    "update with V' transposed (2.9)": ("s = R_FMA(X[i + (size_t)k * rows], W[k + j * bb], s);",
                                        "s = R_FMA(X[i + (size_t)k * rows], W[j + k * bb], s);"),
    "column norm without the root": ("sigma[j] = R_SQRT(dot(m, G + (size_t)j * ldg, G + (size_t)j * ldg));",
                                     "sigma[j] = dot(m, G + (size_t)j * ldg, G + (size_t)j * ldg);"),
    "DRDSSQ large-entry scale sign": ("if (b > nu_h) { double y = ldexp(a, l2);",
                                      "if (b > nu_h) { double y = ldexp(a, -l2);"),
    "DRDSSQ odd exponent": ("int mp = -(((m % 2) + 2) % 2);", "int mp = 0;"),
    "QR reflector sign (2.1)": ("c[r] = R_FMA(-f, x[r], c[r]);", "c[r] = R_FMA(f, x[r], c[r]);"),
    "adjoint F sign": ("real F = 1.0 / (s[j] * s[j] - s[i] * s[i]);", "real F = 1.0 / (s[i] * s[i] - s[j] * s[j]);"),
    "adjoint V term dropped": ("v = F * a * s[j] + s[i] * (F * c);", "v = F * a * s[j];"),
    "adjoint projector term dropped": ("Z[r + (size_t)j * m] = (dU[r + (size_t)j * m] - a) / s[j];",
                                       "Z[r + (size_t)j * m] = dU[r + (size_t)j * m] / s[j];"),
    "pointwise stop after any sweep (4.5)": ("if (rot == 0) { converged = 1; ++sweep; break; }",
                                             "if (rot >= 0) { converged = 1; ++sweep; break; }"),
    "block stop after any sweep (4.5)": ("if (B == 0) { converged = 1; ++sweep; break; }",
                                         "if (B >= 0) { converged = 1; ++sweep; break; }"),
    "border columns rotated (R7)": ("        return 0;                                       /* R7 */",
                                    "        ;                                               /* R7 */"),
    "hyperbolic type boundary (Sec. 4.3)": ("int t = (k < nplus && l >= nplus) ? -1 : 1;",
                                            "int t = (k < nplus && l > nplus) ? -1 : 1;"),
    "zero Cholesky pivot not a breakdown (R5)": ("if (!(d > 0.0)) {", "if (d < 0.0) {"),
    "QR pivot: smallest column (2.1)": ("if (nrm[k] > nrm[best]) best = k;", "if (nrm[k] < nrm[best]) best = k;"),
    "QR tau sign (2.1)": ("tau[j] = (beta - alpha) / beta;", "tau[j] = (alpha - beta) / beta;"),
    "Q applied in the wrong order (2.1)": ("for (int j = n - 1; j >= 0; --j) {", "for (int j = 0; j < n; ++j) {"),
}


PIVOTS_SRC = os.path.join(ROOT, "oracle", "pivots.py")
PIVOT_PINS = ["tests/test_oracle_pivots.py", "tests/test_abi.py"]
PIVOT_MUTATIONS = {
    "R_n enumerated column-wise": ("return [(i, j) for i in range(n) for j in range(i + 1, n)]",
                                   "return [(i, j) for j in range(n) for i in range(j)]"),
    "Alg. 3.2 NE/SW order swapped": ('step += [ne, sw] if kind == "R" else [sw, ne]',
                                     'step += [sw, ne] if kind == "R" else [ne, sw]'),
    "Alg. 3.2 NW/SE order swapped": ("step += [(2 * p, 2 * q), (2 * p + 1, 2 * q + 1)]",
                                     "step += [(2 * p + 1, 2 * q + 1), (2 * p, 2 * q)]"),
    "reverse keeps the in-step order": ("return [list(reversed(step)) for step in reversed(strategy)]",
                                        "return [list(step) for step in reversed(strategy)]"),
    "modulus idle index": ("istar = next(i for i in range(N) if (2 * i) % N == s)",
                           "istar = next(i for i in range(N) if (2 * i + 1) % N == s)"),
    "norm order ties reversed": ("return sorted(idx, key=lambda B: (-float(block_norms[B]), B))",
                                 "return sorted(idx, key=lambda B: (-float(block_norms[B]), -B))"),
    "remap without (lower, higher)": ("[(min(perm[p], perm[q]), max(perm[p], perm[q])) for (p, q) in step]",
                                      "[(perm[p], perm[q]) for (p, q) in step]"),
}


def _run_pins(file_name: str, env_vars, pins, text: str):
    d = tempfile.mkdtemp(prefix="jo_mutant_")
    try:
        src = os.path.join(d, file_name)
        with open(src, "w") as f:
            f.write(text)
        env = dict(os.environ, **{k: v.format(src=src, dir=d) for k, v in env_vars.items()})
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *pins],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
        return r.returncode, r.stdout[-2500:] + r.stderr[-1000:]
    finally:
        shutil.rmtree(d, ignore_errors=True)


def _check(path, mutations, file_name, env_vars, pins):
    base = open(path).read()
    cases = {"unmodified copy": base}
    for name, (old, new) in mutations.items():
        assert base.count(old) == 1, f"{name}: the text to mutate must occur exactly once"
        cases[name] = base.replace(old, new)
    run = lambda text: _run_pins(file_name, env_vars, pins, text)     # noqa: E731
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = dict(zip(cases, ex.map(run, cases.values())))
    rc, out = results.pop("unmodified copy")
    assert rc == 0, out
    survivors = [name for name, (code, _) in results.items() if code == 0]
    assert not survivors, f"planted mistakes no pin catches: {survivors}"


def test_pins_catch_every_planted_mistake():
    _check(SRC, MUTATIONS, "jacobi_oracle.c", {"JO_ORACLE_SRC": "{src}", "JO_ORACLE_BUILD": "{dir}/_build"}, PINS)


def test_pivot_pins_catch_every_planted_mistake():
    from paper_1401_2720_gb300 import build_ext

    build_ext.build()       # once here, so the parallel runs of tests/test_abi.py find it built
    _check(PIVOTS_SRC, PIVOT_MUTATIONS, "pivots.py", {"JO_PIVOTS_SRC": "{src}"}, PIVOT_PINS)


PY_PINS = ["tests/test_oracle_rotation.py", "tests/test_oracle_svd.py", "tests/test_oracle_adjoint.py",
           "tests/test_oracle_quad.py", "tests/test_oracle_pivots.py"]
PY_MUTATIONS = {
    "final sort ascending": ('order = np.argsort(-s, kind="stable")', 'order = np.argsort(s, kind="stable")'),
    "J- block sorted ascending": ('nplus + np.argsort(-s[nplus:], kind="stable")',
                                  'nplus + np.argsort(s[nplus:], kind="stable")'),
    "U not normalised": ("U = np.where(s[order] > 0, G[:, order] / s[order], 0.0)",
                         "U = np.where(s[order] > 0, G[:, order], 0.0)"),
    "HSVD V = W, not J W J": ("W = j[:, None] * W * j[None, :]", "W = W"),
    "border identity in the top rows": ("B[m:, nplus:nplus + k] = np.eye(k)", "B[:k, nplus:nplus + k] = np.eye(k)"),
    "columns after the border not shifted": ("B[:m, nplus + k:] = A[:, nplus:]", "B[:m, nplus:n] = A[:, nplus:]"),
    "QR: the method on R, not R^T": ("RT = np.asfortranarray(np.triu(W[:n, :]).T)",
                                     "RT = np.asfortranarray(np.triu(W[:n, :]))"),
    "QR: V without the column permutation": ("V[piv, :] = X", "V[:, :] = X"),
    "dynamic ordering not re-ranked": ("perm = pivots.norm_order(block_norms(G, b))", "perm = list(range(nb))"),
}


def _run_tree(text: str):
    """The pins on a copy of the tree whose oracle/__init__.py is `text`."""
    d = tempfile.mkdtemp(prefix="jo_mutant_tree_")
    try:
        skip = shutil.ignore_patterns("_build", "_lib", "__pycache__", "csrc", "*.so")
        for sub in ("oracle", "tests", "paper_1401_2720_gb300"):
            shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub), ignore=skip)
        with open(os.path.join(d, "oracle", "__init__.py"), "w") as f:
            f.write(text)
        env = {k: v for k, v in os.environ.items() if not k.startswith("JO_")}
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PY_PINS],
                           cwd=d, env=env, capture_output=True, text=True, timeout=900)
        return r.returncode, r.stdout[-2500:] + r.stderr[-1000:]
    finally:
        shutil.rmtree(d, ignore_errors=True)


def test_python_layer_pins_catch_every_planted_mistake():
    base = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    cases = {"unmodified copy": base}
    for name, (old, new) in PY_MUTATIONS.items():
        assert base.count(old) == 1, f"{name}: the text to mutate must occur exactly once"
        cases[name] = base.replace(old, new)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = dict(zip(cases, ex.map(_run_tree, cases.values())))
    rc, out = results.pop("unmodified copy")
    assert rc == 0, out
    survivors = [name for name, (code, _) in results.items() if code == 0]
    assert not survivors, f"planted mistakes no pin catches: {survivors}"
