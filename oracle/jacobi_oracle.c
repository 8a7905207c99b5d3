/*
 * Oracle for the one-sided Jacobi (H)SVD -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, sequential FP64 C.  Only tests/, the smoke check and the
 * benchmark's CPU-baseline leg may load this library; the product path never
 * links or calls it.  It shares no code, header or table with the CUDA path.
 *
 * Compiled with -O2 -ffp-contract=off so that every a*b+c below is two
 * roundings unless fma() is written explicitly.
 *
 * Layout: every matrix is column-major; element (i,j) of a matrix with
 * leading dimension ld is X[i + j*ld].  Pivot tables are int arrays of
 * shape [steps][pairs][2], 0-based, with first < second in every pair.
 *
 * Contents (paper: Novakovic, "A hierarchically blocked Jacobi SVD
 * algorithm for single and multiple graphics processing units"):
 *   jo_rot         rotation parameters, Eqs. (4.3)-(4.6)           (Sec. 4.3.1)
 *   jo_hestenes    pointwise one-sided Jacobi, Eqs. (2.3)-(2.5)      (Sec. 2)
 *                  with the relative test, the trig/hyperbolic choice,
 *                  the P2 sorting swap and the counters of Sec. 4.3
 *   jo_block_pstep one p-step of the block-oriented method:
 *                  Gram (2.7), Cholesky (Sec. 4.1), one inner sweep
 *                  (Sec. 4.3), update (2.9)                         (Sec. 2, 4)
 *   jo_block_svd   block sweeps with the proper-rotation stop rule  (Sec. 4.5)
 *   jo_colnorms    sigma_i = ||g_i||_2                              (Sec. 4, Sigma)
 *   jo_svd_adjoint reverse-mode derivative of A = U diag(s) V^T (published
 *                  SVD adjoint; the paper has no counterpart)
 *
 * Readings of the paper taken here (each is repeated where it is used):
 *   R1  diagonal update after a trigonometric rotation is
 *       hpp' = hpp - tan*hpq, hqq' = hqq + tan*hpq (the printed signs in
 *       Sec. 4.3 subphase 5 are inconsistent with (4.1)/(4.3)).
 *   R2  "if numerically |coth 2phi| = 1, substitute 5/4" is read as
 *       |coth 2phi| <= 1 -> sign-preserving 5/4.
 *   R3  hpq == 0 means "relatively orthogonal" (no rotation).
 *   R4  the update (2.9) is skipped only if V' is exactly I (no rotation and
 *       no swap happened).
 *   R5  a non-positive (or NaN) Cholesky pivot is a breakdown: the pivot
 *       column of L is set to zero and the event is counted.
 *   R7  identity bordering [[G, 0], [0, I]] (used when n is not a multiple of
 *       2b): the border columns are exactly orthogonal to every column and
 *       are neither rotated nor swapped by the P2 sort, so they keep their
 *       positions (otherwise a sort swap with a unit-norm border column can
 *       carry a matrix column past its partner for a whole sweep and end the
 *       iteration with the pair unrotated).
 *   R6  sgn(x) is copysign(1, x), so sgn(+0) = +1 and sgn(-0) = -1.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define JO_EPS 0x1p-53                 /* eps = 2^-53, App. A */
#define JO_SQRT_2_OVER_EPS 0x1p27      /* sqrt(2/eps) = 2^27 exactly, Sec. 4.3.1 */

/* ------------------------------------------------------------------------ */
/* Sec. 4.3.1, Eqs. (4.3)-(4.6).
 * t = +1: trigonometric rotation (ct = cot, tn = tan, cs = cos);
 * t = -1: hyperbolic rotation (ct = coth, tn = tanh, cs = cosh).
 * cs_form selects cs_1 (1) or cs_2 (2) of Eq. (4.6); the method uses cs_2.
 * Returns 1 if the rotation is proper (cs != 1), else 0.                  */
int jo_rot(double hpp, double hqq, double hpq, int t, int cs_form,
           double *cs, double *tn)
{
    const double tt = (double)t;
    double h = hqq - tt * hpp;                         /* (4.3) */
    double ct2 = tt * (h / (2.0 * hpq));               /* (4.3) */
    if (t < 0 && fabs(ct2) <= 1.0)                     /* R2 */
        ct2 = copysign(1.25, ct2);
    double act2 = fabs(ct2);
    double act;                                        /* |ct phi|, (4.4) */
    if (act2 >= JO_SQRT_2_OVER_EPS)
        act = 2.0 * act2;
    else if (t > 0 && act2 < sqrt(JO_EPS))
        act = act2 + 1.0;
    else
        act = act2 + sqrt(fma(ct2, ct2, tt));
    double tnv = copysign(1.0 / act, ct2);             /* (4.5), R6 */
    double csv;
    if (act >= JO_SQRT_2_OVER_EPS)
        csv = 1.0;
    else if (cs_form == 1)
        csv = 1.0 / sqrt(fma(tt * tnv, tnv, 1.0));     /* cs_1 of (4.6) */
    else
        csv = act / sqrt(fma(act, act, tt));           /* cs_2 of (4.6) */
    *cs = csv;
    *tn = tnv;
    return csv != 1.0;
}

void jo_rot_batch(int n, const double *hpp, const double *hqq,
                  const double *hpq, const int *t, int cs_form,
                  double *cs, double *tn, int *proper)
{
    for (int i = 0; i < n; ++i)
        proper[i] = jo_rot(hpp[i], hqq[i], hpq[i], t[i], cs_form, &cs[i], &tn[i]);
}

/* ------------------------------------------------------------------------ */
static double dot(int len, const double *x, const double *y)
{
    double s = 0.0;
    for (int i = 0; i < len; ++i)
        s = fma(x[i], y[i], s);
    return s;
}

/* Apply the rotation of Eq. (4.1) (trig) or (4.2) (hyperbolic) to the
 * column pair (x, y) of length len: an FMA, then a multiply if cs != 1.  */
static void apply_rot(int len, double *x, double *y, int t, double cs, double tn)
{
    for (int i = 0; i < len; ++i) {
        double xi = x[i], yi = y[i], xn, yn;
        if (t > 0) {                       /* [x y] * [[1, tn], [-tn, 1]] */
            xn = fma(-tn, yi, xi);
            yn = fma(tn, xi, yi);
        } else {                           /* [x y] * [[1, tn], [tn, 1]] */
            xn = fma(tn, yi, xi);
            yn = fma(tn, xi, yi);
        }
        if (cs != 1.0) { xn = cs * xn; yn = cs * yn; }
        x[i] = xn;
        y[i] = yn;
    }
}

static void swap_cols(int len, double *x, double *y)
{
    for (int i = 0; i < len; ++i) { double s = x[i]; x[i] = y[i]; y[i] = s; }
}

/* One pivot pair of the one-sided method (Sec. 2 and the subphases 1-7 of
 * Sec. 4.3).  Columns gp, gq (length m) of the matrix being orthogonalized
 * and vp, vq (length nv; nv = 0 skips V).  k < l are the global column
 * indices that decide the rotation type against nplus.  c_eps = eps*sqrt(nhat).
 * Returns bit 0: rotation applied (rho), bit 1: proper (cs != 1),
 * bit 2: columns swapped by P2.                                            */
static int jo_pair(int m, double *gp, double *gq, int nv, double *vp, double *vq,
                   int k, int l, int nplus, double c_eps, int bord_lo, int bord_hi)
{
    if ((k >= bord_lo && k < bord_hi) || (l >= bord_lo && l < bord_hi))
        return 0;                                       /* R7 */
    double hpp = dot(m, gp, gp);
    double hqq = dot(m, gq, gq);
    double hpq = dot(m, gp, gq);
    /* relative orthogonality test, Sec. 4.3 subphase 2; R3 */
    int rho = !(hpq == 0.0 || fabs(hpq) < c_eps * (sqrt(hpp) * sqrt(hqq)));
    /* rotation type by the global indices, Sec. 4.3 subphase 4 (0-based:
     * k < nplus <= l means "k <= n+ < l" in the paper's 1-based terms)   */
    int t = (k < nplus && l >= nplus) ? -1 : 1;
    int flags = 0;
    double cs = 1.0, tn = 0.0;
    if (rho) {
        int proper = jo_rot(hpp, hqq, hpq, t, 2, &cs, &tn);
        flags |= 1 | (proper ? 2 : 0);
    }
    int swap = 0;
    if (t > 0) {
        /* Sec. 4.3 subphase 5, R1: new diagonal after the rotation */
        double npp = rho ? fma(-tn, hpq, hpp) : hpp;
        double nqq = rho ? fma(tn, hpq, hqq) : hqq;
        if (l < nplus && npp < nqq) swap = 1;          /* J+ block: non-increasing */
        if (k >= nplus && npp > nqq) swap = 1;         /* J- block: non-decreasing */
    }
    if (rho) {
        apply_rot(m, gp, gq, t, cs, tn);
        if (nv) apply_rot(nv, vp, vq, t, cs, tn);
    }
    if (swap) {
        swap_cols(m, gp, gq);
        if (nv) swap_cols(nv, vp, vq);
        flags |= 4;
    }
    return flags;
}

/* ------------------------------------------------------------------------ */
/* Pointwise one-sided Jacobi (Sec. 2, Eqs. (2.3)-(2.5)), pairs taken in the
 * order of a cyclic p-strategy table of order n (steps x n/2 pairs), one pair
 * after another.  G (m x n) is overwritten by U*Sigma; V (n x n, may be NULL)
 * accumulates the rotations (for the HSVD the accumulated matrix is
 * W = V^{-T}, Sec. 4).  Stops after a sweep with no rotation (the pointwise
 * rule, Sec. 4.5) or after max_sweeps sweeps.
 * stats[0] = sweeps done, stats[1] = 1 if converged, stats[2] = total
 * rotations, stats[3] = total proper rotations, stats[4] = total swaps;
 * rot_per_sweep[s] (if not NULL, length max_sweeps) = rotations in sweep s. */
void jo_hestenes(int m, int n, int nplus, double *G, int ldg, double *V, int ldv,
                 const int *table, int nsteps, int npairs, int max_sweeps,
                 double nhat, long long *stats, long long *rot_per_sweep)
{
    const double c_eps = JO_EPS * sqrt(nhat);
    long long tot_rot = 0, tot_proper = 0, tot_swap = 0;
    int sweep, converged = 0;
    for (sweep = 0; sweep < max_sweeps; ++sweep) {
        long long rot = 0;
        for (int s = 0; s < nsteps; ++s) {
            for (int i = 0; i < npairs; ++i) {
                int p = table[2 * (s * npairs + i)];
                int q = table[2 * (s * npairs + i) + 1];
                int f = jo_pair(m, G + (size_t)p * ldg, G + (size_t)q * ldg,
                                V ? n : 0,
                                V ? V + (size_t)p * ldv : NULL,
                                V ? V + (size_t)q * ldv : NULL,
                                p, q, nplus, c_eps, 0, 0);
                rot += f & 1;
                tot_proper += (f >> 1) & 1;
                tot_swap += (f >> 2) & 1;
            }
        }
        tot_rot += rot;
        if (rot_per_sweep) rot_per_sweep[sweep] = rot;
        if (rot == 0) { converged = 1; ++sweep; break; }
    }
    stats[0] = sweep;
    stats[1] = converged;
    stats[2] = tot_rot;
    stats[3] = tot_proper;
    stats[4] = tot_swap;
}

/* ------------------------------------------------------------------------ */
/* Cholesky H = L L^T without pivoting (Sec. 4.1), on the lower triangle of
 * the bb x bb matrix H (ld = bb).  Column by column; each entry receives its
 * updates -L[i,j]*L[k,j] in the order j = 0, 1, ..., then the division by
 * the pivot L[k,k] = sqrt(.).  R5: a pivot that is not > 0 is a breakdown,
 * and its column of L is set to zero.  Returns the number of breakdowns.  */
static int cholesky_lower(int bb, double *H, double *L)
{
    int breakdowns = 0;
    memset(L, 0, sizeof(double) * (size_t)bb * bb);
    for (int k = 0; k < bb; ++k) {
        double d = H[k + k * bb];
        for (int j = 0; j < k; ++j)
            d = fma(-L[k + j * bb], L[k + j * bb], d);
        if (!(d > 0.0)) {
            ++breakdowns;
            continue;                              /* column k stays zero */
        }
        double lkk = sqrt(d);
        L[k + k * bb] = lkk;
        for (int i = k + 1; i < bb; ++i) {
            double s = H[i + k * bb];
            for (int j = 0; j < k; ++j)
                s = fma(-L[i + j * bb], L[k + j * bb], s);
            L[i + k * bb] = s / lkk;
        }
    }
    return breakdowns;
}

/* One p-step of the block-oriented one-sided Jacobi method (Sec. 2, Sec. 4).
 * Block-columns have width b; bb = 2b is the pivot block order.
 * step_pairs: npairs block pairs (P < Q) of this p-step, 0-based.
 * inner_table: (bb-1) steps x b pairs over 0..bb-1 (the inner p-strategy).
 * inner_sweeps: M_s (1 = block-oriented variant, Sec. 4.3).
 * For each block pair:
 *   H = [G_P G_Q]^T [G_P G_Q]                          (2.7), plain dots
 *   H = L L^T, R = L^T                                 Sec. 4.1
 *   V' = I; inner sweeps on R with the relative test of order nhat = bb,
 *   the rotation type from the global column indices, the P2 sort  Sec. 4.3
 *   [G_P G_Q] := [G_P G_Q] V', [V_P V_Q] := [V_P V_Q] V'  (2.9), R4
 * stats (accumulated): [0] rotations, [1] proper rotations, [2] block pairs
 * updated, [3] Cholesky breakdowns.  Columns in [bord_lo, bord_hi) are an
 * identity border (R7; pass bord_lo = bord_hi for none).                    */
void jo_block_pstep(int m, int n, int nplus, int b, double *G, int ldg,
                    double *V, int ldv, const int *step_pairs, int npairs,
                    const int *inner_table, int inner_sweeps, int bord_lo, int bord_hi,
                    long long *stats)
{
    const int bb = 2 * b;
    const double c_eps = JO_EPS * sqrt((double)bb);
    double *X = (double *)malloc(sizeof(double) * (size_t)m * bb);
    double *Y = (double *)malloc(sizeof(double) * (size_t)(m > n ? m : n) * bb);
    double *H = (double *)malloc(sizeof(double) * (size_t)bb * bb);
    double *L = (double *)malloc(sizeof(double) * (size_t)bb * bb);
    double *R = (double *)malloc(sizeof(double) * (size_t)bb * bb);
    double *W = (double *)malloc(sizeof(double) * (size_t)bb * bb);
    int *gidx = (int *)malloc(sizeof(int) * (size_t)bb);

    for (int ip = 0; ip < npairs; ++ip) {
        int P = step_pairs[2 * ip], Q = step_pairs[2 * ip + 1];
        for (int j = 0; j < b; ++j) {
            gidx[j] = P * b + j;
            gidx[b + j] = Q * b + j;
        }
        /* X = [G_P G_Q] */
        for (int j = 0; j < bb; ++j)
            memcpy(X + (size_t)j * m, G + (size_t)gidx[j] * ldg, sizeof(double) * m);
        /* Gram matrix, lower triangle (2.7) */
        for (int j = 0; j < bb; ++j)
            for (int i = j; i < bb; ++i)
                H[i + j * bb] = dot(m, X + (size_t)i * m, X + (size_t)j * m);
        stats[3] += cholesky_lower(bb, H, L);
        /* R = L^T, V' = I */
        for (int j = 0; j < bb; ++j)
            for (int i = 0; i < bb; ++i) {
                R[i + j * bb] = L[j + i * bb];
                W[i + j * bb] = (i == j) ? 1.0 : 0.0;
            }
        /* inner sweeps (M_s), Sec. 4.3 */
        int changed = 0;
        for (int r = 0; r < inner_sweeps; ++r) {
            long long a_r = 0;
            for (int s = 0; s < bb - 1; ++s) {
                for (int y = 0; y < b; ++y) {
                    int p = inner_table[2 * (s * b + y)];
                    int q = inner_table[2 * (s * b + y) + 1];
                    int f = jo_pair(bb, R + (size_t)p * bb, R + (size_t)q * bb,
                                    bb, W + (size_t)p * bb, W + (size_t)q * bb,
                                    gidx[p], gidx[q], nplus, c_eps, bord_lo, bord_hi);
                    a_r += f & 1;
                    stats[1] += (f >> 1) & 1;
                    if (f) changed = 1;
                }
            }
            stats[0] += a_r;
            if (a_r == 0) break;
        }
        if (!changed)                                   /* R4 */
            continue;
        stats[2] += 1;
        /* (2.9): [A_P A_Q] := [A_P A_Q] V' for A = G, then A = V */
        for (int pass = 0; pass < 2; ++pass) {
            double *A = pass == 0 ? G : V;
            int rows = pass == 0 ? m : n;
            int lda = pass == 0 ? ldg : ldv;
            if (!A) continue;
            for (int j = 0; j < bb; ++j)
                memcpy(X + (size_t)j * rows, A + (size_t)gidx[j] * lda, sizeof(double) * rows);
            for (int j = 0; j < bb; ++j)
                for (int i = 0; i < rows; ++i) {
                    double s = 0.0;
                    for (int k = 0; k < bb; ++k)
                        s = fma(X[i + (size_t)k * rows], W[k + j * bb], s);
                    Y[i + (size_t)j * rows] = s;
                }
            for (int j = 0; j < bb; ++j)
                memcpy(A + (size_t)gidx[j] * lda, Y + (size_t)j * rows, sizeof(double) * rows);
        }
    }
    free(X); free(Y); free(H); free(L); free(R); free(W); free(gidx);
}

/* Block sweeps of the block-oriented method until a block sweep has no
 * proper rotation (the GPU-wide criterion of Sec. 4.5) or max_sweeps.
 * table: (nb-1) steps x nb/2 block pairs.  stats: [0] sweeps, [1] converged,
 * [2] rotations, [3] proper rotations, [4] block pairs updated,
 * [5] breakdowns; proper_per_sweep[s] (optional) = B of sweep s.          */
void jo_block_svd(int m, int n, int nplus, int b, double *G, int ldg,
                  double *V, int ldv, const int *table, int nsteps, int npairs,
                  const int *inner_table, int inner_sweeps, int max_sweeps,
                  int bord_lo, int bord_hi, long long *stats, long long *proper_per_sweep)
{
    long long acc[4] = {0, 0, 0, 0};
    int sweep, converged = 0;
    for (sweep = 0; sweep < max_sweeps; ++sweep) {
        long long before = acc[1];
        for (int s = 0; s < nsteps; ++s)
            jo_block_pstep(m, n, nplus, b, G, ldg, V, ldv,
                           table + (size_t)2 * s * npairs, npairs,
                           inner_table, inner_sweeps, bord_lo, bord_hi, acc);
        long long B = acc[1] - before;
        if (proper_per_sweep) proper_per_sweep[sweep] = B;
        if (B == 0) { converged = 1; ++sweep; break; }
    }
    stats[0] = sweep;
    stats[1] = converged;
    stats[2] = acc[0];
    stats[3] = acc[1];
    stats[4] = acc[2];
    stats[5] = acc[3];
}

/* ------------------------------------------------------------------------ */
/* sigma_j = ||g_j||_2 by a plain sum of squares (Sec. 4, kernel Sigma; the
 * scaled DRDSSQ of App. A reduces to this when nothing over- or underflows). */
void jo_colnorms(int m, int n, const double *G, int ldg, double *sigma)
{
    for (int j = 0; j < n; ++j)
        sigma[j] = sqrt(dot(m, G + (size_t)j * ldg, G + (size_t)j * ldg));
}

/* ------------------------------------------------------------------------ */
/* Reverse-mode derivative of A = U diag(s) V^T, U m x n with orthonormal
 * columns, V n x n orthogonal, distinct s (the paper has no counterpart; this
 * is the published SVD adjoint):
 *   dA = U [ (F o (U^T dU - dU^T U)) S + diag(ds) + S (F o (V^T dV - dV^T V)) ] V^T
 *        + (I - U U^T) dU S^{-1} V^T,
 *   F_ij = 1 / (s_j^2 - s_i^2) for i != j, F_ii = 0.
 * Written out with plain loops in the order of the formula.               */
void jo_svd_adjoint(int m, int n, const double *U, const double *s,
                    const double *V, const double *dU, const double *ds,
                    const double *dV, double *dA)
{
    size_t nn = (size_t)n * n;
    double *J = (double *)calloc(nn, sizeof(double));    /* U^T dU */
    double *K = (double *)calloc(nn, sizeof(double));    /* V^T dV */
    double *M = (double *)calloc(nn, sizeof(double));    /* inner bracket */
    double *T = (double *)calloc((size_t)m * n, sizeof(double));
    double *Z = (double *)calloc((size_t)m * n, sizeof(double));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double a = 0.0, c = 0.0;
            for (int r = 0; r < m; ++r) a = fma(U[r + (size_t)i * m], dU[r + (size_t)j * m], a);
            for (int r = 0; r < n; ++r) c = fma(V[r + (size_t)i * n], dV[r + (size_t)j * n], c);
            J[i + (size_t)j * n] = a;
            K[i + (size_t)j * n] = c;
        }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double v;
            if (i == j) {
                v = ds[i];
            } else {
                double F = 1.0 / (s[j] * s[j] - s[i] * s[i]);
                double a = J[i + (size_t)j * n] - J[j + (size_t)i * n];
                double c = K[i + (size_t)j * n] - K[j + (size_t)i * n];
                v = F * a * s[j] + s[i] * (F * c);
            }
            M[i + (size_t)j * n] = v;
        }
    /* T = U M */
    for (int r = 0; r < m; ++r)
        for (int j = 0; j < n; ++j) {
            double a = 0.0;
            for (int k = 0; k < n; ++k) a = fma(U[r + (size_t)k * m], M[k + (size_t)j * n], a);
            T[r + (size_t)j * m] = a;
        }
    /* Z = (I - U U^T) dU S^{-1}:  Z = dU S^{-1} - U (U^T dU) S^{-1} */
    for (int r = 0; r < m; ++r)
        for (int j = 0; j < n; ++j) {
            double a = 0.0;
            for (int k = 0; k < n; ++k) a = fma(U[r + (size_t)k * m], J[k + (size_t)j * n], a);
            Z[r + (size_t)j * m] = (dU[r + (size_t)j * m] - a) / s[j];
        }
    /* dA = (T + Z) V^T */
    for (int r = 0; r < m; ++r)
        for (int c = 0; c < n; ++c) {
            double a = 0.0;
            for (int k = 0; k < n; ++k)
                a = fma(T[r + (size_t)k * m] + Z[r + (size_t)k * m], V[c + (size_t)k * n], a);
            dA[r + (size_t)c * m] = a;
        }
    free(J); free(K); free(M); free(T); free(Z);
}
