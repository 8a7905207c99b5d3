/*
 * Oracle for the one-sided Jacobi (H)SVD -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow C.  Only tests/, the smoke check and the benchmark's
 * CPU-baseline leg may load this library; the product path never links or
 * calls it.  It shares no code, header or table with the CUDA path.
 *
 * Compiled with -O2 -ffp-contract=off so that every a*b+c below is two
 * roundings unless R_FMA() is written explicitly.
 *
 * The arithmetic is written once over the scalar type `real` and compiled
 * twice: as double (libjacobi_oracle.so: the parity reference and the timed
 * CPU baseline) and, with -DJO_QUAD, as IEEE binary128 (_Float128,
 * libjacobi_oracle_q.so: ground truth for small sizes and for finite
 * differences of the SVD; its entry points take and return double arrays
 * and are prefixed jo_q_).  eps is the unit roundoff of `real`.
 *
 * The pivot pairs of one p-step are disjoint (Sec. 3), so they may be
 * processed by several threads (jo_set_threads): every pair's arithmetic is
 * the same sequential code whichever thread runs it, so the results are
 * bitwise identical for any thread count.
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
#define __STDC_WANT_IEC_60559_TYPES_EXT__ 1
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#ifdef JO_QUAD
typedef _Float128 real;
/* a multiply then an add, two binary128 roundings (error <= 2^-112
 * relative): glibc's fmaf128 is a software routine ~30x slower, and a
 * ground truth for FP64 results needs no single-rounding fma             */
#define R_FMA(a, b, c) ((a) * (b) + (c))
#define R_SQRT sqrtf128
#define R_FABS fabsf128
#define R_COPYSIGN copysignf128
#define JO_API static __attribute__((unused))
#else
typedef double real;
#define R_FMA fma
#define R_SQRT sqrt
#define R_FABS fabs
#define R_COPYSIGN copysign
#define JO_API
#endif

#ifdef JO_QUAD
#define JO_EPS ((real)0x1p-113)          /* eps of binary128 */
#define JO_SQRT_2_OVER_EPS ((real)0x1p57) /* sqrt(2/eps) = 2^57 exactly */
#else
#define JO_EPS 0x1p-53                 /* eps = 2^-53, App. A */
#define JO_SQRT_2_OVER_EPS 0x1p27      /* sqrt(2/eps) = 2^27 exactly, Sec. 4.3.1 */
#endif

/* ------------------------------------------------------------------------ */
/* Worker threads over the disjoint pivot pairs of one p-step.             */
static int jo_threads = 1;

JO_API void jo_set_threads(int t) { jo_threads = t < 1 ? 1 : t; }

typedef void (*pair_fn)(int i, void *arg, int tid);
typedef struct { pair_fn fn; void *arg; int tid, nthreads, count; } worker_arg;

static void *worker_main(void *p)
{
    worker_arg *w = (worker_arg *)p;
    for (int i = w->tid; i < w->count; i += w->nthreads) w->fn(i, w->arg, w->tid);
    return NULL;
}

/* fn(i, arg, tid) for every i < count; thread tid takes i = tid, tid + T, ... */
static void run_pairs(int count, pair_fn fn, void *arg, int nthreads)
{
    int T = nthreads < count ? nthreads : count;
    if (T <= 1) {
        for (int i = 0; i < count; ++i) fn(i, arg, 0);
        return;
    }
    pthread_t th[64];
    worker_arg wa[64];
    if (T > 64) T = 64;
    for (int t = 0; t < T; ++t) {
        wa[t].fn = fn; wa[t].arg = arg; wa[t].tid = t; wa[t].nthreads = T; wa[t].count = count;
    }
    for (int t = 1; t < T; ++t) pthread_create(&th[t], NULL, worker_main, &wa[t]);
    worker_main(&wa[0]);
    for (int t = 1; t < T; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.3.1, Eqs. (4.3)-(4.6).
 * t = +1: trigonometric rotation (ct = cot, tn = tan, cs = cos);
 * t = -1: hyperbolic rotation (ct = coth, tn = tanh, cs = cosh).
 * cs_form selects cs_1 (1) or cs_2 (2) of Eq. (4.6); the method uses cs_2.
 * Returns 1 if the rotation is proper (cs != 1), else 0.                  */
JO_API int jo_rot(real hpp, real hqq, real hpq, int t, int cs_form,
           real *cs, real *tn)
{
    const real tt = (real)t;
    real h = hqq - tt * hpp;                         /* (4.3) */
    real ct2 = tt * (h / (2.0 * hpq));               /* (4.3) */
    if (t < 0 && R_FABS(ct2) <= 1.0)                     /* R2 */
        ct2 = R_COPYSIGN(1.25, ct2);
    real act2 = R_FABS(ct2);
    real act;                                        /* |ct phi|, (4.4) */
    if (act2 >= JO_SQRT_2_OVER_EPS)
        act = 2.0 * act2;
    else if (t > 0 && act2 < R_SQRT(JO_EPS))
        act = act2 + 1.0;
    else
        act = act2 + R_SQRT(R_FMA(ct2, ct2, tt));
    real tnv = R_COPYSIGN(1.0 / act, ct2);             /* (4.5), R6 */
    real csv;
    if (act >= JO_SQRT_2_OVER_EPS)
        csv = 1.0;
    else if (cs_form == 1)
        csv = 1.0 / R_SQRT(R_FMA(tt * tnv, tnv, 1.0));     /* cs_1 of (4.6) */
    else
        csv = act / R_SQRT(R_FMA(act, act, tt));           /* cs_2 of (4.6) */
    *cs = csv;
    *tn = tnv;
    return csv != 1.0;
}

JO_API void jo_rot_batch(int n, const real *hpp, const real *hqq,
                  const real *hpq, const int *t, int cs_form,
                  real *cs, real *tn, int *proper)
{
    for (int i = 0; i < n; ++i)
        proper[i] = jo_rot(hpp[i], hqq[i], hpq[i], t[i], cs_form, &cs[i], &tn[i]);
}

/* ------------------------------------------------------------------------ */
static real dot(int len, const real *x, const real *y)
{
    real s = 0.0;
    for (int i = 0; i < len; ++i)
        s = R_FMA(x[i], y[i], s);
    return s;
}

/* Apply the rotation of Eq. (4.1) (trig) or (4.2) (hyperbolic) to the
 * column pair (x, y) of length len: an FMA, then a multiply if cs != 1.  */
static void apply_rot(int len, real *x, real *y, int t, real cs, real tn)
{
    for (int i = 0; i < len; ++i) {
        real xi = x[i], yi = y[i], xn, yn;
        if (t > 0) {                       /* [x y] * [[1, tn], [-tn, 1]] */
            xn = R_FMA(-tn, yi, xi);
            yn = R_FMA(tn, xi, yi);
        } else {                           /* [x y] * [[1, tn], [tn, 1]] */
            xn = R_FMA(tn, yi, xi);
            yn = R_FMA(tn, xi, yi);
        }
        if (cs != 1.0) { xn = cs * xn; yn = cs * yn; }
        x[i] = xn;
        y[i] = yn;
    }
}

static void swap_cols(int len, real *x, real *y)
{
    for (int i = 0; i < len; ++i) { real s = x[i]; x[i] = y[i]; y[i] = s; }
}

/* One pivot pair of the one-sided method (Sec. 2 and the subphases 1-7 of
 * Sec. 4.3).  Columns gp, gq (length m) of the matrix being orthogonalized
 * and vp, vq (length nv; nv = 0 skips V).  k < l are the global column
 * indices that decide the rotation type against nplus.  c_eps = eps*R_SQRT(nhat).
 * Returns bit 0: rotation applied (rho), bit 1: proper (cs != 1),
 * bit 2: columns swapped by P2.                                            */
static int jo_pair(int m, real *gp, real *gq, int nv, real *vp, real *vq,
                   int k, int l, int nplus, real c_eps, int bord_lo, int bord_hi)
{
    if ((k >= bord_lo && k < bord_hi) || (l >= bord_lo && l < bord_hi))
        return 0;                                       /* R7 */
    real hpp = dot(m, gp, gp);
    real hqq = dot(m, gq, gq);
    real hpq = dot(m, gp, gq);
    /* relative orthogonality test, Sec. 4.3 subphase 2; R3 */
    int rho = !(hpq == 0.0 || R_FABS(hpq) < c_eps * (R_SQRT(hpp) * R_SQRT(hqq)));
    /* rotation type by the global indices, Sec. 4.3 subphase 4 (0-based:
     * k < nplus <= l means "k <= n+ < l" in the paper's 1-based terms)   */
    int t = (k < nplus && l >= nplus) ? -1 : 1;
    int flags = 0;
    real cs = 1.0, tn = 0.0;
    if (rho) {
        int proper = jo_rot(hpp, hqq, hpq, t, 2, &cs, &tn);
        flags |= 1 | (proper ? 2 : 0);
    }
    int swap = 0;
    if (t > 0) {
        /* Sec. 4.3 subphase 5, R1: new diagonal after the rotation */
        real npp = rho ? R_FMA(-tn, hpq, hpp) : hpp;
        real nqq = rho ? R_FMA(tn, hpq, hqq) : hqq;
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
typedef struct {
    int m, n, nplus, ldg, ldv;
    real *G, *V;
    const int *step;
    real c_eps;
    long long cnt[64][3];                  /* per thread: rotations, proper, swaps */
} hestenes_step;

static void hestenes_pair(int i, void *arg, int tid)
{
    hestenes_step *a = (hestenes_step *)arg;
    int p = a->step[2 * i], q = a->step[2 * i + 1];
    int f = jo_pair(a->m, a->G + (size_t)p * a->ldg, a->G + (size_t)q * a->ldg,
                    a->V ? a->n : 0,
                    a->V ? a->V + (size_t)p * a->ldv : NULL,
                    a->V ? a->V + (size_t)q * a->ldv : NULL,
                    p, q, a->nplus, a->c_eps, 0, 0);
    a->cnt[tid][0] += f & 1;
    a->cnt[tid][1] += (f >> 1) & 1;
    a->cnt[tid][2] += (f >> 2) & 1;
}

JO_API void jo_hestenes(int m, int n, int nplus, real *G, int ldg, real *V, int ldv,
                        const int *table, int nsteps, int npairs, int max_sweeps,
                        double nhat, long long *stats, long long *rot_per_sweep)
{
    hestenes_step a;
    a.m = m; a.n = n; a.nplus = nplus; a.G = G; a.ldg = ldg; a.V = V; a.ldv = ldv;
    a.c_eps = JO_EPS * R_SQRT((real)nhat);
    long long tot_rot = 0, tot_proper = 0, tot_swap = 0;
    int sweep, converged = 0;
    for (sweep = 0; sweep < max_sweeps; ++sweep) {
        long long rot = 0;
        for (int s = 0; s < nsteps; ++s) {
            a.step = table + (size_t)2 * s * npairs;
            memset(a.cnt, 0, sizeof a.cnt);
            run_pairs(npairs, hestenes_pair, &a, jo_threads);
            for (int t = 0; t < 64; ++t) {
                rot += a.cnt[t][0];
                tot_proper += a.cnt[t][1];
                tot_swap += a.cnt[t][2];
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
 * the pivot L[k,k] = R_SQRT(.).  R5: a pivot that is not > 0 is a breakdown,
 * and its column of L is set to zero.  Returns the number of breakdowns.  */
static int cholesky_lower(int bb, real *H, real *L)
{
    int breakdowns = 0;
    memset(L, 0, sizeof(real) * (size_t)bb * bb);
    for (int k = 0; k < bb; ++k) {
        real d = H[k + k * bb];
        for (int j = 0; j < k; ++j)
            d = R_FMA(-L[k + j * bb], L[k + j * bb], d);
        if (!(d > 0.0)) {
            ++breakdowns;
            continue;                              /* column k stays zero */
        }
        real lkk = R_SQRT(d);
        L[k + k * bb] = lkk;
        for (int i = k + 1; i < bb; ++i) {
            real s = H[i + k * bb];
            for (int j = 0; j < k; ++j)
                s = R_FMA(-L[i + j * bb], L[k + j * bb], s);
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
typedef struct {
    int m, n, nplus, b, ldg, ldv, inner_sweeps, bord_lo, bord_hi;
    real *G, *V;
    const int *step_pairs, *inner_table;
    long long cnt[64][4];                  /* per thread: the stats of jo_block_pstep */
} block_step;

static void block_pair(int ip, void *arg, int tid)
{
    block_step *a = (block_step *)arg;
    const int m = a->m, n = a->n, b = a->b, bb = 2 * b;
    real *G = a->G, *V = a->V;
    const int *inner_table = a->inner_table;
    long long *stats = a->cnt[tid];
    const real c_eps = JO_EPS * R_SQRT((real)bb);
    real *X = (real *)malloc(sizeof(real) * (size_t)m * bb);
    real *Y = (real *)malloc(sizeof(real) * (size_t)(m > n ? m : n) * bb);
    real *H = (real *)malloc(sizeof(real) * (size_t)bb * bb);
    real *L = (real *)malloc(sizeof(real) * (size_t)bb * bb);
    real *R = (real *)malloc(sizeof(real) * (size_t)bb * bb);
    real *W = (real *)malloc(sizeof(real) * (size_t)bb * bb);
    int *gidx = (int *)malloc(sizeof(int) * (size_t)bb);

    int P = a->step_pairs[2 * ip], Q = a->step_pairs[2 * ip + 1];
    for (int j = 0; j < b; ++j) {
        gidx[j] = P * b + j;
        gidx[b + j] = Q * b + j;
    }
    /* X = [G_P G_Q] */
    for (int j = 0; j < bb; ++j)
        memcpy(X + (size_t)j * m, G + (size_t)gidx[j] * a->ldg, sizeof(real) * m);
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
    for (int r = 0; r < a->inner_sweeps; ++r) {
        long long a_r = 0;
        for (int s = 0; s < bb - 1; ++s) {
            for (int y = 0; y < b; ++y) {
                int p = inner_table[2 * (s * b + y)];
                int q = inner_table[2 * (s * b + y) + 1];
                int f = jo_pair(bb, R + (size_t)p * bb, R + (size_t)q * bb,
                                bb, W + (size_t)p * bb, W + (size_t)q * bb,
                                gidx[p], gidx[q], a->nplus, c_eps, a->bord_lo, a->bord_hi);
                a_r += f & 1;
                stats[1] += (f >> 1) & 1;
                if (f) changed = 1;
            }
        }
        stats[0] += a_r;
        if (a_r == 0) break;
    }
    if (changed) {                                      /* R4 */
        stats[2] += 1;
        /* (2.9): [A_P A_Q] := [A_P A_Q] V' for A = G, then A = V */
        for (int pass = 0; pass < 2; ++pass) {
            real *A = pass == 0 ? G : V;
            int rows = pass == 0 ? m : n;
            int lda = pass == 0 ? a->ldg : a->ldv;
            if (!A) continue;
            for (int j = 0; j < bb; ++j)
                memcpy(X + (size_t)j * rows, A + (size_t)gidx[j] * lda, sizeof(real) * rows);
            for (int j = 0; j < bb; ++j)
                for (int i = 0; i < rows; ++i) {
                    real s = 0.0;
                    for (int k = 0; k < bb; ++k)
                        s = R_FMA(X[i + (size_t)k * rows], W[k + j * bb], s);
                    Y[i + (size_t)j * rows] = s;
                }
            for (int j = 0; j < bb; ++j)
                memcpy(A + (size_t)gidx[j] * lda, Y + (size_t)j * rows, sizeof(real) * rows);
        }
    }
    free(X); free(Y); free(H); free(L); free(R); free(W); free(gidx);
}

JO_API void jo_block_pstep(int m, int n, int nplus, int b, real *G, int ldg,
                           real *V, int ldv, const int *step_pairs, int npairs,
                           const int *inner_table, int inner_sweeps, int bord_lo, int bord_hi,
                           long long *stats)
{
    block_step a;
    a.m = m; a.n = n; a.nplus = nplus; a.b = b; a.G = G; a.ldg = ldg; a.V = V; a.ldv = ldv;
    a.step_pairs = step_pairs; a.inner_table = inner_table; a.inner_sweeps = inner_sweeps;
    a.bord_lo = bord_lo; a.bord_hi = bord_hi;
    memset(a.cnt, 0, sizeof a.cnt);
    run_pairs(npairs, block_pair, &a, jo_threads);
    for (int t = 0; t < 64; ++t)
        for (int c = 0; c < 4; ++c) stats[c] += a.cnt[t][c];
}

/* Block sweeps of the block-oriented method until a block sweep has no
 * proper rotation (the GPU-wide criterion of Sec. 4.5) or max_sweeps.
 * table: (nb-1) steps x nb/2 block pairs.  stats: [0] sweeps, [1] converged,
 * [2] rotations, [3] proper rotations, [4] block pairs updated,
 * [5] breakdowns; proper_per_sweep[s] (optional) = B of sweep s.          */
JO_API void jo_block_svd(int m, int n, int nplus, int b, real *G, int ldg,
                  real *V, int ldv, const int *table, int nsteps, int npairs,
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
JO_API void jo_colnorms(int m, int n, const real *G, int ldg, real *sigma)
{
    for (int j = 0; j < n; ++j)
        sigma[j] = R_SQRT(dot(m, G + (size_t)j * ldg, G + (size_t)j * ldg));
}

/* ------------------------------------------------------------------------ */
/* Reverse-mode derivative of A = U diag(s) V^T, U m x n with orthonormal
 * columns, V n x n orthogonal, distinct s (the paper has no counterpart; this
 * is the published SVD adjoint):
 *   dA = U [ (F o (U^T dU - dU^T U)) S + diag(ds) + S (F o (V^T dV - dV^T V)) ] V^T
 *        + (I - U U^T) dU S^{-1} V^T,
 *   F_ij = 1 / (s_j^2 - s_i^2) for i != j, F_ii = 0.
 * Written out with plain loops in the order of the formula.               */
JO_API void jo_svd_adjoint(int m, int n, const real *U, const real *s,
                    const real *V, const real *dU, const real *ds,
                    const real *dV, real *dA)
{
    size_t nn = (size_t)n * n;
    real *J = (real *)calloc(nn, sizeof(real));    /* U^T dU */
    real *K = (real *)calloc(nn, sizeof(real));    /* V^T dV */
    real *M = (real *)calloc(nn, sizeof(real));    /* inner bracket */
    real *T = (real *)calloc((size_t)m * n, sizeof(real));
    real *Z = (real *)calloc((size_t)m * n, sizeof(real));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            real a = 0.0, c = 0.0;
            for (int r = 0; r < m; ++r) a = R_FMA(U[r + (size_t)i * m], dU[r + (size_t)j * m], a);
            for (int r = 0; r < n; ++r) c = R_FMA(V[r + (size_t)i * n], dV[r + (size_t)j * n], c);
            J[i + (size_t)j * n] = a;
            K[i + (size_t)j * n] = c;
        }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            real v;
            if (i == j) {
                v = ds[i];
            } else {
                real F = 1.0 / (s[j] * s[j] - s[i] * s[i]);
                real a = J[i + (size_t)j * n] - J[j + (size_t)i * n];
                real c = K[i + (size_t)j * n] - K[j + (size_t)i * n];
                v = F * a * s[j] + s[i] * (F * c);
            }
            M[i + (size_t)j * n] = v;
        }
    /* T = U M */
    for (int r = 0; r < m; ++r)
        for (int j = 0; j < n; ++j) {
            real a = 0.0;
            for (int k = 0; k < n; ++k) a = R_FMA(U[r + (size_t)k * m], M[k + (size_t)j * n], a);
            T[r + (size_t)j * m] = a;
        }
    /* Z = (I - U U^T) dU S^{-1}:  Z = dU S^{-1} - U (U^T dU) S^{-1} */
    for (int r = 0; r < m; ++r)
        for (int j = 0; j < n; ++j) {
            real a = 0.0;
            for (int k = 0; k < n; ++k) a = R_FMA(U[r + (size_t)k * m], J[k + (size_t)j * n], a);
            Z[r + (size_t)j * m] = (dU[r + (size_t)j * m] - a) / s[j];
        }
    /* dA = (T + Z) V^T */
    for (int r = 0; r < m; ++r)
        for (int c = 0; c < n; ++c) {
            real a = 0.0;
            for (int k = 0; k < n; ++k)
                a = R_FMA(T[r + (size_t)k * m] + Z[r + (size_t)k * m], V[c + (size_t)k * n], a);
            dA[r + (size_t)c * m] = a;
        }
    free(J); free(K); free(M); free(T); free(Z);
}

/* ------------------------------------------------------------------------ */
/* DRDSSQ (App. A): the sum of squares of x (length n, finite entries) without
 * overflow or underflow, as ||x||^2 = sigma2 * 2^e with e even and
 * 0.5 <= sigma2 < 2 (sigma2 = 0, e = 0 for a zero vector).  Double build only.
 * Steps, in the appendix's order:
 *   M = max |x_i|, m = min over the non-zero |x_i|;
 *   safe bounds mu~ = sqrt(mu / gamma), nu^ = sqrt(nu / delta_n),
 *   delta_n = 2^ceil(lg n) delta^(1 + ceil(lg n)), gamma = 1 - eps,
 *   delta = 1 + eps, mu / nu the smallest / largest normal numbers;
 *   partial sums: sigma_1^2 of the x_i in [mu~, nu^] (unscaled), sigma_2^2 of
 *   (s_2 x_i) for |x_i| > nu^ (s_2 = 2^l the largest with s_2 M <= nu^),
 *   sigma_0^2 of (s_0 x_i) for |x_i| < mu~ (s_0 = 2^k the smallest with
 *   s_0 m >= mu~), the exponents found by the appendix's frexp comparison;
 *   each non-zero (s_i^-2, sigma_i^2) brought to the common form (even scale
 *   exponent, 0.5 <= sigma^2 < 2) and the partial sums added smallest first,
 *   the smaller rescaled to the larger's scale.                             */
#ifndef JO_QUAD
static int drdssq_exp(double f, double t, int upper)
{
    /* s = 2^j with s f <= t (upper: the largest such j) or s f >= t (the
     * smallest such j): the appendix's frexp rule */
    int fe, te;
    double fy = frexp(f, &fe), ty = frexp(t, &te);
    (void)upper;
    return (f <= t) ? (te - fe) + (fy < ty) : (te - fe) - (fy > ty);
}

static void common_form(double sum, int scale_exp2, int *e, double *f)
{
    /* value = sum * 2^scale_exp2, scale_exp2 even: write as f 2^e with e even,
     * 0.5 <= f < 2 */
    int me;
    double y = frexp(sum, &me);          /* sum = y 2^me, 0.5 <= y < 1 */
    y *= 2.0;                            /* 1 <= y < 2, sum = y 2^(me-1) */
    int m = me - 1;
    int mp = -(((m % 2) + 2) % 2);       /* m' = -(m mod 2) in {-1, 0} */
    *f = ldexp(y, mp);                   /* 2^m' y */
    *e = scale_exp2 + m - mp;            /* stays even */
}

JO_API void jo_drdssq(int n, const double *x, int incx, int *e_out, double *f_out)
{
    const double mu = 0x1p-1022, nu = 0x1.fffffffffffffp+1023, eps = JO_EPS;
    double M = 0.0, mn = nu;
    for (int i = 0; i < n; ++i) {
        double a = fabs(x[(size_t)i * incx]);
        if (a > M) M = a;
        if (a > 0.0 && a < mn) mn = a;
    }
    if (M == 0.0) { *e_out = 0; *f_out = 0.0; return; }
    int L = 0;
    while ((1 << L) < n) ++L;                                   /* ceil(lg n) */
    double delta_n = ldexp(pow(1.0 + eps, 1 + L), L);
    double mu_t = sqrt(mu / (1.0 - eps));
    double nu_h = sqrt(nu / delta_n);
    double s1 = 0.0, s0 = 0.0, s2 = 0.0;
    int k0 = 0, l2 = 0;
    if (M > nu_h) l2 = drdssq_exp(M, nu_h, 1);
    if (mn < mu_t) k0 = drdssq_exp(mn, nextafter(mu_t, 2.0 * mu_t), 0);
    for (int i = 0; i < n; ++i) {
        double a = x[(size_t)i * incx];
        double b = fabs(a);
        if (b > nu_h) { double y = ldexp(a, l2); s2 = fma(y, y, s2); }
        else if (b < mu_t) { double y = ldexp(a, k0); s0 = fma(y, y, s0); }
        else s1 = fma(a, a, s1);
    }
    /* (s_i^-2, sigma_i^2) in common form; ||x||^2 = sigma^2 * 2^(-2 j) */
    int ne = 0, es[3];
    double fs[3];
    if (s0 > 0.0) { common_form(s0, -2 * k0, &es[ne], &fs[ne]); ++ne; }
    if (s1 > 0.0) { common_form(s1, 0, &es[ne], &fs[ne]); ++ne; }
    if (s2 > 0.0) { common_form(s2, -2 * l2, &es[ne], &fs[ne]); ++ne; }
    /* add smallest first: order by (e, f) lexicographically */
    for (int a = 0; a < ne; ++a)
        for (int b = a + 1; b < ne; ++b)
            if (es[b] < es[a] || (es[b] == es[a] && fs[b] < fs[a])) {
                int te = es[a]; es[a] = es[b]; es[b] = te;
                double tf = fs[a]; fs[a] = fs[b]; fs[b] = tf;
            }
    int e = es[0];
    double f = fs[0];
    for (int a = 1; a < ne; ++a) {
        /* smaller (e, f) rescaled to the larger's scale es[a] >= e */
        double sum = ldexp(f, e - es[a]) + fs[a];
        common_form(sum, es[a], &e, &f);
    }
    *e_out = e;
    *f_out = f;
}
#endif

/* ------------------------------------------------------------------------ */
/* QR factorization with column pivoting, A P = Q [R; 0] (the preprocessing of
 * Sec. 2, Eqs. (2.1)-(2.2)) by Householder reflections: at step j the column
 * of largest norm over rows j..m-1 among columns j..n-1 (ties: the lowest
 * index) is swapped to position j, then H_j = I - tau_j v v^T (v_j = 1) with
 * H_j x = beta e_1, beta = -sign(alpha) ||x||, tau = (beta - alpha) / beta,
 * v = x / (alpha - beta), is applied to columns j..n-1.  On return A holds R
 * on and above the diagonal and the v below it; piv[j] = original column now
 * at position j.                                                            */
JO_API void jo_qrcp(int m, int n, real *A, int lda, real *tau, int *piv)
{
    real *nrm = (real *)malloc(sizeof(real) * (size_t)(n > 0 ? n : 1));
    for (int k = 0; k < n; ++k) piv[k] = k;
    for (int j = 0; j < n; ++j) {
        for (int k = j; k < n; ++k)
            nrm[k] = dot(m - j, A + j + (size_t)k * lda, A + j + (size_t)k * lda);
        int best = j;
        for (int k = j + 1; k < n; ++k)
            if (nrm[k] > nrm[best]) best = k;
        if (best != j) {
            swap_cols(m, A + (size_t)j * lda, A + (size_t)best * lda);
            int t = piv[j]; piv[j] = piv[best]; piv[best] = t;
        }
        real *x = A + j + (size_t)j * lda;
        real alpha = x[0];
        real sig = R_SQRT(dot(m - j, x, x));
        if (sig == 0.0) { tau[j] = 0.0; continue; }
        real beta = alpha >= 0.0 ? -sig : sig;
        tau[j] = (beta - alpha) / beta;
        real scal = 1.0 / (alpha - beta);
        x[0] = beta;
        for (int r = 1; r < m - j; ++r) x[r] = x[r] * scal;
        for (int k = j + 1; k < n; ++k) {
            real *c = A + j + (size_t)k * lda;
            real w = c[0];
            for (int r = 1; r < m - j; ++r) w = R_FMA(x[r], c[r], w);
            real f = tau[j] * w;
            c[0] = c[0] - f;
            for (int r = 1; r < m - j; ++r) c[r] = R_FMA(-f, x[r], c[r]);
        }
    }
    free(nrm);
}

/* X := Q X for the Q of jo_qrcp (reflectors in A, tau), X m x ncol.        */
JO_API void jo_apply_q(int m, int n, const real *A, int lda, const real *tau, int ncol, real *X, int ldx)
{
    for (int j = n - 1; j >= 0; --j) {
        if (tau[j] == 0.0) continue;
        const real *v = A + j + (size_t)j * lda;
        for (int k = 0; k < ncol; ++k) {
            real *c = X + j + (size_t)k * ldx;
            real w = c[0];
            for (int r = 1; r < m - j; ++r) w = R_FMA(v[r], c[r], w);
            real f = tau[j] * w;
            c[0] = c[0] - f;
            for (int r = 1; r < m - j; ++r) c[r] = R_FMA(-f, v[r], c[r]);
        }
    }
}

#ifdef JO_QUAD
/* ------------------------------------------------------------------------ */
/* binary128 entry points (double arrays in and out).                       */

/* Pointwise one-sided Jacobi SVD of A (m x n, column-major, ld lda) carried
 * out in binary128 with the pivot table `table` (as for jo_hestenes; the
 * relative test uses nhat = m and eps = 2^-113), then sigma_i = ||g_i||,
 * u_i = g_i / sigma_i, V, stably sorted by sigma non-increasing.  S (n),
 * U (m x n, ld m, may be NULL) and V (n x n, ld n, may be NULL) receive the
 * results rounded to double; stats[0] = sweeps, stats[1] = converged.     */
static void q_svd(int m, int n, const real *A, const int *table, int nsteps, int npairs, int max_sweeps,
                  real *S, real *U, real *V, long long *stats)
{
    real *G = (real *)malloc(sizeof(real) * (size_t)m * n);
    real *W = (real *)malloc(sizeof(real) * (size_t)n * n);
    real *s = (real *)malloc(sizeof(real) * (size_t)n);
    int *ord = (int *)malloc(sizeof(int) * (size_t)n);
    long long st[5];
    memcpy(G, A, sizeof(real) * (size_t)m * n);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) W[i + (size_t)j * n] = (i == j) ? 1.0 : 0.0;
    jo_hestenes(m, n, n, G, m, W, n, table, nsteps, npairs, max_sweeps, (double)m, st, NULL);
    jo_colnorms(m, n, G, m, s);
    /* stable insertion sort of the column indices by sigma, non-increasing */
    for (int j = 0; j < n; ++j) {
        int k = j;
        while (k > 0 && s[ord[k - 1]] < s[j]) { ord[k] = ord[k - 1]; --k; }
        ord[k] = j;
    }
    for (int i = 0; i < n; ++i) {
        const int c = ord[i];
        S[i] = s[c];
        if (U)
            for (int r = 0; r < m; ++r) U[r + (size_t)i * m] = s[c] > 0 ? G[r + (size_t)c * m] / s[c] : 0.0;
        if (V)
            for (int r = 0; r < n; ++r) V[r + (size_t)i * n] = W[r + (size_t)c * n];
    }
    stats[0] = st[0];
    stats[1] = st[1];
    free(G); free(W); free(s); free(ord);
}

void jo_q_set_threads(int t) { jo_set_threads(t); }

/* ||x||^2 in binary128 (no overflow or underflow for double inputs), as
 * f 2^e with 0.5 <= f < 1 (f = 0 for a zero vector), f rounded to double.   */
void jo_q_sumsq(int n, const double *x, int *e_out, double *f_out)
{
    real s = 0.0;
    for (int i = 0; i < n; ++i) s += (real)x[i] * (real)x[i];
    if (s == 0) { *e_out = 0; *f_out = 0.0; return; }
    int e = 0;
    while (s >= 1) { s /= 2; ++e; }
    while (s < 0.5) { s *= 2; --e; }
    *e_out = e;
    *f_out = (double)s;
}

void jo_q_svd(int m, int n, const double *A, int lda, const int *table, int nsteps, int npairs,
              int max_sweeps, double *S, double *U, double *V, long long *stats)
{
    real *Aq = (real *)malloc(sizeof(real) * (size_t)m * n);
    real *Sq = (real *)malloc(sizeof(real) * (size_t)n);
    real *Uq = U ? (real *)malloc(sizeof(real) * (size_t)m * n) : NULL;
    real *Vq = V ? (real *)malloc(sizeof(real) * (size_t)n * n) : NULL;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < m; ++i) Aq[i + (size_t)j * m] = A[i + (size_t)j * lda];
    q_svd(m, n, Aq, table, nsteps, npairs, max_sweeps, Sq, Uq, Vq, stats);
    for (int i = 0; i < n; ++i) S[i] = (double)Sq[i];
    if (U) for (size_t e = 0; e < (size_t)m * n; ++e) U[e] = (double)Uq[e];
    if (V) for (size_t e = 0; e < (size_t)n * n; ++e) V[e] = (double)Vq[e];
    free(Aq); free(Sq); free(Uq); free(Vq);
}

/* L(X) = sum_i w_i sigma_i(X) + <C, U(X) V(X)^T> for the binary128 SVD of X
 * (the products u_i v_i^T do not depend on the signs of the pair).        */
static real q_loss(int m, int n, const real *X, const double *w, const double *C, const int *table, int nsteps,
                   int npairs, int max_sweeps, int *ok)
{
    real *S = (real *)malloc(sizeof(real) * (size_t)n);
    real *U = (real *)malloc(sizeof(real) * (size_t)m * n);
    real *V = (real *)malloc(sizeof(real) * (size_t)n * n);
    long long st[2];
    q_svd(m, n, X, table, nsteps, npairs, max_sweeps, S, U, V, st);
    if (!st[1]) *ok = 0;
    real L = 0.0;
    for (int i = 0; i < n; ++i) L += (real)w[i] * S[i];
    for (int c = 0; c < n; ++c)
        for (int r = 0; r < m; ++r) {
            real uv = 0.0;
            for (int i = 0; i < n; ++i) uv = R_FMA(U[r + (size_t)i * m], V[c + (size_t)i * n], uv);
            L += (real)C[r + (size_t)c * m] * uv;
        }
    free(S); free(U); free(V);
    return L;
}

/* Central difference (L(A + h E) - L(A - h E)) / (2 h) of q_loss in
 * binary128: A +- h E and every step after it are binary128, the quotient is
 * rounded to double.  *ok = 0 if either SVD hit the sweep limit.           */
double jo_q_loss_fd(int m, int n, const double *A, const double *E, double h, const double *w, const double *C,
                    const int *table, int nsteps, int npairs, int max_sweeps, int *ok)
{
    real *Xp = (real *)malloc(sizeof(real) * (size_t)m * n);
    real *Xm = (real *)malloc(sizeof(real) * (size_t)m * n);
    const real hq = (real)h;
    for (size_t e = 0; e < (size_t)m * n; ++e) {
        Xp[e] = (real)A[e] + hq * (real)E[e];
        Xm[e] = (real)A[e] - hq * (real)E[e];
    }
    *ok = 1;
    real Lp = q_loss(m, n, Xp, w, C, table, nsteps, npairs, max_sweeps, ok);
    real Lm = q_loss(m, n, Xm, w, C, table, nsteps, npairs, max_sweeps, ok);
    free(Xp); free(Xm);
    return (double)((Lp - Lm) / (2 * hq));
}
#endif
