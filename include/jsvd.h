/*
 * jsvd.h -- C ABI of the GB300-native block-oriented one-sided Jacobi (H)SVD.
 *
 * Method: V. Novakovic, "A hierarchically blocked Jacobi SVD algorithm for
 * single and multiple graphics processing units" (SIAM J. Sci. Comput.).
 * One block p-step (Sec. 2, Sec. 4) processes every pivot block-pair (G_p, G_q)
 * of a parallel p-strategy (Sec. 3) independently:
 *   H_pq = [G_p G_q]^T [G_p G_q],  H_pq = R^T R (Cholesky, Eq. (2.7), Sec. 4.1)
 *   one inner sweep of the pointwise one-sided Jacobi method on R with the
 *   rotations of Eqs. (4.3)-(4.6), accumulated into V'           (Sec. 4.3)
 *   [G_p G_q] := [G_p G_q] V',  [V_p V_q] := [V_p V_q] V'          (Eq. (2.9))
 * Block sweeps repeat until a sweep performs no proper rotation (Sec. 4.5).
 *
 * Conventions shared by every entry point:
 *  - Matrices are FP64, column-major: element (i,j) of X with leading
 *    dimension ldx is X[i + j*ldx].
 *  - Pointers named "device" must be CUDA device (or managed) memory on the
 *    context's device; the caller owns them.  The library owns its workspace.
 *  - All GPU work is ordered on the stream given to jsvd_create /
 *    jsvd_set_stream (NULL = the legacy default stream).  Calls that report
 *    statistics (info) synchronise that stream before returning.
 *  - Return value: 0 on success; -i if argument i (1-based) is invalid;
 *    a positive JSVD_* status otherwise.  jsvd_status_string() describes it,
 *    jsvd_last_error() gives the context's last detailed message.
 *  - Nothing here is thread-safe on one context; use one context per thread.
 */
#ifndef JSVD_H
#define JSVD_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define JSVD_SUCCESS          0
#define JSVD_NOT_CONVERGED    1  /* sweep limit reached; results are the last iterate */
#define JSVD_ERR_NONFINITE    2  /* input holds Inf or NaN; outputs untouched */
#define JSVD_ERR_CUDA         3  /* a CUDA call failed; see jsvd_last_error() */
#define JSVD_ERR_ALLOC        4  /* workspace allocation failed */
#define JSVD_ERR_UNSUPPORTED  5  /* option combination not supported */
#define JSVD_ERR_TIMEOUT      6  /* a bounded device-side wait gave up */
#define JSVD_ERR_TOO_LARGE    7  /* jsvd_dgesvj_noalloc: problem exceeds its static scratch */
#define JSVD_ERR_INTERNAL     8  /* an internal consistency check failed; see jsvd_last_error() */

/* ---- pivot strategies (Sec. 3) ---------------------------------------- */
#define JSVD_STRAT_MODULUS   0  /* modulus ordering: odd-order modulus completed to even order */
#define JSVD_STRAT_ROW       1  /* R||: p-strategy closest to row-cyclic (Def. 3.1, Alg. 3.1/3.2) */
#define JSVD_STRAT_COL       2  /* C||: p-strategy closest to column-cyclic */
#define JSVD_STRAT_ROW_REV   3  /* reverse of R|| (the paper's default) */
#define JSVD_STRAT_COL_REV   4  /* reverse of C|| */

/* ---- precision modes -------------------------------------------------- */
#define JSVD_PREC_FP64       0  /* all sweeps in FP64 */
#define JSVD_PREC_MIXED      1  /* FP32 block sweeps, then FP64 sweeps to convergence */

/* ---- how the FP64 block contractions are evaluated ----------------------
 * The Gram matrix of a pivot pair (Eq. (2.7)) and the block update (Eq. (2.9))
 * of the FP64 sweeps.  The paper forms both with FP64 arithmetic.  The split
 * forms evaluate them on the bf16 tensor cores from exact digit slices of
 * power-of-two scaled fixed-point operands (exact FP32 accumulation of the
 * digit products, one FP64 rounding per result); with the column scaling they
 * apply, their error is at or below that of the FP64 FMA form.
 *   SPLIT:       Gram and update on tcgen05 with tensor-memory accumulators,
 *                both from 8 8-bit slices (36 products) -- the default.
 *   SPLIT_SYNC:  both from 9 7-bit slices (45 products) on mma.sync.
 * Used by jsvd_dgesvj, jsvd_dhsvj and the FP64 stage of the mixed solver; the
 * batched solver runs the mma.sync forms for both split modes. */
#define JSVD_CONTRACT_FP64        0  /* FP64 FMA kernels */
#define JSVD_CONTRACT_SPLIT       1  /* split digits; tcgen05 update */
#define JSVD_CONTRACT_SPLIT_SYNC  2  /* split digits; mma.sync update */

typedef struct jsvd_ctx *jsvd_ctx_t;

typedef struct {
    int b;               /* block-column width: 8, 16 or 32 (0: chosen by size) */
    int strategy;        /* outer p-strategy, JSVD_STRAT_* (Sec. 3) */
    int inner_strategy;  /* inner p-strategy; -1: same as strategy (Sec. 4.3) */
    int inner_sweeps;    /* M_s: 1 = block-oriented variant, >1 = up to that many
                            inner sweeps (full block variant), Sec. 4.3 */
    int max_sweeps;      /* limit on block sweeps (0: 30) */
    int precision;       /* JSVD_PREC_* */
    int sort;            /* 1: sigma non-increasing (per sign block for the HSVD) */
    int contraction;     /* JSVD_CONTRACT_* (default SPLIT); used by every FP64 solver */
    int dynamic_order;   /* 1: before every block sweep the block-columns are ordered by
                            descending Frobenius norm and the p-strategy is applied to that
                            order (each pair kept as (lower, higher) block index); 0: the
                            static order (single-matrix solvers; the batched one ignores it) */
    int preprocess;      /* jsvd_dgesvj_batched only: 1 = every matrix with m >= 2n (and n <= 1024)
                            is first factored A P = Q [R; 0] by Householder QR with column
                            pivoting and the method runs on the n x n R^T (Sec. 2, Eqs.
                            (2.1)-(2.2)); U = Q [Y; 0], V = P X from R^T = X S Y^T */
} jsvd_opts;

typedef struct {
    int sweeps;                 /* FP64 block sweeps performed */
    int sweeps_low;             /* FP32 block sweeps (mixed precision), else 0 */
    int converged;              /* 1 if the last sweep had no proper rotation */
    int b;                      /* block width used */
    long long rotations;        /* rotations applied (all inner pairs with rho = 1) */
    long long proper_rotations; /* rotations with cos != 1 (Sec. 4.3 subphase 4) */
    long long pairs_updated;    /* block pairs whose V' != I (Eq. (2.9) applied) */
    long long breakdowns;       /* non-positive Cholesky pivots met (column zeroed) */
    double off_norm;            /* max |h_ij|/sqrt(h_ii h_jj) over the pivot Grams of
                                   the last sweep */
} jsvd_info;

/* Fill *opts with the defaults: b = 0, strategy = JSVD_STRAT_ROW_REV,
 * inner_strategy = -1, inner_sweeps = 1, max_sweeps = 30, FP64, sort = 1,
 * contraction = JSVD_CONTRACT_SPLIT, dynamic_order = 0, preprocess = 0. */
void jsvd_default_opts(jsvd_opts *opts);

/* Create a context on CUDA device `device`, issuing work on `stream`
 * (a cudaStream_t, may be NULL).  The context owns a growable workspace. */
int jsvd_create(jsvd_ctx_t *ctx, int device, void *stream);
int jsvd_destroy(jsvd_ctx_t ctx);
int jsvd_set_stream(jsvd_ctx_t ctx, void *stream);
const char *jsvd_last_error(jsvd_ctx_t ctx);
const char *jsvd_status_string(int status);

/* One-sided Jacobi SVD  A = U diag(S) V^T  (Sec. 2, Eqs. (2.3)-(2.9); Sec. 4).
 * Column norms (the kernel Sigma) are computed by DRDSSQ (App. A).  When the
 * largest column norm of A lies outside [2^-400, 2^400] ([2^-50, 2^50] for
 * JSVD_PREC_MIXED), the working copy of A is first scaled by the power of two
 * that brings it to about 1 (exact) and S is scaled back at the end, so that
 * the Gram matrices neither overflow nor underflow; inputs whose column norms
 * span more than about 2^500 around the largest still lose the columns below
 * that range in the Gram matrices (their singular values then come from their
 * own norms; the paper's remedy is a QR factorization at every level).
 *   m, n  : m >= n >= 1 (a wider matrix must be passed transposed: -2)
 *   A     : device, m x n, lda >= m; read only
 *   S     : device, n singular values (non-increasing when opts->sort)
 *   U     : device, m x n (ldu >= m), left singular vectors (u_i = g_i / s_i,
 *           a zero column where s_i = 0)
 *   V     : device, n x n (ldv >= n), right singular vectors; may be NULL
 *   opts  : may be NULL (defaults); info: may be NULL.
 * n that is not a multiple of 2b is bordered internally with an identity
 * block; the border never appears in the outputs.                          */
int jsvd_dgesvj(jsvd_ctx_t ctx, int m, int n, const double *A, int lda,
                double *S, double *U, int ldu, double *V, int ldv,
                const jsvd_opts *opts, jsvd_info *info);

/* Hyperbolic SVD  G = U diag(S) V^T  with  V^T J V = J,
 * J = diag(+1 x n_plus, -1 x (n - n_plus))  (Eq. (2.10); Sec. 4).
 * Pairs of columns k <= n_plus < l are rotated hyperbolically (Eq. (4.2)),
 * the others trigonometrically; only trigonometric pairs are sorted, so S is
 * non-increasing inside each sign block.  Arguments as for jsvd_dgesvj;
 * 0 <= n_plus <= n.  n_plus = n gives exactly jsvd_dgesvj.                 */
int jsvd_dhsvj(jsvd_ctx_t ctx, int m, int n, int n_plus, const double *G, int ldg,
               double *S, double *U, int ldu, double *V, int ldv,
               const jsvd_opts *opts, jsvd_info *info);

/* Batched SVD of `batch` independent matrices of uneven sizes, in one CUDA
 * graph launch (not in the paper; the per-matrix method is the one above).
 *   m, n   : host arrays (batch): m[i] >= n[i] >= 1, n[i] <= 1024 after
 *            bordering to a multiple of 2b
 *   b      : host array of block widths (8, 16 or 32) or NULL: opts->b, else
 *            8 for n <= 256 and 16 above
 *   A      : device, packed: A_i (m_i x n_i, column-major, ld m_i) starts at
 *            A + a_off[i]; read only
 *   S, U, V: device, packed likewise: S_i (n_i) at S + s_off[i], U_i (m_i x n_i,
 *            ld m_i) at U + u_off[i], V_i (n_i x n_i, ld n_i) at V + v_off[i];
 *            V may be NULL (then v_off may be NULL)
 *   a_off, s_off, u_off, v_off: host arrays (batch) of element offsets
 *   infos  : host array (batch) or NULL; filled after the run completes.
 * Every matrix runs the block-oriented method to its own convergence (or
 * opts->max_sweeps); opts->precision must be JSVD_PREC_FP64.  Returns
 * JSVD_NOT_CONVERGED if any matrix hit the sweep limit.                     */
int jsvd_dgesvj_batched(jsvd_ctx_t ctx, int batch, const int *m, const int *n, const int *b,
                        const double *A, const long long *a_off, double *S, const long long *s_off,
                        double *U, const long long *u_off, double *V, const long long *v_off,
                        const jsvd_opts *opts, jsvd_info *infos);

/* Reverse-mode derivative (adjoint) of A_i = U_i diag(S_i) V_i^T for a batch
 * packed as in jsvd_dgesvj_batched (not in the paper; the published SVD
 * adjoint with F_ij = 1/(s_j^2 - s_i^2) evaluated in the split form
 * (a+c)/(2(s_j-s_i)) + (a-c)/(2(s_j+s_i))).  dU, dS, dV are packed like U, S,
 * V and may each be NULL (zero cotangent); dA_i (m_i x n_i, ld m_i) is written
 * at dA + a_off[i].  Needs distinct, positive singular values; U_i with
 * orthonormal columns and V_i orthogonal.  All pointers device except the
 * host arrays m, n and the offsets.                                          */
int jsvd_dgesvj_backward(jsvd_ctx_t ctx, int batch, const int *m, const int *n, const double *U,
                         const long long *u_off, const double *S, const long long *s_off, const double *V,
                         const long long *v_off, const double *dU, const double *dS, const double *dV,
                         double *dA, const long long *a_off);

/* jsvd_dgesvj for callers that cannot allocate device memory (a framework
 * whose memory pool owns all device memory, a process under a cudaMalloc
 * cap).  The paper has no counterpart.  Same arguments and results as
 * jsvd_dgesvj, FP64 only (opts->precision must be JSVD_PREC_FP64), without a
 * context: the work runs on `stream` (a cudaStream_t, NULL = legacy default
 * stream) of the current device.  Like jsvd_dgesvj, the call synchronises
 * that stream once per block sweep (to read the rotation counters) and
 * before it returns.
 * All scratch lives in one static __device__ array of 64 MiB inside the
 * library, which every GPU that loads the library holds until the process
 * exits; the call makes no cudaMalloc, cudaMallocHost or cudaFree and uses no
 * allocating library routine (only a few small host-side C++ vectors).  A
 * problem whose scratch (about 8 * (m+k)*n_pad + 8 * n_pad^2 bytes plus the
 * Gram partials; n_pad = n rounded up to a multiple of 2b) exceeds the array
 * is rejected with JSVD_ERR_TOO_LARGE before any GPU work (m = n = 1024 fits,
 * 2048 does not); S, U and V are then left untouched.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call shares the one array and leaves its
 * contents behind; the solver initialises everything it reads.  Calls whose
 * GPU work overlaps (two streams, two host threads) race on the array.      */
int jsvd_dgesvj_noalloc(int m, int n, const double *A, int lda, double *S, double *U, int ldu,
                        double *V, int ldv, const jsvd_opts *opts, jsvd_info *info, void *stream);

/* The block p-strategy table of order nblocks (even, >= 2) for `strategy`:
 * out_pairs (host, 2*(nblocks-1)*(nblocks/2) ints) receives, p-step by p-step,
 * the 0-based pairs (p, q), p < q.  The R/C families need nblocks = 2^k * o
 * with 2o <= 24 (Alg. 3.1 is run at order 2o, Alg. 3.2 expands it).
 * Host only; needs no GPU.                                                  */
int jsvd_pivot_table(int strategy, int nblocks, int *out_pairs);

/* One block p-step of the FP64 block-oriented method (Sec. 2 and Sec. 4: for
 * every pivot pair (P, Q) of row `step` of the block p-strategy table of
 * order n/b for `strategy`, the Gram matrix (2.7), its Cholesky factor
 * R = L^T (Sec. 4.1), one inner sweep of the pointwise method on R with the
 * same strategy at order 2b (Sec. 4.3, Eqs. (4.3)-(4.6)), and the update
 * (2.9) of G and V), with the kernels and the launch configuration of one
 * p-step of jsvd_dgesvj.  G (device, m x n, column-major, ld ldg) and V
 * (device, n x n, ld ldv; NULL: G only) are read and overwritten in place.
 * b in {8, 16, 32}; n a multiple of 2b with n/b an order the strategy admits
 * (no bordering: jsvd_pivot_table accepts it); 0 <= step < n/b - 1;
 * contraction = JSVD_CONTRACT_*.  No initial scaling is applied, so the
 * squared column norms must stay inside the FP64 range.  info (host, may be
 * NULL) receives the step's rotation, proper-rotation, updated-pair and
 * breakdown counts and the normalised off-diagonal maximum (sweeps = 0).
 * Synchronises the context stream.  Returns 0, a negative argument index, or
 * JSVD_ERR_NONFINITE / JSVD_ERR_UNSUPPORTED / JSVD_ERR_ALLOC / JSVD_ERR_CUDA /
 * JSVD_ERR_TIMEOUT.                                                          */
int jsvd_block_pstep(jsvd_ctx_t ctx, int m, int n, int b, int strategy, int step, double *G, int ldg,
                     double *V, int ldv, int contraction, jsvd_info *info);

/* Sums of squares of the columns of A (device, m x n, ld lda) by DRDSSQ
 * (App. A), the parallel scaled sum the solvers use for the column norms of
 * the kernel Sigma and for their initial scaling: ||a_j||^2 = f[j] 2^e[j]
 * with e[j] even and 0.5 <= f[j] < 2 (0 and 0 for a zero column), without
 * overflow or underflow for any finite input.  e, f: device arrays of n.
 * Synchronises the context stream.                                          */
int jsvd_column_sumsq(jsvd_ctx_t ctx, int m, int n, const double *A, int lda, int *e, double *f);

/* The block p-strategy table of one sweep under the dynamic ordering
 * (jsvd_opts.dynamic_order), computed on the GPU by the kernel the solver
 * uses: perm (device, nblocks) receives the block-columns sorted by
 * block_norms (device, nblocks) descending, ties by index, and pairs (device,
 * 2*(nblocks-1)*(nblocks/2)) the static table of `strategy` with every pair
 * (p, q) replaced by (min, max)(perm[p], perm[q]).  Synchronises the context
 * stream.  Not in the paper (its orderings are static, Sec. 3); exposed so
 * that the remapped table can be checked bit for bit.                       */
int jsvd_sorted_pivot_table(jsvd_ctx_t ctx, int strategy, int nblocks, const double *block_norms, int *perm,
                            int *pairs);

/* Rotation parameters of Eqs. (4.3)-(4.6) (cs_2 form) evaluated on the GPU
 * by the same device code the sweep kernels use.  All arrays are device
 * memory of length count; hyperbolic[i] != 0 selects Eq. (4.2).  proper[i]
 * = 1 if cs != 1.  Exposed so that the rotation arithmetic can be compared
 * bit for bit with an independent CPU evaluation.                          */
int jsvd_rotation_params(jsvd_ctx_t ctx, int count, const double *hpp,
                         const double *hqq, const double *hpq,
                         const int *hyperbolic, double *cs, double *tn,
                         int *proper);

/* The relative orthogonality test of Sec. 4.3 as the sweep kernels evaluate
 * it: rho[i] = 1 unless hpq[i] == 0 or |hpq[i]| < c_eps * (sqrt(hpp[i]) *
 * sqrt(hqq[i])) with every operation correctly rounded.  The kernels decide
 * most cases from the squares and fall back to the square roots inside a
 * guard band; exposed so that the decisions can be compared bit for bit with
 * a CPU evaluation.  All arrays are device memory of length count; the call
 * synchronises the context stream.                                          */
int jsvd_relative_test(jsvd_ctx_t ctx, int count, const double *hpp, const double *hqq,
                       const double *hpq, double c_eps, int *rho);

/* ---- instrumentation ---------------------------------------------------
 * Kernel classes: 0 = Gram partials, 1 = per-pair Cholesky + inner sweep,
 * 2 = block update (Eq. (2.9)) on the solve's main stream (G, or G and V when
 * there is no side stream), 3 = update of V on the side stream (it runs in the
 * gaps of the main stream, so its event time includes waiting for SMs),
 * 4 = everything else (bordering copy, V = I, column norms, output assembly,
 * mixed-precision, batched and adjoint kernels).
 * jsvd_profile(ctx, 1) clears the tallies and starts timing: every launch of
 * a class-0..3 kernel is then bracketed by CUDA events recorded on the stream
 * it runs on and the elapsed times are summed at each sweep boundary.
 * Launch counts and algorithmic FLOP counts are tallied whether or not
 * timing is on (cleared by jsvd_profile).  jsvd_profile_read copies ms[i],
 * launches[i] and flops[i] for i < nclass (nclass <= 5); any pointer may be
 * NULL.  Algorithmic FLOPs per pivot block pair with bb = 2b: Gram
 * m*bb*(bb+1), inner sweep 9*bb*bb*(bb-1) + bb^3/3, update 2*m*bb*bb for G
 * and 2*n*bb*bb for V (only pairs with V' != I), with the caller's m, n.     */
int jsvd_profile(jsvd_ctx_t ctx, int enable);
int jsvd_profile_read(jsvd_ctx_t ctx, double *ms, long long *launches, double *flops, int nclass);

/* FP64 throughput of this GPU, measured now: a DFMA-chain kernel and an FP64
 * mma.sync (m8n8k4) kernel, each filling every SM for about `seconds`
 * (0 < seconds <= 60) after a warm-up of the same length, timed with CUDA
 * events on the context's stream.  Results in TFLOP/s (2 per FMA); either
 * pointer may be NULL.  Allocates and frees a small scratch buffer.        */
int jsvd_fp64_peak(jsvd_ctx_t ctx, double seconds, double *dfma_tflops, double *dmma_tflops);

/* Measured throughput of the bf16 tensor-core instruction the split
 * contractions issue (mma.sync m16n8k16, FP32 accumulation), all SMs busy for
 * about `seconds` (0 < seconds <= 60) after an equal warm-up: the ceiling of
 * those kernels' roofline.  Not part of the paper.  Returns 0, or -1 (null
 * ctx), -2 (seconds out of range), JSVD_ERR_CUDA. */
int jsvd_bf16_mma_peak(jsvd_ctx_t ctx, double seconds, double *tflops);

#ifdef __cplusplus
}
#endif
#endif /* JSVD_H */
