// QR preprocessing of the batched solver (Sec. 2, Eqs. (2.1)-(2.2)).
//
// A matrix with m >= 2n is first factored A P = Q [R; 0] by Householder
// reflections with column pivoting (at step j the remaining column of largest
// norm over rows j..m-1 is moved to position j, ties to the lowest index; the
// norms are recomputed exactly at every step).  The one-sided method then runs
// on the n x n lower-triangular R^T (n rows instead of m per sweep; with the
// pivoting, R^T's columns are close to orthogonal, so fewer sweeps are
// needed).  From R^T = X S Y^T:  A = (Q [Y; 0]) S (P X)^T, i.e.
//   U = Q [Y; 0]   (the reflectors applied to Y bordered by zero rows),
//   V = P X        (row piv[j] of V is row j of X).
// One CTA per matrix for the factorization and for the back-transformation;
// matrices with m < 2n are passed through unchanged.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "driver.h"
#include "jsvd.h"

namespace {

constexpr int kQrThreads = 256;
constexpr int kQrWarps = kQrThreads / 32;
constexpr int kMaxQrN = 1024;

struct QMat {
    int m, n, pre;          // pre: factored (m >= 2n)
    int m_in;               // rows of the matrix the solver sees: n if pre, else m
    long long a_off;        // user A
    long long w_off;        // workspace copy of A (reflectors below the diagonal, R above)
    long long t_off;        // tau, piv (n)
    long long in_off;       // solver input (R^T, n x n; or A, m x n)
    long long u2_off, s2_off, v2_off;       // solver outputs
    long long u_off, s_off, v_off;          // user outputs
};

__device__ __forceinline__ double warp_sum(double s) {
    for (int o = 16; o > 0; o >>= 1) s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, o));
    return s;
}

// Householder QR with column pivoting of one matrix per CTA; writes the
// solver's input (R^T, or the unfactored matrix).
__global__ void __launch_bounds__(kQrThreads) k_qrcp(const QMat *qm, const double *__restrict__ A,
                                                      double *__restrict__ W, double *__restrict__ tau,
                                                      int *__restrict__ piv, double *__restrict__ In) {
    __shared__ double s_norm[kMaxQrN];
    __shared__ double s_scal;
    __shared__ int s_best;
    const QMat M = qm[blockIdx.x];
    const int m = M.m, n = M.n, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const double *a = A + M.a_off;
    double *in = In + M.in_off;
    if (!M.pre) {
        for (long long e = tid; e < (long long)m * n; e += kQrThreads) in[e] = a[e];
        return;
    }
    double *w = W + M.w_off;
    double *t = tau + M.t_off;
    int *p = piv + M.t_off;
    for (long long e = tid; e < (long long)m * n; e += kQrThreads) w[e] = a[e];
    for (int k = tid; k < n; k += kQrThreads) p[k] = k;
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        // squared norms of the trailing columns over rows j..m-1 (fixed order:
        // lane-strided FMA sums, then a shuffle tree)
        for (int k = j + warp; k < n; k += kQrWarps) {
            const double *col = w + (size_t)k * m;
            double s = 0.0;
            for (int r = j + lane; r < m; r += 32) s = __fma_rn(col[r], col[r], s);
            s = warp_sum(s);
            if (lane == 0) s_norm[k] = s;
        }
        __syncthreads();
        if (tid == 0) {
            int best = j;
            for (int k = j + 1; k < n; ++k)
                if (s_norm[k] > s_norm[best]) best = k;
            s_best = best;
        }
        __syncthreads();
        const int best = s_best;
        if (best != j) {
            for (int r = tid; r < m; r += kQrThreads) {
                const double x = w[(size_t)j * m + r];
                w[(size_t)j * m + r] = w[(size_t)best * m + r];
                w[(size_t)best * m + r] = x;
            }
            if (tid == 0) {
                const int q = p[j];
                p[j] = p[best];
                p[best] = q;
                s_norm[best] = s_norm[j];    // (not used again; kept consistent)
            }
        }
        __syncthreads();
        // the reflector H_j = I - tau v v^T with H_j x = beta e_1, v_j = 1
        if (tid == 0) {
            const double alpha = w[(size_t)j * m + j];
            double nrm2 = 0.0;
            for (int r = j; r < m; ++r) nrm2 = __fma_rn(w[(size_t)j * m + r], w[(size_t)j * m + r], nrm2);
            const double sig = __dsqrt_rn(nrm2);
            if (sig == 0.0) {
                t[j] = 0.0;
                s_scal = 0.0;
            } else {
                const double beta = alpha >= 0.0 ? -sig : sig;
                t[j] = __ddiv_rn(beta - alpha, beta);
                s_scal = __drcp_rn(alpha - beta);
                w[(size_t)j * m + j] = beta;
            }
        }
        __syncthreads();
        const double scal = s_scal;
        const double tj = t[j];
        for (int r = j + 1 + tid; r < m; r += kQrThreads) w[(size_t)j * m + r] = scal == 0.0 ? 0.0 : w[(size_t)j * m + r] * scal;
        __syncthreads();
        if (tj != 0.0) {
            // columns k > j: wk = v^T x_k, x_k -= tau wk v
            const double *v = w + (size_t)j * m;
            for (int k = j + 1 + warp; k < n; k += kQrWarps) {
                double *col = w + (size_t)k * m;
                double s = lane == 0 ? col[j] : 0.0;
                for (int r = j + 1 + lane; r < m; r += 32) s = __fma_rn(v[r], col[r], s);
                s = warp_sum(s);
                const double f = tj * s;
                if (lane == 0) col[j] = __fma_rn(-f, 1.0, col[j]);
                for (int r = j + 1 + lane; r < m; r += 32) col[r] = __fma_rn(-f, v[r], col[r]);
            }
        }
        __syncthreads();
    }
    // R^T (n x n, ld n): element (i, c) = R(c, i) for c <= i
    for (long long e = tid; e < (long long)n * n; e += kQrThreads) {
        const int i = (int)(e % n), c = (int)(e / n);
        in[e] = c <= i ? w[(size_t)i * m + c] : 0.0;
    }
}

// Outputs: for a factored matrix U = Q [Y; 0] (reflectors applied in reverse
// order to Y, the solver's V), V = P X (the solver's U, rows permuted), S; for
// the others the solver's outputs are copied.
__global__ void __launch_bounds__(kQrThreads) k_qr_finish(const QMat *qm, const double *__restrict__ W,
                                                           const double *__restrict__ tau,
                                                           const int *__restrict__ piv,
                                                           const double *__restrict__ U2, const double *__restrict__ S2,
                                                           const double *__restrict__ V2, double *__restrict__ U,
                                                           double *__restrict__ S, double *__restrict__ V) {
    const QMat M = qm[blockIdx.x];
    const int m = M.m, n = M.n, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const double *u2 = U2 + M.u2_off, *v2 = V2 + M.v2_off;
    double *u = U + M.u_off;
    for (int k = tid; k < n; k += kQrThreads) S[M.s_off + k] = S2[M.s2_off + k];
    if (!M.pre) {
        for (long long e = tid; e < (long long)m * n; e += kQrThreads) u[e] = u2[e];
        if (V)
            for (long long e = tid; e < (long long)n * n; e += kQrThreads) V[M.v_off + e] = v2[e];
        return;
    }
    const double *w = W + M.w_off;
    const double *t = tau + M.t_off;
    const int *p = piv + M.t_off;
    if (V)
        for (long long e = tid; e < (long long)n * n; e += kQrThreads) {
            const int r = (int)(e % n), c = (int)(e / n);
            V[M.v_off + (size_t)c * n + p[r]] = u2[e];          // solver's U is n x n here
        }
    // U = [Y; 0]
    for (long long e = tid; e < (long long)m * n; e += kQrThreads) {
        const int r = (int)(e % m), c = (int)(e / m);
        u[e] = r < n ? v2[(size_t)c * n + r] : 0.0;
    }
    __syncthreads();
    for (int j = n - 1; j >= 0; --j) {
        const double tj = t[j];
        if (tj != 0.0) {
            const double *v = w + (size_t)j * m;
            for (int c = warp; c < n; c += kQrWarps) {
                double *col = u + (size_t)c * m;
                double s = lane == 0 ? col[j] : 0.0;
                for (int r = j + 1 + lane; r < m; r += 32) s = __fma_rn(v[r], col[r], s);
                s = warp_sum(s);
                const double f = tj * s;
                if (lane == 0) col[j] = col[j] - f;
                for (int r = j + 1 + lane; r < m; r += 32) col[r] = __fma_rn(-f, v[r], col[r]);
            }
        }
        __syncthreads();
    }
}

}  // namespace

// The batched SVD with the QR preprocessing of the matrices with m >= 2n.
int jsvd_ctx::solve_batched_qr(int batch, const int *m, const int *n, const int *bs, const double *A,
                               const long long *a_off, double *S, const long long *s_off, double *U,
                               const long long *u_off, double *V, const long long *v_off, const jsvd_opts *opts,
                               jsvd_info *infos) {
    std::vector<QMat> q(batch);
    std::vector<int> m_in(batch), n_in(batch);
    std::vector<long long> in_off(batch), u2_off(batch), s2_off(batch), v2_off(batch);
    long long w_tot = 0, t_tot = 0, in_tot = 0, u2_tot = 0, s2_tot = 0, v2_tot = 0;
    bool any = false;
    for (int i = 0; i < batch; ++i) {
        QMat &Q = q[i];
        Q.m = m[i];
        Q.n = n[i];
        Q.pre = (m[i] >= 2 * n[i] && n[i] >= 2 && n[i] <= kMaxQrN) ? 1 : 0;
        any = any || Q.pre;
        Q.m_in = Q.pre ? n[i] : m[i];
        Q.a_off = a_off[i];
        Q.w_off = w_tot;
        if (Q.pre) w_tot += (long long)m[i] * n[i];
        Q.t_off = t_tot;
        t_tot += n[i];
        Q.in_off = in_tot;
        in_tot += (long long)Q.m_in * n[i];
        Q.u2_off = u2_tot;
        u2_tot += (long long)Q.m_in * n[i];
        Q.s2_off = s2_tot;
        s2_tot += n[i];
        Q.v2_off = v2_tot;
        v2_tot += (long long)n[i] * n[i];
        Q.u_off = u_off[i];
        Q.s_off = s_off[i];
        Q.v_off = v_off ? v_off[i] : 0;
        m_in[i] = Q.m_in;
        n_in[i] = n[i];
        in_off[i] = Q.in_off;
        u2_off[i] = Q.u2_off;
        s2_off[i] = Q.s2_off;
        v2_off[i] = Q.v2_off;
    }
    if (!any) return solve_batched(batch, m, n, bs, A, a_off, S, s_off, U, u_off, V, v_off, opts, infos);
    int rc;
    if ((rc = ensure(q_meta, sizeof(QMat) * (size_t)batch))) return rc;
    if ((rc = ensure(q_w, sizeof(double) * (size_t)(w_tot > 0 ? w_tot : 1)))) return rc;
    if ((rc = ensure(q_tau, sizeof(double) * (size_t)t_tot))) return rc;
    if ((rc = ensure(q_piv, sizeof(int) * (size_t)t_tot))) return rc;
    if ((rc = ensure(q_in, sizeof(double) * (size_t)in_tot))) return rc;
    if ((rc = ensure(q_u, sizeof(double) * (size_t)u2_tot))) return rc;
    if ((rc = ensure(q_s, sizeof(double) * (size_t)s2_tot))) return rc;
    if ((rc = ensure(q_v, sizeof(double) * (size_t)v2_tot))) return rc;
    // the host image outlives the stream-ordered copy (kept in the context)
    q_meta_host.resize(sizeof(QMat) * (size_t)batch);
    memcpy(q_meta_host.data(), q.data(), q_meta_host.size());
    cudaMemcpyAsync(q_meta.ptr, q_meta_host.data(), q_meta_host.size(), cudaMemcpyHostToDevice, stream);
    k_qrcp<<<batch, kQrThreads, 0, stream>>>((const QMat *)q_meta.ptr, A, (double *)q_w.ptr, (double *)q_tau.ptr,
                                             (int *)q_piv.ptr, (double *)q_in.ptr);
    prof_launches[4] += 1;
    if ((rc = check("qr preprocessing"))) return rc;
    rc = solve_batched(batch, m_in.data(), n_in.data(), bs, (const double *)q_in.ptr, in_off.data(),
                       (double *)q_s.ptr, s2_off.data(), (double *)q_u.ptr, u2_off.data(), (double *)q_v.ptr,
                       v2_off.data(), opts, infos);
    if (rc != JSVD_SUCCESS && rc != JSVD_NOT_CONVERGED) return rc;
    const int rc_solve = rc;
    k_qr_finish<<<batch, kQrThreads, 0, stream>>>((const QMat *)q_meta.ptr, (const double *)q_w.ptr,
                                                  (const double *)q_tau.ptr, (const int *)q_piv.ptr,
                                                  (const double *)q_u.ptr, (const double *)q_s.ptr,
                                                  (const double *)q_v.ptr, U, S, V);
    prof_launches[4] += 1;
    if ((rc = check("qr back-transformation"))) return rc;
    if ((rc = sync("qr back-transformation"))) return rc;
    return rc_solve;
}
