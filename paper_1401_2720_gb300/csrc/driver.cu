// Host driver and C ABI (include/jsvd.h): context and workspace, bordering,
// the block-sweep loop with the GPU-wide stopping rule (Sec. 4.5), singular
// value extraction (kernel Sigma, Sec. 4) and the final ordering.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <vector>

#include "jsvd.h"
#include "jsvd_internal.h"
#include "driver.h"
#include "gemm_fp64.cuh"
#include "rotation.cuh"
#include "sweep_fp64.cuh"

using namespace jsvd;

// ---------------------------------------------------------------------------
// small kernels: bordering copy, V = I, norms, output assembly

// Workspace column c of the bordered matrix: real columns keep their order;
// the k border columns sit at [ins, ins + k) and carry a 1 in row m + (c-ins).
__global__ void k_init_g(const double *__restrict__ A, int lda, int m, int n, int ins, int k,
                         double *__restrict__ G, int ldg, int g_rows, int n_pad,
                         unsigned long long *err) {
    const size_t total = (size_t)g_rows * n_pad;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % g_rows), c = (int)(e / g_rows);
        double v = 0.0;
        if (c >= ins && c < ins + k) {
            v = (r == m + (c - ins)) ? 1.0 : 0.0;
        } else if (r < m) {
            const int src = c < ins ? c : c - k;
            v = A[(size_t)src * lda + r];
            if (!isfinite(v)) atomicOr(err, 1ull);
        }
        G[(size_t)c * ldg + r] = v;
    }
}

__global__ void k_eye(double *__restrict__ V, int ldv, int v_rows, int n_pad) {
    const size_t total = (size_t)v_rows * n_pad;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % v_rows), c = (int)(e / v_rows);
        V[(size_t)c * ldv + r] = (r == c) ? 1.0 : 0.0;
    }
}

// DRDSSQ (App. A) for one column x of length n, one warp: ||x||^2 = f 2^e
// with e even and 0.5 <= f < 2 (f = 0, e = 0 for a zero column), no overflow
// or underflow on the way.  M = max|x_i| and m = min of the non-zero |x_i| by
// warp reductions; the entries inside the safe range [mu~, nu^] are summed
// unscaled, those above (below) it scaled by 2^l (2^k) chosen by the
// appendix's frexp rule; the partial sums are combined in the common form,
// smallest first.
__device__ void common_form_dev(double sum, int scale_exp2, int *e, double *f) {
    int me;
    double y = frexp(sum, &me) * 2.0;                 // 1 <= y < 2, sum = y 2^(me-1)
    const int m = me - 1;
    const int mp = -(((m % 2) + 2) % 2);
    *f = ldexp(y, mp);
    *e = scale_exp2 + m - mp;
}
__device__ int drdssq_exp_dev(double f, double t) {
    int fe, te;
    const double fy = frexp(f, &fe), ty = frexp(t, &te);
    return (f <= t) ? (te - fe) + (fy < ty) : (te - fe) - (fy > ty);
}
__device__ void drdssq_warp(const double *__restrict__ x, int n, int *e_out, double *f_out) {
    const int lane = threadIdx.x & 31;
    const double mu = 0x1p-1022, nu = 0x1.fffffffffffffp+1023, eps = 0x1p-53;
    double M = 0.0, mn = nu;
    for (int r = lane; r < n; r += 32) {
        const double a = fabs(x[r]);
        M = fmax(M, a);
        if (a > 0.0) mn = fmin(mn, a);
    }
    for (int o = 16; o > 0; o >>= 1) {
        M = fmax(M, __shfl_xor_sync(0xffffffffu, M, o));
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
    if (M == 0.0) {
        *e_out = 0;
        *f_out = 0.0;
        return;
    }
    int L = 0;
    while ((1 << L) < n) ++L;                          // ceil(lg n)
    double dl = 1.0;
    for (int i = 0; i <= L; ++i) dl = __dmul_rn(dl, 1.0 + eps);
    const double delta_n = ldexp(dl, L);
    const double mu_t = sqrt(mu / (1.0 - eps)), nu_h = sqrt(nu / delta_n);
    const int l2 = M > nu_h ? drdssq_exp_dev(M, nu_h) : 0;
    const int k0 = mn < mu_t ? drdssq_exp_dev(mn, nextafter(mu_t, 2.0 * mu_t)) : 0;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int r = lane; r < n; r += 32) {
        const double a = x[r], b = fabs(a);
        if (b > nu_h) { const double y = ldexp(a, l2); s2 = __fma_rn(y, y, s2); }
        else if (b < mu_t) { const double y = ldexp(a, k0); s0 = __fma_rn(y, y, s0); }
        else s1 = __fma_rn(a, a, s1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 = __dadd_rn(s0, __shfl_xor_sync(0xffffffffu, s0, o));
        s1 = __dadd_rn(s1, __shfl_xor_sync(0xffffffffu, s1, o));
        s2 = __dadd_rn(s2, __shfl_xor_sync(0xffffffffu, s2, o));
    }
    int ne = 0, es[3];
    double fs[3];
    if (s0 > 0.0) { common_form_dev(s0, -2 * k0, &es[ne], &fs[ne]); ++ne; }
    if (s1 > 0.0) { common_form_dev(s1, 0, &es[ne], &fs[ne]); ++ne; }
    if (s2 > 0.0) { common_form_dev(s2, -2 * l2, &es[ne], &fs[ne]); ++ne; }
    for (int a = 0; a < ne; ++a)
        for (int b = a + 1; b < ne; ++b)
            if (es[b] < es[a] || (es[b] == es[a] && fs[b] < fs[a])) {
                const int te = es[a]; es[a] = es[b]; es[b] = te;
                const double tf = fs[a]; fs[a] = fs[b]; fs[b] = tf;
            }
    int e = es[0];
    double f = fs[0];
    for (int a = 1; a < ne; ++a) common_form_dev(ldexp(f, e - es[a]) + fs[a], es[a], &e, &f);
    *e_out = e;
    *f_out = f;
}

// e[c], f[c] = DRDSSQ of column c (rows [0, rows)); *emax (if not null) =
// max over the non-zero columns of e + 8192.
__global__ void k_col_drdssq(const double *__restrict__ G, int ldg, int rows, int ncols, int *__restrict__ e,
                             double *__restrict__ f, unsigned long long *__restrict__ emax) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (w >= ncols) return;
    int ee;
    double ff;
    drdssq_warp(G + (size_t)w * ldg, rows, &ee, &ff);
    if ((threadIdx.x & 31) == 0) {
        if (e) e[w] = ee;
        if (f) f[w] = ff;
        if (emax && ff > 0.0) atomicMax(emax, (unsigned long long)(ee + 8192));
    }
}

// X *= 2^k (exact for the entries this is applied to: the scale is chosen so
// that no entry over- or underflows beyond what the input already did).
__global__ void k_scale_pow2(double *__restrict__ X, size_t count, int k) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
        X[e] = ldexp(X[e], k);
}

// sigma_c = ||g_c||_2 by DRDSSQ (one warp per column); border[c] = 1 if
// column c has support in the border rows.
__global__ void k_colnorms(const double *__restrict__ G, int ldg, int rows, int m, int k,
                           int n_pad, double *__restrict__ sigma, int *__restrict__ border) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (warp >= n_pad) return;
    const double *g = G + (size_t)warp * ldg;
    int bd = 0;
    for (int r = m + lane; r < m + k && r < rows; r += 32)
        if (g[r] != 0.0) bd = 1;
    bd = __any_sync(0xffffffffu, bd);
    int e;
    double f;
    drdssq_warp(g, rows, &e, &f);            // App. A: ||g||^2 = f 2^e, e even
    if (lane == 0) {
        sigma[warp] = ldexp(__dsqrt_rn(f), e / 2);
        border[warp] = bd;
    }
}

// Output column i takes workspace column perm[i]:
//   U(:, i) = g / sigma (zero column if sigma = 0), S(i) = sigma 2^-unscale
//   (undoing the solver's initial power-of-two scaling of G),
//   V(r, i) = js(r) * W(row(r), perm[i]) * js(i)   (V = J W J for the HSVD).
__global__ void k_finalize(const double *__restrict__ G, int ldg, const double *__restrict__ W,
                           int ldw, const double *__restrict__ sigma, const int *__restrict__ perm,
                           int m, int n, int ins, int k, int nplus, int hyperbolic, int unscale,
                           double *__restrict__ S, double *__restrict__ U, int ldu,
                           double *__restrict__ Vo, int ldv) {
    const int i = blockIdx.y;
    const int c = perm[i];
    const double sg = sigma[c];
    if (blockIdx.x == 0 && threadIdx.x == 0) S[i] = ldexp(sg, -unscale);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
        const double g = G[(size_t)c * ldg + r];
        U[(size_t)i * ldu + r] = sg > 0.0 ? __ddiv_rn(g, sg) : 0.0;
    }
    if (Vo) {
        const double ji = (i < nplus) ? 1.0 : -1.0;
        for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
            const int rw = r < ins ? r : r + k;
            double v = W[(size_t)c * ldw + rw];
            if (hyperbolic) {
                const double jr = (r < nplus) ? 1.0 : -1.0;
                v = v * jr * ji;
            }
            Vo[(size_t)i * ldv + r] = v;
        }
    }
}

// Output position of every workspace column (perm[position] = column): the
// border [ins, ins + k) is skipped; the columns < nplus_w (J = +1) come first,
// then the others; with `sort` each block is ordered by sigma non-increasing,
// ties by column index (a stable sort: the rank of column c is the number of
// block columns that precede it).  A matrix column with support in the border
// rows breaks an invariant of the bordering: bit 1 of *err is set.
__global__ void k_sigma_perm(const double *__restrict__ sigma, const int *__restrict__ border, int n_pad, int ins,
                             int k, int nplus_w, int sort, int *__restrict__ perm,
                             unsigned long long *__restrict__ err) {
    __shared__ double s_sig[256];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const bool real = c < n_pad && !(c >= ins && c < ins + k);
    const bool pos = c < nplus_w;
    const double sc = c < n_pad ? sigma[c] : 0.0;
    int rank = 0;
    for (int base = 0; base < n_pad; base += 256) {
        __syncthreads();
        if (base + (int)threadIdx.x < n_pad) s_sig[threadIdx.x] = sigma[base + threadIdx.x];
        __syncthreads();
        if (!real) continue;
        const int lim = min(256, n_pad - base);
        for (int t = 0; t < lim; ++t) {
            const int o = base + t;
            if ((o >= ins && o < ins + k) || (o < nplus_w) != pos) continue;
            const double so = s_sig[t];
            rank += sort ? (so > sc || (so == sc && o < c)) : (o < c);
        }
    }
    if (!real) return;
    if (border[c]) atomicOr(err, 2ull);
    // the J = -1 block starts after the nplus_w - k real columns of the J = +1 block
    perm[(pos ? 0 : nplus_w - k) + rank] = c;
}

// Dynamic block ordering (one reading of "column-norm-sorted orderings"):
// bnorm[B] = sum of the squared norms of the b columns of block-column B
// (rows [0, rows)), one warp per block-column.
__global__ void k_block_norms(const void *__restrict__ Gv, int fp32, int ldg, int rows, int b, int nb,
                              double *__restrict__ bnorm) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
    if (w >= nb) return;
    double s = 0.0;
    for (int c = 0; c < b; ++c) {
        const size_t col = (size_t)(w * b + c) * ldg;
        for (int r = lane; r < rows; r += 32) {
            const double x = fp32 ? (double)reinterpret_cast<const float *>(Gv)[col + r]
                                  : reinterpret_cast<const double *>(Gv)[col + r];
            s = __fma_rn(x, x, s);
        }
    }
    for (int off = 16; off > 0; off >>= 1) s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, off));
    if (lane == 0) bnorm[w] = s;
}

// perm[i] = the block-column of rank i when ordered by bnorm descending, ties
// by block index (a stable sort: the rank of block B is the number of blocks
// that precede it); then the sweep's table: pair (p, q) of the static table
// becomes (min, max)(perm[p], perm[q]).
__global__ void k_block_order(const double *__restrict__ bnorm, int nb, const int *__restrict__ stab, int npairs_total,
                              int *__restrict__ perm, int *__restrict__ dtab) {
    extern __shared__ int s_perm[];
    for (int B = threadIdx.x; B < nb; B += blockDim.x) {
        const double v = bnorm[B];
        int rank = 0;
        for (int o = 0; o < nb; ++o) {
            const double u = bnorm[o];
            rank += (u > v || (u == v && o < B)) ? 1 : 0;
        }
        s_perm[rank] = B;
    }
    __syncthreads();
    for (int B = threadIdx.x; B < nb; B += blockDim.x) perm[B] = s_perm[B];
    for (int e = threadIdx.x; e < npairs_total; e += blockDim.x) {
        const int p = s_perm[stab[2 * e]], q = s_perm[stab[2 * e + 1]];
        dtab[2 * e] = min(p, q);
        dtab[2 * e + 1] = max(p, q);
    }
}

__global__ void k_to_f32(const double *__restrict__ x, float *__restrict__ y, size_t count) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
        y[e] = (float)x[e];
}

__global__ void k_eye_f32(float *__restrict__ V, int ldv, int v_rows, int n_pad) {
    const size_t total = (size_t)v_rows * n_pad;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % v_rows), c = (int)(e / v_rows);
        V[(size_t)c * ldv + r] = (r == c) ? 1.f : 0.f;
    }
}

// E := J S - I (in place), n x n, ld n, J = diag(+1 x nplus, -1 x (n - nplus)).
__global__ void k_jsub_eye(double *__restrict__ S, int n, int nplus) {
    const size_t total = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % n);
        double v = r < nplus ? S[e] : -S[e];
        if (r == (int)(e / n)) v -= 1.0;
        S[e] = v;
    }
}

// M := I - E/2 + (3/8) E^2 (into E2), the first terms of (I + E)^{-1/2}.
__global__ void k_polar_combine(const double *__restrict__ E, double *__restrict__ E2, int n) {
    const size_t total = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        double v = __fma_rn(0.375, E2[e], -0.5 * E[e]);
        if (e % n == e / n) v += 1.0;
        E2[e] = v;
    }
}

__global__ void k_rot_params(int count, const double *hpp, const double *hqq, const double *hpq,
                             const int *hyp, double *cs, double *tn, int *proper) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const Rot r = rot_params(hpp[i], hqq[i], hpq[i], hyp[i] != 0);
    cs[i] = r.cs;
    tn[i] = r.tn;
    proper[i] = r.cs != 1.0;
}

__global__ void k_rel_test(int count, const double *hpp, const double *hqq, const double *hpq, double c_eps,
                           int *rho) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    rho[i] = needs_rotation(hpp[i], hqq[i], hpq[i], c_eps, __dmul_rn(c_eps, c_eps)) ? 1 : 0;
}

// ---------------------------------------------------------------------------
// context

void jsvd_ctx::set_error(const char *where, cudaError_t e) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
    last_error = buf;
}

int jsvd_ctx::check(const char *where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(where, e);
        return JSVD_ERR_CUDA;
    }
    return 0;
}

int jsvd_ctx::ensure(Buffer &buf, size_t bytes) {
    if (buf.bytes >= bytes) return 0;
    if (buf.ptr) cudaFree(buf.ptr);
    buf.ptr = nullptr;
    buf.bytes = 0;
    cudaError_t e = cudaMalloc(&buf.ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc", e);
        return JSVD_ERR_ALLOC;
    }
    buf.bytes = bytes;
    return 0;
}

int jsvd_ctx::table(int strategy, int n, const int **dev) {
    auto key = std::make_pair(strategy, n);
    auto it = tables.find(key);
    if (it == tables.end()) {
        std::vector<int> t;
        int rc = build_pstrategy(strategy, n, t);
        if (rc) {
            last_error = "no pivot table of order " + std::to_string(n) + " for this strategy";
            return JSVD_ERR_UNSUPPORTED;
        }
        Buffer b;
        if (int r2 = ensure(b, t.size() * sizeof(int))) return r2;
        cudaMemcpyAsync(b.ptr, t.data(), t.size() * sizeof(int), cudaMemcpyHostToDevice, stream);
        if (int r3 = check("table upload")) return r3;
        it = tables.emplace(key, b).first;
        host_tables[key] = t;
    }
    *dev = (const int *)it->second.ptr;
    return 0;
}

int jsvd_ctx::inner_table(int strategy, int BB, const unsigned char **dev) {
    auto key = std::make_pair(strategy, -BB);
    auto it = tables.find(key);
    if (it == tables.end()) {
        std::vector<int> t;
        int rc = build_pstrategy(strategy, BB, t);
        if (rc) {
            last_error = "no inner pivot table of order " + std::to_string(BB);
            return JSVD_ERR_UNSUPPORTED;
        }
        // the host copy is kept in the context, so it outlives the
        // stream-ordered copy
        std::vector<unsigned char> &u = host_inner[BB * 8 + strategy];
        u.assign(t.begin(), t.end());
        Buffer b;
        if (int r2 = ensure(b, u.size())) return r2;
        cudaMemcpyAsync(b.ptr, u.data(), u.size(), cudaMemcpyHostToDevice, stream);
        if (int r3 = check("inner table upload")) return r3;
        it = tables.emplace(key, b).first;
    }
    *dev = (const unsigned char *)it->second.ptr;
    return 0;
}

jsvd_ctx::~jsvd_ctx() {
    if (owns_memory) release_memory();
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    for (cudaEvent_t e : ring_events) cudaEventDestroy(e);
    if (vstream) cudaStreamDestroy(vstream);
    if (mstream) cudaStreamDestroy(mstream);
}

void jsvd_ctx::release_memory() {
    for (Buffer *b : {&g, &v, &part, &vprime, &vflag, &counters, &sigma, &border, &perm, &bslice, &bexp, &dexp, &gexp,
                      &dyn_tab, &dyn_norm, &q_meta, &q_w, &q_tau, &q_piv, &q_in, &q_u, &q_s, &q_v,
                      &g32, &v32,
                      &tmp_a, &tmp_b, &tmp_g, &b_mats, &b_units, &b_g, &b_v, &b_part, &b_vp, &b_vflag,
                      &b_tab, &b_cnt, &b_stat, &b_starts, &b_sigma, &b_border, &b_perm, &b_misc, &b_bsl,
                      &b_bex, &b_dex, &b_gexp, &adj_w,
                      &adj_meta, &adj_desc})
        if (b->ptr) cudaFree(b->ptr);
    for (auto &kv : tables)
        if (kv.second.ptr) cudaFree(kv.second.ptr);
    if (host_counters) cudaFreeHost(host_counters);
}

int jsvd_ctx::ensure_side_stream() {
    if (!vstream) {
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (cudaStreamCreateWithPriority(&mstream, cudaStreamNonBlocking, greatest) != cudaSuccess)
            return check("main stream");
        if (cudaStreamCreateWithPriority(&vstream, cudaStreamNonBlocking, least) != cudaSuccess)
            return check("side stream");
        ring_events.resize(2 * kVRing + 2);
        for (auto &e : ring_events)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return check("ring events");
    }
    return 0;
}

int jsvd_ctx::ensure_events(size_t count) {
    while (events.size() < count) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return check("cudaEventCreate");
        events.push_back(e);
    }
    return 0;
}

int jsvd_ctx::sync(const char *where) {
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        set_error(where, e);
        return JSVD_ERR_CUDA;
    }
    return check(where);
}

// Mixed precision, stage 2.  V32 (FP32, n x n inside an ld-v32 buffer) is
// J-orthogonal (orthogonal for the SVD, J = I) to about the FP32 unit
// roundoff.  Its J-polar factor
//   Q = V32 M^{-1/2},  M = J V32^T J V32 = I + E,
// is exactly J-orthogonal (Q^T J Q = J), and for the SVD it is the polar
// factor.  With ||E|| ~ 1e-6 the series (I + E)^{-1/2} = I - E/2 + 3E^2/8 - ...
// truncated after E^2 leaves ~||E||^3, below the FP64 unit roundoff.  Then
// G := G Q and V := Q, all in FP64.  Columns < nplus have J = +1.
int jsvd_ctx::polar_and_apply(double *G, int ldg, int n, int nplus, const float *V32, int ldv32, double *V,
                              int ldv) {
    int rc;
    const size_t nn = (size_t)n * n;
    if ((rc = ensure(tmp_a, sizeof(double) * nn))) return rc;
    if ((rc = ensure(tmp_b, sizeof(double) * nn))) return rc;
    if ((rc = ensure(tmp_g, sizeof(double) * (size_t)ldg * n))) return rc;
    double *E = (double *)tmp_a.ptr, *E2 = (double *)tmp_b.ptr, *G2 = (double *)tmp_g.ptr;
    // S = V32^T J V32 = V32(+)^T V32(+) - V32(-)^T V32(-)  (row blocks of V32)
    gemm(true, false, Elt::F32, Elt::F32, n, n, nplus, 1.0, V32, ldv32, V32, ldv32, 0.0, E, n, stream);
    if (nplus < n)
        gemm(true, false, Elt::F32, Elt::F32, n, n, n - nplus, -1.0, V32 + nplus, ldv32, V32 + nplus, ldv32, 1.0,
             E, n, stream);
    k_jsub_eye<<<1024, 256, 0, stream>>>(E, n, nplus);
    gemm(false, false, Elt::F64, Elt::F64, n, n, n, 1.0, E, n, E, n, 0.0, E2, n, stream);
    k_polar_combine<<<1024, 256, 0, stream>>>(E, E2, n);
    gemm(false, false, Elt::F32, Elt::F64, n, n, n, 1.0, V32, ldv32, E2, n, 0.0, V, ldv, stream);
    gemm(false, false, Elt::F64, Elt::F64, ldg, n, n, 1.0, G, ldg, V, ldv, 0.0, G2, ldg, stream);
    cudaMemcpyAsync(G, G2, sizeof(double) * (size_t)ldg * n, cudaMemcpyDeviceToDevice, stream);
    prof_launches[4] += 6;
    const double nd = (double)n;
    prof_flops[4] += 2.0 * nd * nd * nd * 3.0 + 2.0 * (double)ldg * nd * nd;
    return check("polar");
}

// ---------------------------------------------------------------------------
// the solver

namespace {

int choose_b(const jsvd_opts &o, int n) {
    if (o.b) return o.b;
    if (n >= 1024) return 32;
    if (n >= 96) return 16;
    return 8;
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Elements of one pair's split right factor (one version) for pivot order BB.
size_t split_b_elems_rt(int BB) {
    switch (BB) {
        case 16: return split_b_elems<16>();
        case 32: return split_b_elems<32>();
        default: return split_b_elems<64>();
    }
}

}  // namespace

// The solve runs on a high-priority stream of the library (the V updates on a
// low-priority side stream fill its gaps), ordered after the caller's earlier
// work on the context stream and before its later work.
int jsvd_ctx::solve(int m, int n, int nplus_in, const double *A, int lda, double *S, double *U, int ldu,
                    double *Vout, int ldv, const jsvd_opts *opts_in, jsvd_info *info, bool hyperbolic) {
    if (!side_streams)
        return solve_on_stream(m, n, nplus_in, A, lda, S, U, ldu, Vout, ldv, opts_in, info, hyperbolic);
    int rc = ensure_side_stream();
    if (rc) return rc;
    cudaStream_t user = stream;
    cudaEventRecord(ring_events[2 * kVRing + 1], user);
    cudaStreamWaitEvent(mstream, ring_events[2 * kVRing + 1], 0);
    stream = mstream;
    rc = solve_on_stream(m, n, nplus_in, A, lda, S, U, ldu, Vout, ldv, opts_in, info, hyperbolic);
    cudaEventRecord(ring_events[2 * kVRing + 1], mstream);
    cudaStreamWaitEvent(user, ring_events[2 * kVRing + 1], 0);
    stream = user;
    return rc;
}

int jsvd_ctx::solve_on_stream(int m, int n, int nplus_in, const double *A, int lda, double *S, double *U,
                              int ldu, double *Vout, int ldv, const jsvd_opts *opts_in, jsvd_info *info,
                              bool hyperbolic) {
    jsvd_opts o;
    jsvd_default_opts(&o);
    if (opts_in) o = *opts_in;
    if (o.max_sweeps <= 0) o.max_sweeps = 30;
    if (o.inner_sweeps <= 0) o.inner_sweeps = 1;
    if (o.inner_strategy < 0) o.inner_strategy = o.strategy;
    if (o.strategy < 0 || o.strategy > 4 || o.inner_strategy > 4) return JSVD_ERR_UNSUPPORTED;
    if (o.precision != JSVD_PREC_FP64 && o.precision != JSVD_PREC_MIXED) {
        last_error = "unknown precision mode";
        return JSVD_ERR_UNSUPPORTED;
    }
    if (o.contraction != JSVD_CONTRACT_FP64 && o.contraction != JSVD_CONTRACT_SPLIT &&
        o.contraction != JSVD_CONTRACT_SPLIT_SYNC) {
        last_error = "unknown contraction mode";
        return JSVD_ERR_UNSUPPORTED;
    }
    const int b = choose_b(o, n);
    if (b != 8 && b != 16 && b != 32) {
        last_error = "block width must be 8, 16 or 32";
        return JSVD_ERR_UNSUPPORTED;
    }
    const int BB = 2 * b;
    const int nplus = hyperbolic ? nplus_in : n;

    // bordering: n_pad = b * n_b with n_b even and admissible for the strategy
    int nb = (int)((n + b - 1) / b);
    nb = admissible_order(o.strategy, nb < 2 ? 2 : nb);
    const int n_pad = nb * b;
    const int k = n_pad - n;
    const int ins = nplus;                    // border inserted at the J boundary
    const int nplus_w = nplus + k;            // border columns are J = +1
    const int m_b = m + k;
    const int g_rows = (int)round_up(m_b, kRowAlign);
    const int v_rows = (int)round_up(n_pad, kRowAlign);
    const int npairs = nb / 2;
    const int g_chunks = g_rows / kGramRows;

    int rc;
    if ((rc = ensure(g, sizeof(double) * (size_t)g_rows * n_pad))) return rc;
    if ((rc = ensure(v, sizeof(double) * (size_t)v_rows * n_pad))) return rc;
    if ((rc = ensure(part, sizeof(double) * (size_t)npairs * g_chunks * (BB * (BB + 1) / 2)))) return rc;
    const int ring = side_streams ? kVRing : 1;
    if ((rc = ensure(vprime, sizeof(double) * (size_t)npairs * BB * BB * ring))) return rc;
    if ((rc = ensure(vflag, sizeof(int) * (size_t)npairs * ring))) return rc;
    // Split contractions update V in the same launch as G (one slot): their
    // issue-heavy update CTAs slowed the latency-bound Jacobi kernel by more
    // than the overlap gained (measured on every workload but the 8192^2 one,
    // where the two were within 2 %).  The FP64 FMA form overlaps the V update
    // on the side stream.
    const bool split = o.contraction == JSVD_CONTRACT_SPLIT || o.contraction == JSVD_CONTRACT_SPLIT_SYNC;
    // the tcgen05 Gram and update (8-bit digit images) or the mma.sync ones (7-bit)
    const bool tc = o.contraction == JSVD_CONTRACT_SPLIT;
    const size_t bsl_pairs = (size_t)npairs * 2 * (size_t)split_b_elems_rt(BB);
    if (split) {
        if ((rc = ensure(bslice, sizeof(uint16_t) * bsl_pairs))) return rc;
        if ((rc = ensure(bexp, sizeof(int) * (size_t)npairs * 2 * BB))) return rc;
        if ((rc = ensure(dexp, sizeof(int) * (size_t)npairs * BB))) return rc;
        if ((rc = ensure(gexp, sizeof(int) * (size_t)n_pad))) return rc;
    }
    if (side_streams && (rc = ensure_side_stream())) return rc;
    if ((rc = ensure(counters, sizeof(unsigned long long) * kCntSize))) return rc;
    if ((rc = ensure(sigma, sizeof(double) * (size_t)n_pad))) return rc;
    if ((rc = ensure(border, sizeof(int) * (size_t)n_pad))) return rc;
    if ((rc = ensure(perm, sizeof(int) * (size_t)n_pad))) return rc;
    if (!host_counters) {
        if (cudaMallocHost(&host_counters, sizeof(unsigned long long) * kCntSize) != cudaSuccess) {
            cudaGetLastError();
            return JSVD_ERR_ALLOC;
        }
    }
    const int *dtab = nullptr;
    const unsigned char *dinner = nullptr;
    if ((rc = table(o.strategy, nb, &dtab))) return rc;
    if ((rc = inner_table(o.inner_strategy, BB, &dinner))) return rc;

    double *G = (double *)g.ptr, *V = (double *)v.ptr;
    unsigned long long *cnt = (unsigned long long *)counters.ptr;
    const bool mixed = o.precision == JSVD_PREC_MIXED;
    const bool want_v = Vout != nullptr || mixed;

    cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * kCntSize, stream);
    k_init_g<<<1024, 256, 0, stream>>>(A, lda, m, n, ins, k, G, g_rows, g_rows, n_pad, cnt + kCntErr);
    prof_launches[4] += 1;
    if (want_v) {
        k_eye<<<1024, 256, 0, stream>>>(V, v_rows, v_rows, n_pad);
        prof_launches[4] += 1;
    }
    // column norms by DRDSSQ (App. A): the largest norm decides the initial
    // scaling below
    k_col_drdssq<<<(n_pad * 32 + 255) / 256, 256, 0, stream>>>(G, g_rows, g_rows, n_pad, nullptr, nullptr,
                                                               cnt + kCntNormExp);
    prof_launches[4] += 1;
    if (profiling && (rc = ensure_events(6 * (size_t)(nb - 1)))) return rc;
    if ((rc = check("init"))) return rc;
    cudaMemcpyAsync(host_counters, cnt, sizeof(unsigned long long) * kCntSize, cudaMemcpyDeviceToHost, stream);
    if ((rc = sync("init"))) return rc;
    if (host_counters[kCntErr]) {
        last_error = "input holds Inf or NaN";
        return JSVD_ERR_NONFINITE;
    }
    // Initial rescaling (App. A: "the input factor should be initially
    // rescaled"): if the largest column norm 2^(e/2) lies outside [2^-lim,
    // 2^lim] (lim = 400 for the FP64 sweeps; 50 when the first sweeps run in
    // FP32), G is multiplied by 2^-(e/2), exactly, so that the Gram matrices
    // (squares of column norms) neither overflow nor underflow; S is scaled
    // back at the end, U and V do not change.
    int prescale = 0;
    if (host_counters[kCntNormExp] != 0) {
        const int half = ((int)host_counters[kCntNormExp] - 8192) / 2;
        const int lim = (o.precision == JSVD_PREC_MIXED) ? 50 : 400;
        if (half > lim || half < -lim) {
            prescale = -half;
            k_scale_pow2<<<1024, 256, 0, stream>>>(G, (size_t)g_rows * n_pad, prescale);
            prof_launches[4] += 1;
        }
    }

    PStepArgs a{};
    a.ldg = g_rows; a.g_rows = g_rows;
    a.ldv = v_rows; a.v_rows = v_rows;
    a.table = dtab; a.npairs = npairs; a.inner = dinner;
    const bool dynamic = o.dynamic_order != 0;
    const int tab_pairs = (nb - 1) * npairs;
    if (dynamic) {
        if ((rc = ensure(dyn_tab, sizeof(int) * 2 * (size_t)tab_pairs + sizeof(int) * nb))) return rc;
        if ((rc = ensure(dyn_norm, sizeof(double) * (size_t)nb))) return rc;
    }
    // order the block-columns by descending norm for the coming sweep (the
    // static table is applied to that order)
    auto reorder = [&]() {
        int *dt = (int *)dyn_tab.ptr;
        k_block_norms<<<(nb * 32 + 255) / 256, 256, 0, stream>>>(a.G, a.fp32, a.ldg, a.g_rows, b, nb,
                                                                 (double *)dyn_norm.ptr);
        k_block_order<<<1, 1024, sizeof(int) * nb, stream>>>((const double *)dyn_norm.ptr, nb, dtab, tab_pairs,
                                                             dt + 2 * tab_pairs, dt);
        prof_launches[4] += 2;
        a.table = dt;
    };
    a.b = b; a.nplus = nplus_w; a.inner_sweeps = o.inner_sweeps;
    a.bord_lo = ins; a.bord_hi = ins + k;
    a.part = (double *)part.ptr; a.g_chunks = g_chunks; a.g_parts = g_chunks;
    a.vprime = (double *)vprime.ptr; a.vflag = (int *)vflag.ptr;
    a.counters = cnt;

    const double bbd = (double)BB;
    const double fl_gram = (double)npairs * m * bbd * (bbd + 1.0);
    // Cholesky once per pair, then 9 bb^2 (bb - 1) per inner sweep performed
    const double fl_chol = bbd * bbd * bbd / 3.0;
    const double fl_inner = 9.0 * bbd * bbd * (bbd - 1.0);
    const double fl_upd_g_pair = 2.0 * (double)m * bbd * bbd;
    const double fl_upd_v_pair = want_v ? 2.0 * (double)n * bbd * bbd : 0.0;

    jsvd_info inf{};
    inf.b = b;
    // Block sweeps until a sweep has no proper rotation (Sec. 4.5), the limit,
    // or (stop_frac > 0) a sweep with fewer proper rotations than stop_frac
    // times the first sweep's.
    auto sweep_loop = [&](int limit, int *done, int *conv, double stop_frac) -> int {
        *done = 0;
        *conv = 0;
        unsigned long long first_proper = 0;
        while (*done < limit) {
            if (dynamic) reorder();
            cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * kCntSize, stream);
            const bool side = side_streams && a.V != nullptr && !a.split;
            const int nslot = side ? ring : 1;
            for (int s = 0; s < nb - 1; ++s) {
                // V' and its flags rotate through a ring of slots so that the V
                // update of step s can still read its slot while steps s+1.. run
                const int slot = s % nslot;
                a.step = s;
                a.vprime = (double *)vprime.ptr + (size_t)slot * npairs * BB * BB;
                a.vflag = (int *)vflag.ptr + (size_t)slot * npairs;
                if (a.split) {
                    a.bslice = (uint16_t *)bslice.ptr + (size_t)slot * bsl_pairs;
                    a.bexp = (int *)bexp.ptr + (size_t)slot * npairs * 2 * BB;
                    a.dexp = (int *)dexp.ptr + (size_t)slot * npairs * BB;
                }
                cudaEvent_t *ev = profiling ? &events[6 * (size_t)s] : nullptr;
                if (side && s >= ring) cudaStreamWaitEvent(stream, ring_events[ring + slot], 0);
                if (ev) cudaEventRecord(ev[0], stream);
                launch_phase(BB, Phase::Gram, a, stream);
                if (ev) cudaEventRecord(ev[1], stream);
                launch_phase(BB, Phase::Jacobi, a, stream);
                if (ev) cudaEventRecord(ev[2], stream);
                if (side) {
                    // [V_p V_q] := [V_p V_q] V' does not feed the next Gram: it runs on
                    // the side stream, overlapping the next steps' Gram and Jacobi
                    cudaEventRecord(ring_events[slot], stream);
                    cudaStreamWaitEvent(vstream, ring_events[slot], 0);
                    if (ev) cudaEventRecord(ev[4], vstream);
                    launch_phase(BB, Phase::UpdateV, a, vstream);
                    if (ev) cudaEventRecord(ev[5], vstream);
                    cudaEventRecord(ring_events[ring + slot], vstream);
                    launch_phase(BB, Phase::UpdateG, a, stream);
                } else {
                    launch_phase(BB, Phase::UpdateGV, a, stream);
                }
                if (ev) cudaEventRecord(ev[3], stream);
            }
            if (side) {
                cudaEventRecord(ring_events[2 * ring], vstream);
                cudaStreamWaitEvent(stream, ring_events[2 * ring], 0);
            }
            prof_launches[0] += nb - 1;
            prof_launches[1] += nb - 1;
            prof_launches[2] += nb - 1;
            if (side) prof_launches[3] += nb - 1;
            if (int r = check("p-step")) return r;
            cudaMemcpyAsync(host_counters, cnt, sizeof(unsigned long long) * kCntSize,
                            cudaMemcpyDeviceToHost, stream);
            if (int r = sync("sweep")) return r;
            ++*done;
            prof_flops[0] += fl_gram * (nb - 1);
            prof_flops[1] += fl_chol * (double)npairs * (nb - 1) + fl_inner * (double)host_counters[kCntInner];
            if (side) {
                prof_flops[2] += fl_upd_g_pair * (double)host_counters[kCntUpdated];
                prof_flops[3] += fl_upd_v_pair * (double)host_counters[kCntUpdated];
            } else {
                prof_flops[2] += (fl_upd_g_pair + fl_upd_v_pair) * (double)host_counters[kCntUpdated];
            }
            if (profiling) {
                for (int s = 0; s < nb - 1; ++s) {
                    const cudaEvent_t *ev = &events[6 * (size_t)s];
                    float ms = 0.f;
                    for (int c = 0; c < 3; ++c) {
                        cudaEventElapsedTime(&ms, ev[c], ev[c + 1]);
                        prof_ms[c] += ms;
                    }
                    if (side) {
                        cudaEventElapsedTime(&ms, ev[4], ev[5]);
                        prof_ms[3] += ms;
                    }
                }
            }
            inf.rotations += (long long)host_counters[kCntRot];
            inf.proper_rotations += (long long)host_counters[kCntProper];
            inf.pairs_updated += (long long)host_counters[kCntUpdated];
            inf.breakdowns += (long long)host_counters[kCntBreak];
            double off;
            unsigned long long bits = host_counters[kCntOff];
            memcpy(&off, &bits, sizeof off);
            inf.off_norm = off;
            if (verbose)
                fprintf(stderr, "[jsvd] %s sweep %d: rotations %llu proper %llu updated %llu off %.3e\n",
                        a.fp32 ? "fp32" : "fp64", *done, host_counters[kCntRot], host_counters[kCntProper],
                        host_counters[kCntUpdated], off);
            if (host_counters[kCntErr] & 4ull) {
                last_error = "a bounded wait of the tensor-core update gave up";
                return JSVD_ERR_TIMEOUT;
            }
            if (host_counters[kCntProper] == 0) { *conv = 1; break; }
            if (*done == 1) first_proper = host_counters[kCntProper];
            if (stop_frac > 0.0 && (double)host_counters[kCntProper] < stop_frac * (double)first_proper) break;
        }
        return 0;
    };

    if (mixed) {
        // Stage 1: FP32 block sweeps on copies G32 = fl32(G), V32 = I, with the
        // relative test at the FP32 unit roundoff.
        if ((rc = ensure(g32, sizeof(float) * (size_t)g_rows * n_pad))) return rc;
        if ((rc = ensure(v32, sizeof(float) * (size_t)v_rows * n_pad))) return rc;
        float *G32 = (float *)g32.ptr, *V32 = (float *)v32.ptr;
        k_to_f32<<<1024, 256, 0, stream>>>(G, G32, (size_t)g_rows * n_pad);
        k_eye_f32<<<1024, 256, 0, stream>>>(V32, v_rows, v_rows, n_pad);
        prof_launches[4] += 2;
        a.G = G32; a.V = V32; a.fp32 = 1; a.eps = 0x1p-24; a.split = 0;
        int low_done = 0, low_conv = 0;
        // The FP32 stage is a preconditioner: it ends once a sweep makes
        // fewer than 30 % as many proper rotations as its first one.  Its later
        // sweeps only polish what the FP64 sweeps redo at FP64 accuracy, and an
        // FP32 sweep costs ~3/4 of a tensor-core FP64 one (8192 x 4096, sigma
        // in [1e-12, 1]: thresholds 0.05 / 0.15 / 0.3 / 0.6 gave 18+21 /
        // 17+21 / 14+21 / 7+27 FP32+FP64 sweeps, 5.12 / 5.03 / 4.73 / 4.94 s)
        if ((rc = sweep_loop(o.max_sweeps, &low_done, &low_conv, 0.3))) return rc;
        inf.sweeps_low = low_done;
        // Stage 2: Q = polar factor of V32 in FP64, G := G Q, V := Q.
        if ((rc = polar_and_apply(G, g_rows, n_pad, nplus_w, V32, v_rows, V, v_rows))) return rc;
    }
    a.G = G; a.V = want_v ? V : nullptr; a.fp32 = 0; a.eps = kEps; a.split = split ? 1 : 0; a.tc = tc ? 1 : 0;
    if (split) {
        // Gram partials of 256 rows; column exponent bounds of the current G
        a.g_chunks = g_rows / kGramRowsSplit;
        a.g_parts = tc ? gram_tc_parts(a) : a.g_chunks;
        a.gexp = (int *)gexp.ptr;
        launch_col_maxexp(G, g_rows, g_rows, n_pad, a.gexp, stream);
        prof_launches[4] += 1;
    }
    int converged = 0, sweeps = 0;
    if ((rc = sweep_loop(o.max_sweeps, &sweeps, &converged, 0.0))) return rc;
    inf.sweeps = sweeps;
    inf.converged = converged;

    // kernel Sigma: column norms, border detection, ordering, outputs
    double *dsig = (double *)sigma.ptr;
    int *dbd = (int *)border.ptr;
    k_colnorms<<<(n_pad * 32 + 255) / 256, 256, 0, stream>>>(G, g_rows, m_b, m, k, n_pad, dsig, dbd);
    k_sigma_perm<<<(n_pad + 255) / 256, 256, 0, stream>>>(dsig, dbd, n_pad, ins, k, nplus_w, o.sort ? 1 : 0,
                                                          (int *)perm.ptr, cnt + kCntErr);
    dim3 grid((std::max(m, n) + 255) / 256 < 8 ? (std::max(m, n) + 255) / 256 : 8, n);
    k_finalize<<<grid, 256, 0, stream>>>(G, g_rows, V, v_rows, dsig, (int *)perm.ptr, m, n, ins, k,
                                         nplus, hyperbolic ? 1 : 0, prescale, S, U, ldu, Vout, ldv);
    prof_launches[4] += 3;  // column norms, ordering, output assembly
    if ((rc = check("finalize"))) return rc;
    cudaMemcpyAsync(host_counters, cnt, sizeof(unsigned long long) * kCntSize, cudaMemcpyDeviceToHost, stream);
    if ((rc = sync("finalize"))) return rc;
    if (host_counters[kCntErr] & 2ull) {
        last_error = "a matrix column has support in the border rows";
        return JSVD_ERR_INTERNAL;
    }
    if (info) *info = inf;
    return converged ? JSVD_SUCCESS : JSVD_NOT_CONVERGED;
}

// One block p-step of the FP64 method on the caller's G and V, with the
// kernels and launch configuration of a p-step of the solve: G and V are
// copied into the row-padded workspaces, the step's Gram, Jacobi and update
// kernels run, and the results are copied back.
int jsvd_ctx::block_pstep(int m, int n, int b, int strategy, int step, double *Gc, int ldg, double *Vc, int ldv,
                          int contraction, jsvd_info *info) {
    if (b != 8 && b != 16 && b != 32) {
        last_error = "block width must be 8, 16 or 32";
        return JSVD_ERR_UNSUPPORTED;
    }
    if (strategy < 0 || strategy > 4) return JSVD_ERR_UNSUPPORTED;
    if (contraction != JSVD_CONTRACT_FP64 && contraction != JSVD_CONTRACT_SPLIT &&
        contraction != JSVD_CONTRACT_SPLIT_SYNC) {
        last_error = "unknown contraction mode";
        return JSVD_ERR_UNSUPPORTED;
    }
    const int BB = 2 * b, nb = n / b, npairs = nb / 2;
    if (n % BB != 0 || admissible_order(strategy, nb) != nb) {
        last_error = "n must be a multiple of 2b with n/b an order the strategy admits";
        return JSVD_ERR_UNSUPPORTED;
    }
    if (step < 0 || step >= nb - 1) return -6;
    const int g_rows = (int)round_up(m, kRowAlign), v_rows = (int)round_up(n, kRowAlign);
    const int g_chunks = g_rows / kGramRows;
    const bool split = contraction != JSVD_CONTRACT_FP64, tc = contraction == JSVD_CONTRACT_SPLIT;
    int rc;
    if ((rc = ensure(g, sizeof(double) * (size_t)g_rows * n))) return rc;
    if (Vc && (rc = ensure(v, sizeof(double) * (size_t)v_rows * n))) return rc;
    if ((rc = ensure(part, sizeof(double) * (size_t)npairs * g_chunks * (BB * (BB + 1) / 2)))) return rc;
    if ((rc = ensure(vprime, sizeof(double) * (size_t)npairs * BB * BB))) return rc;
    if ((rc = ensure(vflag, sizeof(int) * (size_t)npairs))) return rc;
    if ((rc = ensure(counters, sizeof(unsigned long long) * kCntSize))) return rc;
    if (split) {
        if ((rc = ensure(bslice, sizeof(uint16_t) * (size_t)npairs * 2 * split_b_elems_rt(BB)))) return rc;
        if ((rc = ensure(bexp, sizeof(int) * (size_t)npairs * 2 * BB))) return rc;
        if ((rc = ensure(dexp, sizeof(int) * (size_t)npairs * BB))) return rc;
        if ((rc = ensure(gexp, sizeof(int) * (size_t)n))) return rc;
    }
    if (!host_counters) {
        if (cudaMallocHost(&host_counters, sizeof(unsigned long long) * kCntSize) != cudaSuccess) {
            cudaGetLastError();
            return JSVD_ERR_ALLOC;
        }
    }
    const int *dtab = nullptr;
    const unsigned char *dinner = nullptr;
    if ((rc = table(strategy, nb, &dtab))) return rc;
    if ((rc = inner_table(strategy, BB, &dinner))) return rc;
    double *G = (double *)g.ptr, *V = Vc ? (double *)v.ptr : nullptr;
    unsigned long long *cnt = (unsigned long long *)counters.ptr;
    cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * kCntSize, stream);
    // the copies in (zero rows below m and n; no bordering)
    k_init_g<<<1024, 256, 0, stream>>>(Gc, ldg, m, n, n, 0, G, g_rows, g_rows, n, cnt + kCntErr);
    if (V) k_init_g<<<1024, 256, 0, stream>>>(Vc, ldv, n, n, n, 0, V, v_rows, v_rows, n, cnt + kCntErr);

    PStepArgs a{};
    a.G = G; a.ldg = g_rows; a.g_rows = g_rows;
    a.V = V; a.ldv = v_rows; a.v_rows = v_rows;
    a.table = dtab; a.npairs = npairs; a.step = step; a.inner = dinner;
    a.b = b; a.nplus = n; a.bord_lo = n; a.bord_hi = n; a.inner_sweeps = 1;
    a.fp32 = 0; a.eps = kEps;
    a.part = (double *)part.ptr; a.vprime = (double *)vprime.ptr; a.vflag = (int *)vflag.ptr;
    a.counters = cnt;
    a.split = split ? 1 : 0; a.tc = tc ? 1 : 0;
    if (split) {
        a.bslice = (uint16_t *)bslice.ptr; a.bexp = (int *)bexp.ptr; a.dexp = (int *)dexp.ptr;
        a.gexp = (int *)gexp.ptr;
        a.g_chunks = g_rows / kGramRowsSplit;
        a.g_parts = tc ? gram_tc_parts(a) : a.g_chunks;
        launch_col_maxexp(G, g_rows, g_rows, n, a.gexp, stream);
    } else {
        a.g_chunks = g_chunks;
        a.g_parts = g_chunks;
    }
    launch_phase(BB, Phase::Gram, a, stream);
    launch_phase(BB, Phase::Jacobi, a, stream);
    launch_phase(BB, Phase::UpdateGV, a, stream);
    prof_launches[4] += (V ? 2 : 1) + (split ? 1 : 0);
    prof_launches[0] += 1; prof_launches[1] += 1; prof_launches[2] += 1;
    if ((rc = check("p-step"))) return rc;
    cudaMemcpy2DAsync(Gc, sizeof(double) * (size_t)ldg, G, sizeof(double) * (size_t)g_rows, sizeof(double) * m, n,
                      cudaMemcpyDeviceToDevice, stream);
    if (V)
        cudaMemcpy2DAsync(Vc, sizeof(double) * (size_t)ldv, V, sizeof(double) * (size_t)v_rows, sizeof(double) * n,
                          n, cudaMemcpyDeviceToDevice, stream);
    cudaMemcpyAsync(host_counters, cnt, sizeof(unsigned long long) * kCntSize, cudaMemcpyDeviceToHost, stream);
    if ((rc = sync("p-step"))) return rc;
    if (host_counters[kCntErr] & 1ull) {
        last_error = "input holds Inf or NaN";
        return JSVD_ERR_NONFINITE;
    }
    if (host_counters[kCntErr] & 4ull) {
        last_error = "a bounded wait of a tensor-core kernel gave up";
        return JSVD_ERR_TIMEOUT;
    }
    if (info) {
        jsvd_info f{};
        f.b = b;
        f.rotations = (long long)host_counters[kCntRot];
        f.proper_rotations = (long long)host_counters[kCntProper];
        f.pairs_updated = (long long)host_counters[kCntUpdated];
        f.breakdowns = (long long)host_counters[kCntBreak];
        double off;
        const unsigned long long bits = host_counters[kCntOff];
        memcpy(&off, &bits, sizeof off);
        f.off_norm = off;
        *info = f;
    }
    return 0;
}

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

void jsvd_default_opts(jsvd_opts *o) {
    if (!o) return;
    o->b = 0;
    o->strategy = JSVD_STRAT_ROW_REV;
    o->inner_strategy = -1;
    o->inner_sweeps = 1;
    o->max_sweeps = 30;
    o->precision = JSVD_PREC_FP64;
    o->sort = 1;
    o->contraction = JSVD_CONTRACT_SPLIT;
    o->dynamic_order = 0;
    o->preprocess = 0;
}

int jsvd_create(jsvd_ctx_t *ctx, int device, void *stream) {
    if (!ctx) return -1;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return -2;
    }
    if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return JSVD_ERR_CUDA; }
    jsvd_ctx *c = new jsvd_ctx();
    c->device = device;
    c->stream = (cudaStream_t)stream;
    const char *v = getenv("JSVD_VERBOSE");
    c->verbose = v && *v && *v != '0';
    *ctx = c;
    return 0;
}

int jsvd_destroy(jsvd_ctx_t ctx) {
    if (!ctx) return -1;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    delete ctx;
    return 0;
}

int jsvd_set_stream(jsvd_ctx_t ctx, void *stream) {
    if (!ctx) return -1;
    ctx->stream = (cudaStream_t)stream;
    return 0;
}

int jsvd_profile(jsvd_ctx_t ctx, int enable) {
    if (!ctx) return -1;
    ctx->profiling = enable != 0;
    for (int i = 0; i < jsvd_ctx::kClasses; ++i) {
        ctx->prof_ms[i] = 0.0;
        ctx->prof_launches[i] = 0;
        ctx->prof_flops[i] = 0.0;
    }
    return 0;
}

int jsvd_profile_read(jsvd_ctx_t ctx, double *ms, long long *launches, double *flops, int nclass) {
    if (!ctx) return -1;
    if (nclass < 0 || nclass > jsvd_ctx::kClasses) return -5;
    for (int i = 0; i < nclass; ++i) {
        if (ms) ms[i] = ctx->prof_ms[i];
        if (launches) launches[i] = ctx->prof_launches[i];
        if (flops) flops[i] = ctx->prof_flops[i];
    }
    return 0;
}

const char *jsvd_last_error(jsvd_ctx_t ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

const char *jsvd_status_string(int s) {
    switch (s) {
        case JSVD_SUCCESS: return "success";
        case JSVD_NOT_CONVERGED: return "sweep limit reached before convergence";
        case JSVD_ERR_NONFINITE: return "input holds Inf or NaN";
        case JSVD_ERR_CUDA: return "CUDA error";
        case JSVD_ERR_ALLOC: return "workspace allocation failed";
        case JSVD_ERR_UNSUPPORTED: return "unsupported option";
        case JSVD_ERR_TIMEOUT: return "bounded device wait gave up";
        case JSVD_ERR_TOO_LARGE: return "problem exceeds the static scratch of the no-allocation entry point";
        case JSVD_ERR_INTERNAL: return "internal consistency check failed";
        default: return s < 0 ? "invalid argument" : "unknown status";
    }
}

int jsvd_dgesvj(jsvd_ctx_t ctx, int m, int n, const double *A, int lda, double *S, double *U,
                int ldu, double *V, int ldv, const jsvd_opts *opts, jsvd_info *info) {
    if (!ctx) return -1;
    if (m < 1 || m < n) return -2;
    if (n < 1) return -3;
    if (!A) return -4;
    if (lda < m) return -5;
    if (!S) return -6;
    if (!U) return -7;
    if (ldu < m) return -8;
    if (V && ldv < n) return -10;
    cudaSetDevice(ctx->device);
    return ctx->solve(m, n, n, A, lda, S, U, ldu, V, ldv, opts, info, false);
}

int jsvd_dhsvj(jsvd_ctx_t ctx, int m, int n, int n_plus, const double *G, int ldg, double *S,
               double *U, int ldu, double *V, int ldv, const jsvd_opts *opts, jsvd_info *info) {
    if (!ctx) return -1;
    if (m < 1 || m < n) return -2;
    if (n < 1) return -3;
    if (n_plus < 0 || n_plus > n) return -4;
    if (!G) return -5;
    if (ldg < m) return -6;
    if (!S) return -7;
    if (!U) return -8;
    if (ldu < m) return -9;
    if (V && ldv < n) return -11;
    cudaSetDevice(ctx->device);
    return ctx->solve(m, n, n_plus, G, ldg, S, U, ldu, V, ldv, opts, info, n_plus < n);
}

int jsvd_block_pstep(jsvd_ctx_t ctx, int m, int n, int b, int strategy, int step, double *G, int ldg, double *V,
                     int ldv, int contraction, jsvd_info *info) {
    if (!ctx) return -1;
    if (m < 1) return -2;
    if (n < 2) return -3;
    if (!G) return -7;
    if (ldg < m) return -8;
    if (V && ldv < n) return -10;
    cudaSetDevice(ctx->device);
    return ctx->block_pstep(m, n, b, strategy, step, G, ldg, V, ldv, contraction, info);
}

int jsvd_column_sumsq(jsvd_ctx_t ctx, int m, int n, const double *A, int lda, int *e, double *f) {
    if (!ctx) return -1;
    if (m < 1) return -2;
    if (n < 1) return -3;
    if (!A) return -4;
    if (lda < m) return -5;
    if (!e) return -6;
    if (!f) return -7;
    cudaSetDevice(ctx->device);
    k_col_drdssq<<<(n * 32 + 255) / 256, 256, 0, ctx->stream>>>(A, lda, m, n, e, f, nullptr);
    if (int rc = ctx->check("column sums of squares")) return rc;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return ctx->check("column sums of squares sync") ? JSVD_ERR_CUDA
                                                                                                         : JSVD_ERR_CUDA;
    return 0;
}

int jsvd_sorted_pivot_table(jsvd_ctx_t ctx, int strategy, int nblocks, const double *block_norms, int *perm,
                            int *pairs) {
    if (!ctx) return -1;
    if (strategy < 0 || strategy > 4) return -2;
    if (nblocks < 2 || nblocks % 2 || nblocks > 8192) return -3;
    if (!block_norms) return -4;
    if (!perm) return -5;
    if (!pairs) return -6;
    cudaSetDevice(ctx->device);
    const int *stab = nullptr;
    if (int rc = ctx->table(strategy, nblocks, &stab)) return rc;
    const int total = (nblocks - 1) * (nblocks / 2);
    k_block_order<<<1, 1024, sizeof(int) * nblocks, ctx->stream>>>(block_norms, nblocks, stab, total, perm, pairs);
    if (int rc = ctx->check("sorted pivot table")) return rc;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return ctx->check("sorted pivot table sync") ? JSVD_ERR_CUDA
                                                                                                        : JSVD_ERR_CUDA;
    return 0;
}

int jsvd_rotation_params(jsvd_ctx_t ctx, int count, const double *hpp, const double *hqq,
                         const double *hpq, const int *hyperbolic, double *cs, double *tn,
                         int *proper) {
    if (!ctx) return -1;
    if (count < 0) return -2;
    if (count == 0) return 0;
    cudaSetDevice(ctx->device);
    k_rot_params<<<(count + 255) / 256, 256, 0, ctx->stream>>>(count, hpp, hqq, hpq, hyperbolic, cs, tn, proper);
    if (int rc = ctx->check("rotation params")) return rc;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return ctx->check("rotation sync") ? JSVD_ERR_CUDA : JSVD_ERR_CUDA;
    return 0;
}

int jsvd_relative_test(jsvd_ctx_t ctx, int count, const double *hpp, const double *hqq, const double *hpq,
                       double c_eps, int *rho) {
    if (!ctx) return -1;
    if (count < 0) return -2;
    if (count == 0) return 0;
    cudaSetDevice(ctx->device);
    k_rel_test<<<(count + 255) / 256, 256, 0, ctx->stream>>>(count, hpp, hqq, hpq, c_eps, rho);
    if (int rc = ctx->check("relative test")) return rc;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return JSVD_ERR_CUDA;
    return 0;
}

}  // extern "C"
