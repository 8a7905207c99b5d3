// Batched SVD of many independent matrices of uneven sizes (jsvd_dgesvj_batched).
//
// Every matrix runs the same block-oriented method as the single-matrix path
// (Sec. 2, 4 of the paper) with its own block width b_i, pivot table of order
// n_b,i and convergence test (Sec. 4.5).  The matrices progress in lock-step
// p-steps: launch (class, step s, kind) covers the work units of every matrix
// of that block-width class that has a p-step s and is still active, so the
// whole GPU is shared by all matrices at all times.  A unit is a (matrix,
// pair, row chunk) for the Gram and update kernels and a (matrix, pair) for
// the Jacobi kernel; a CTA finds its unit by binary search in a per-launch
// table of (matrix, first unit) built once on the host.
//
// The whole solve is ONE graph launch: an init node, a conditional WHILE
// node whose body is one block sweep of all active matrices (its last kernel
// retires converged matrices and sets the loop condition), then the column
// norms, an on-device per-matrix stable sort and the output assembly.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "driver.h"
#include "jsvd.h"
#include "jsvd_internal.h"
#include "split_kernels.cuh"
#include "sweep_device.cuh"

using namespace jsvd;

namespace {

constexpr int kRowPad = 32;       // rows of G and V are padded to multiples of 32 (zero rows)
constexpr int kRing = 4;          // V' slots: the V update of step s may lag the main branch by 3 steps
constexpr int kMaxSortCols = 1024;

struct BMat {
    int m, n, nb, b, n_pad, k, m_b, g_rows, v_rows, g_chunks, npairs, ug, uv;
    int gc_s, ug_s, uv_s;      // split contractions: Gram partials (256 rows), update units (512 rows)
    int tab_off, vflag_off;
    long long g_off, v_off, part_off, vp_off, col_off;
    long long bsl_off, bex_off, dex_off;   // split right factors of the matrix's pairs (per ring slot)
    long long a_off, s_off, u_off, vo_off;
};

struct BUnit {
    int mat;
    int start;
};

struct BStat {
    int sweeps, converged, active, pad;
    long long rot, proper, updated, brk;
    double off;
};

struct LaunchList {
    int offset;   // into the unit-list buffer
    int count;    // entries
    int units;    // CTAs
};

__device__ __forceinline__ int find_unit(const BUnit *list, int count, int x) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (list[mid].start <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct BArgs {
    const BMat *mats;
    const BUnit *units;
    double *G, *V, *part, *vprime;
    int *vflag;
    const int *tables;
    const unsigned char *inner;   // inner table of this class
    unsigned long long *counters; // kCntSize per matrix
    BStat *stats;
    int inner_sweeps;
    int split;                    // tensor-core contractions (split_kernels.cuh)
    uint16_t *bsl;                // split right factors of this ring slot
    int *bexp, *dexp;
    int *gexp;                    // column exponent bounds, indexed by col_off + column
};

template <int BB>
__global__ void __launch_bounds__(Cfg<BB>::kGramThreads) kb_gram(BArgs a, int off, int count, int step) {
    extern __shared__ __align__(16) double smem[];
    const BUnit u = a.units[off + find_unit(a.units + off, count, blockIdx.x)];
    const BMat M = a.mats[u.mat];
    if (!a.stats[u.mat].active) return;
    const int local = blockIdx.x - u.start;
    const int pair = local / M.g_chunks, chunk = local % M.g_chunks;
    const int P = a.tables[M.tab_off + 2 * (step * M.npairs + pair)];
    const int Q = a.tables[M.tab_off + 2 * (step * M.npairs + pair) + 1];
    const int r0 = chunk * kGramRows;
    const int valid = min(kGramRows, M.g_rows - r0);
    gram_unit<BB, double>(a.G + M.g_off, M.g_rows, r0, valid, P, Q, M.b,
                          a.part + M.part_off + ((size_t)pair * M.g_chunks + chunk) * Cfg<BB>::kPacked, smem);
}

// NT = 2 kJacThreads (one inner sweep): V' rotated by a second thread group.
template <int BB, int NT>
__global__ void __launch_bounds__(NT) kb_jacobi(BArgs a, int off, int count, int step) {
    extern __shared__ __align__(16) double smem[];
    const BUnit u = a.units[off + find_unit(a.units + off, count, blockIdx.x)];
    const BMat M = a.mats[u.mat];
    if (!a.stats[u.mat].active) return;
    const int pair = blockIdx.x - u.start;
    const int P = a.tables[M.tab_off + 2 * (step * M.npairs + pair)];
    const int Q = a.tables[M.tab_off + 2 * (step * M.npairs + pair) + 1];
    const int chunks = a.split ? M.gc_s : M.g_chunks;
    jacobi_unit<BB, NT>(a.part + M.part_off + (size_t)pair * chunks * Cfg<BB>::kPacked, chunks, a.inner, P,
                    Q, M.b, M.n_pad, M.n, M.n_pad, a.inner_sweeps, kEps, a.vprime + M.vp_off + (size_t)pair * BB * BB,
                    a.vflag + M.vflag_off + pair, a.counters + (size_t)u.mat * kCntSize, smem,
                    a.split ? a.bsl + M.bsl_off + (size_t)pair * 2 * split_b_elems<BB>() : nullptr,
                    a.split ? a.bexp + M.bex_off + (size_t)pair * 2 * BB : nullptr,
                    a.split ? a.dexp + M.dex_off + (size_t)pair * BB : nullptr,
                    a.split ? a.gexp + M.col_off : nullptr);
}

// which = 0: rows of G, which = 1: rows of V
template <int BB>
__global__ void __launch_bounds__(kUpdThreads) kb_update(BArgs a, int off, int count, int step, int which) {
    constexpr int RU = Cfg<BB>::kUpdRows;
    extern __shared__ __align__(16) double smem[];
    const BUnit u = a.units[off + find_unit(a.units + off, count, blockIdx.x)];
    const BMat M = a.mats[u.mat];
    if (!a.stats[u.mat].active) return;
    const int local = blockIdx.x - u.start;
    const int per = which ? M.uv : M.ug;
    const int pair = local / per, c = local % per;
    if (!a.vflag[M.vflag_off + pair]) return;
    const int P = a.tables[M.tab_off + 2 * (step * M.npairs + pair)];
    const int Q = a.tables[M.tab_off + 2 * (step * M.npairs + pair) + 1];
    double *X;
    int ld, r0, valid;
    if (!which) {
        X = a.G + M.g_off; ld = M.g_rows; r0 = c * RU; valid = min(RU, M.g_rows - r0);
    } else {
        X = a.V + M.v_off; ld = M.v_rows; r0 = c * RU; valid = min(RU, M.v_rows - r0);
    }
    update_unit<BB, double>(X, ld, r0, valid, P, Q, M.b, a.vprime + M.vp_off + (size_t)pair * BB * BB, smem);
}

// Split-contraction Gram: unit = (matrix, pair, 256-row partial).
template <int BB>
__global__ void __launch_bounds__(SplitCfg<BB>::kGThreads, 1) kb_gram_split(BArgs a, int off, int count, int step) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const BUnit u = a.units[off + find_unit(a.units + off, count, blockIdx.x)];
    const BMat M = a.mats[u.mat];
    if (!a.stats[u.mat].active) return;
    const int local = blockIdx.x - u.start;
    const int pair = local / M.gc_s, chunk = local % M.gc_s;
    const int P = a.tables[M.tab_off + 2 * (step * M.npairs + pair)];
    const int Q = a.tables[M.tab_off + 2 * (step * M.npairs + pair) + 1];
    const int r0 = chunk * kGramRowsSplit;
    gram_split_body<BB>(a.G + M.g_off, M.g_rows, P, Q, M.b, a.gexp + M.col_off, (size_t)r0,
                        min(kGramRowsSplit, M.g_rows - r0),
                        a.part + M.part_off + (size_t)pair * M.gc_s * Cfg<BB>::kPacked, chunk, smem_raw);
}

// Split-contraction update, which = 0: rows of G, which = 1: rows of V;
// unit = (matrix, pair, kUpdRowsPerCta rows).
template <int BB>
__global__ void __launch_bounds__(32 * SplitCfg<BB>::kUpdWarps) kb_update_split(BArgs a, int off, int count, int step,
                                                                              int which) {
    using S = SplitCfg<BB>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const BUnit u = a.units[off + find_unit(a.units + off, count, blockIdx.x)];
    const BMat M = a.mats[u.mat];
    if (!a.stats[u.mat].active) return;
    const int local = blockIdx.x - u.start;
    const int per = which ? M.uv_s : M.ug_s;
    const int pair = local / per, c = local % per;
    if (!a.vflag[M.vflag_off + pair]) return;
    const int P = a.tables[M.tab_off + 2 * (step * M.npairs + pair)];
    const int Q = a.tables[M.tab_off + 2 * (step * M.npairs + pair) + 1];
    double *X = which ? a.V + M.v_off : a.G + M.g_off;
    const int ld = which ? M.v_rows : M.g_rows;
    const int r0 = c * S::kUpdRowsPerCta;
    update_split_body<BB, true>(X, ld, (size_t)r0, min(S::kUpdRowsPerCta, ld - r0), P, Q, M.b,
                          a.bsl + M.bsl_off + ((size_t)pair * 2 + which) * split_b_elems<BB>(),
                          a.bexp + M.bex_off + ((size_t)pair * 2 + which) * BB,
                          which ? nullptr : a.dexp + M.dex_off + (size_t)pair * BB,
                          which ? nullptr : a.gexp + M.col_off, smem_raw);
}

// Exponent bounds of every column of every matrix's G (one warp per column).
__global__ void kb_col_maxexp(const BMat *mats, int batch, const long long *col_start, long long total_cols,
                              const double *G, int *gexp) {
    const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (w >= total_cols) return;
    int lo = 0, hi = batch - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (col_start[mid] <= w) lo = mid;
        else hi = mid - 1;
    }
    const BMat M = mats[lo];
    const int c = (int)(w - col_start[lo]);
    const double *g = G + M.g_off + (size_t)c * M.g_rows;
    int e = split::kNoExp;
    for (int r = lane; r < M.g_rows; r += 32) e = max(e, split::exp_bound(g[r], 0));
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if (lane == 0) gexp[w] = e;
}

// Bordered copy of every A_i into its G_i, V_i = I, all matrices active.
__global__ void kb_init(const BMat *mats, int batch, const double *__restrict__ A, double *G, double *V,
                        BStat *stats, unsigned long long *counters, unsigned long long *err) {
    const int i = blockIdx.y;
    if (i >= batch) return;
    const BMat M = mats[i];
    const size_t gtot = (size_t)M.g_rows * M.n_pad, vtot = (size_t)M.v_rows * M.n_pad;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < gtot + vtot;
         e += (size_t)gridDim.x * blockDim.x) {
        if (e < gtot) {
            const int r = (int)(e % M.g_rows), c = (int)(e / M.g_rows);
            double v = 0.0;
            if (c >= M.n) {
                v = (r == M.m + (c - M.n)) ? 1.0 : 0.0;
            } else if (r < M.m) {
                v = A[M.a_off + (size_t)c * M.m + r];
                if (!isfinite(v)) atomicOr(err, 1ull);
            }
            G[M.g_off + (size_t)c * M.g_rows + r] = v;
        } else {
            const size_t f = e - gtot;
            const int r = (int)(f % M.v_rows), c = (int)(f / M.v_rows);
            V[M.v_off + (size_t)c * M.v_rows + r] = (r == c) ? 1.0 : 0.0;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        BStat s{};
        s.active = 1;
        stats[i] = s;
    }
    if (blockIdx.x == 0 && threadIdx.x < kCntSize) counters[(size_t)i * kCntSize + threadIdx.x] = 0ull;
}

// End of a block sweep: fold the counters into the statistics, retire the
// matrices whose sweep had no proper rotation, and keep looping while any
// matrix is active and the sweep limit has not been reached.
__global__ void kb_sweep_end(int batch, BStat *stats, unsigned long long *counters, int *sweep_no,
                             int max_sweeps, cudaGraphConditionalHandle handle) {
    __shared__ int s_active;
    if (threadIdx.x == 0) s_active = 0;
    __syncthreads();
    const int sw = *sweep_no + 1;
    for (int i = threadIdx.x; i < batch; i += blockDim.x) {
        BStat s = stats[i];
        if (s.active) {
            unsigned long long *c = counters + (size_t)i * kCntSize;
            s.sweeps += 1;
            s.rot += (long long)c[kCntRot];
            s.proper += (long long)c[kCntProper];
            s.updated += (long long)c[kCntUpdated];
            s.brk += (long long)c[kCntBreak];
            s.off = __longlong_as_double((long long)c[kCntOff]);
            if (c[kCntProper] == 0) {
                s.converged = 1;
                s.active = 0;
            }
            for (int k = 0; k < kCntSize; ++k) c[k] = 0ull;
            stats[i] = s;
            if (s.active) atomicAdd(&s_active, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *sweep_no = sw;
        cudaGraphSetConditional(handle, (s_active > 0 && sw < max_sweeps) ? 1u : 0u);
    }
}

// sigma of every column of every matrix (one warp per column); columns with
// support in the border rows are marked.
__global__ void kb_colnorms(const BMat *mats, int batch, const long long *col_start, long long total_cols,
                            const double *G, double *sigma, int *border) {
    const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (w >= total_cols) return;
    int lo = 0, hi = batch - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (col_start[mid] <= w) lo = mid;
        else hi = mid - 1;
    }
    const BMat M = mats[lo];
    const int c = (int)(w - col_start[lo]);
    const double *g = G + M.g_off + (size_t)c * M.g_rows;
    double s = 0.0;
    int bd = 0;
    for (int r = lane; r < M.m_b; r += 32) {
        const double x = g[r];
        s = __fma_rn(x, x, s);
        if (r >= M.m && x != 0.0) bd = 1;
    }
    for (int off = 16; off > 0; off >>= 1) s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, off));
    bd = __any_sync(0xffffffffu, bd);
    if (lane == 0) {
        sigma[w] = __dsqrt_rn(s);
        border[w] = bd;
    }
}

// Per matrix: stable order of the non-border columns by sigma, descending
// (bitonic sort of (sigma, index) keys; the border columns, which keep their
// positions n..n_pad-1, go last).
__global__ void __launch_bounds__(512) kb_sort(const BMat *mats, const long long *col_start, const double *sigma,
                                               const int *border, int *perm, int sort) {
    __shared__ double key[kMaxSortCols];
    __shared__ int idx[kMaxSortCols];
    const BMat M = mats[blockIdx.x];
    const long long c0 = col_start[blockIdx.x];
    for (int t = threadIdx.x; t < kMaxSortCols; t += blockDim.x) {
        double kv = -2.0;   // padding after everything
        if (t < M.n_pad) kv = (t >= M.n) ? -1.0 : (sort ? sigma[c0 + t] : 0.0);
        key[t] = kv;
        idx[t] = t;
    }
    __syncthreads();
    // descending by key, ascending by index on ties
    for (int size = 2; size <= kMaxSortCols; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < kMaxSortCols / 2; t += blockDim.x) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool up = ((lo & size) == 0);
                const bool hi_first = key[hi] > key[lo] || (key[hi] == key[lo] && idx[hi] < idx[lo]);
                if (hi_first == up) {
                    const double tk = key[lo]; key[lo] = key[hi]; key[hi] = tk;
                    const int ti = idx[lo]; idx[lo] = idx[hi]; idx[hi] = ti;
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < M.n; t += blockDim.x) perm[c0 + t] = idx[t];
}

// Output assembly: column i of matrix j takes workspace column perm[i].
__global__ void kb_finalize(const BMat *mats, int batch, const long long *col_start, const long long *out_start,
                            long long total_out, const double *G, const double *V, const double *sigma,
                            const int *perm, double *S, double *U, double *Vo) {
    const long long w = blockIdx.x;
    if (w >= total_out) return;
    int lo = 0, hi = batch - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (out_start[mid] <= w) lo = mid;
        else hi = mid - 1;
    }
    const BMat M = mats[lo];
    const int i = (int)(w - out_start[lo]);
    const int c = perm[col_start[lo] + i];
    const double sg = sigma[col_start[lo] + c];
    if (threadIdx.x == 0) S[M.s_off + i] = sg;
    const double *g = G + M.g_off + (size_t)c * M.g_rows;
    for (int r = threadIdx.x; r < M.m; r += blockDim.x)
        U[M.u_off + (size_t)i * M.m + r] = sg > 0.0 ? __ddiv_rn(g[r], sg) : 0.0;
    if (Vo) {
        const double *v = V + M.v_off + (size_t)c * M.v_rows;
        for (int r = threadIdx.x; r < M.n; r += blockDim.x) Vo[M.vo_off + (size_t)i * M.n + r] = v[r];
    }
}

// A kernel launch with an explicit scheduling priority (kept by graph capture).
template <typename... KArgs, typename... Args>
void launch_prio(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st, int prio,
                 Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = prio;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Default block width by size when neither the caller nor opts->b sets one.
int pick_b(int n) { return n <= 256 ? 8 : 16; }

}  // namespace

// ---------------------------------------------------------------------------

int jsvd_ctx::solve_batched(int batch, const int *m, const int *n, const int *bs, const double *A,
                            const long long *a_off, double *S, const long long *s_off, double *U,
                            const long long *u_off, double *Vo, const long long *v_off, const jsvd_opts *opts_in,
                            jsvd_info *infos) {
    jsvd_opts o;
    jsvd_default_opts(&o);
    if (opts_in) o = *opts_in;
    if (o.max_sweeps <= 0) o.max_sweeps = 30;
    if (o.inner_sweeps <= 0) o.inner_sweeps = 1;
    if (o.inner_strategy < 0) o.inner_strategy = o.strategy;
    if (o.precision != JSVD_PREC_FP64) {
        last_error = "the batched solver runs in FP64 only";
        return JSVD_ERR_UNSUPPORTED;
    }
    int rc;
    // the batched solver's split contractions are the mma.sync forms for both
    // split modes
    const bool split = o.contraction == JSVD_CONTRACT_SPLIT || o.contraction == JSVD_CONTRACT_SPLIT_SYNC;
    // ---- per-matrix layout ---------------------------------------------------
    std::vector<BMat> mats(batch);
    std::vector<int> tables;
    std::vector<std::pair<int, int>> tab_keys;  // (nb, offset)
    long long g_tot = 0, v_tot = 0, p_tot = 0, vp_tot = 0, col_tot = 0, out_tot = 0;
    long long bsl_tot = 0, bex_tot = 0, dex_tot = 0;
    int vf_tot = 0;
    std::vector<long long> col_start(batch), out_start(batch);
    for (int i = 0; i < batch; ++i) {
        BMat &M = mats[i];
        M.m = m[i];
        M.n = n[i];
        M.b = (bs && bs[i] > 0) ? bs[i] : (o.b ? o.b : pick_b(M.n));
        if (M.b != 8 && M.b != 16 && M.b != 32) {
            last_error = "batched block width must be 8, 16 or 32";
            return JSVD_ERR_UNSUPPORTED;
        }
        int nb = (M.n + M.b - 1) / M.b;
        M.nb = admissible_order(o.strategy, nb < 2 ? 2 : nb);
        M.n_pad = M.nb * M.b;
        if (M.n_pad > kMaxSortCols) {
            last_error = "batched matrices must have n <= 1024 after bordering";
            return JSVD_ERR_UNSUPPORTED;
        }
        M.k = M.n_pad - M.n;
        M.m_b = M.m + M.k;
        M.g_rows = (M.m_b + kRowPad - 1) / kRowPad * kRowPad;
        M.v_rows = (M.n_pad + kRowPad - 1) / kRowPad * kRowPad;
        M.g_chunks = (M.g_rows + kGramRows - 1) / kGramRows;
        M.npairs = M.nb / 2;
        const int BB = 2 * M.b, RU = 4096 / BB;
        M.ug = (M.g_rows + RU - 1) / RU;
        M.uv = (M.v_rows + RU - 1) / RU;
        M.gc_s = (M.g_rows + kGramRowsSplit - 1) / kGramRowsSplit;
        M.ug_s = (M.g_rows + SplitCfg<64>::kUpdRowsPerCta - 1) / SplitCfg<64>::kUpdRowsPerCta;
        M.uv_s = (M.v_rows + SplitCfg<64>::kUpdRowsPerCta - 1) / SplitCfg<64>::kUpdRowsPerCta;
        const long long belems = BB == 16 ? split_b_elems<16>() : BB == 32 ? split_b_elems<32>() : split_b_elems<64>();
        M.bsl_off = bsl_tot; bsl_tot += (long long)M.npairs * 2 * belems;
        M.bex_off = bex_tot; bex_tot += (long long)M.npairs * 2 * BB;
        M.dex_off = dex_tot; dex_tot += (long long)M.npairs * BB;
        int toff = -1;
        for (auto &kv : tab_keys)
            if (kv.first == M.nb) toff = kv.second;
        if (toff < 0) {
            std::vector<int> t;
            if (build_pstrategy(o.strategy, M.nb, t)) {
                last_error = "no pivot table for a batched matrix";
                return JSVD_ERR_UNSUPPORTED;
            }
            toff = (int)tables.size();
            tables.insert(tables.end(), t.begin(), t.end());
            tab_keys.emplace_back(M.nb, toff);
        }
        M.tab_off = toff;
        M.g_off = g_tot; g_tot += (long long)M.g_rows * M.n_pad;
        M.v_off = v_tot; v_tot += (long long)M.v_rows * M.n_pad;
        M.part_off = p_tot; p_tot += (long long)M.npairs * M.g_chunks * (BB * (BB + 1) / 2);
        M.vp_off = vp_tot; vp_tot += (long long)M.npairs * BB * BB;
        M.vflag_off = vf_tot; vf_tot += M.npairs;
        col_start[i] = col_tot; M.col_off = col_tot; col_tot += M.n_pad;
        out_start[i] = out_tot; out_tot += M.n;
        M.a_off = a_off[i];
        M.s_off = s_off[i];
        M.u_off = u_off[i];
        M.vo_off = v_off ? v_off[i] : 0;
    }
    // ---- launch lists per (class, step, kind) --------------------------------
    struct Planned { int BB, step, kind; LaunchList l; };
    std::vector<Planned> plan;
    std::vector<BUnit> units;
    for (int BB : {16, 32, 64}) {
        int max_steps = 0;
        for (auto &M : mats)
            if (2 * M.b == BB) max_steps = std::max(max_steps, M.nb - 1);
        for (int s = 0; s < max_steps; ++s) {
            for (int kind = 0; kind < 4; ++kind) {   // Gram, Jacobi, update of G, update of V
                if (kind == 3 && !Vo) continue;
                LaunchList l{(int)units.size(), 0, 0};
                for (int i = 0; i < batch; ++i) {
                    const BMat &M = mats[i];
                    if (2 * M.b != BB || s >= M.nb - 1) continue;
                    const int cnt = kind == 0 ? M.npairs * (split ? M.gc_s : M.g_chunks)
                                  : kind == 1 ? M.npairs
                                  : kind == 2 ? M.npairs * (split ? M.ug_s : M.ug)
                                              : M.npairs * (split ? M.uv_s : M.uv);
                    units.push_back(BUnit{i, l.units});
                    l.units += cnt;
                    ++l.count;
                }
                if (l.count) plan.push_back(Planned{BB, s, kind, l});
            }
        }
    }
    // ---- device buffers --------------------------------------------------------
    const size_t need[] = {
        sizeof(BMat) * batch, sizeof(BUnit) * std::max<size_t>(units.size(), 1),
        sizeof(double) * g_tot, sizeof(double) * v_tot, sizeof(double) * std::max<long long>(p_tot, 1),
        sizeof(double) * std::max<long long>(vp_tot, 1) * kRing, sizeof(int) * std::max(vf_tot, 1) * kRing,
        sizeof(int) * tables.size(), sizeof(unsigned long long) * kCntSize * batch, sizeof(BStat) * batch,
        sizeof(long long) * batch * 2, sizeof(double) * col_tot, sizeof(int) * col_tot, sizeof(int) * col_tot,
        sizeof(int) * 4,
        split ? sizeof(uint16_t) * bsl_tot * kRing : 16, split ? sizeof(int) * bex_tot * kRing : 16,
        split ? sizeof(int) * dex_tot * kRing : 16, split ? sizeof(int) * col_tot : 16};
    Buffer *bufs[] = {&b_mats, &b_units, &b_g, &b_v, &b_part, &b_vp, &b_vflag, &b_tab, &b_cnt, &b_stat,
                      &b_starts, &b_sigma, &b_border, &b_perm, &b_misc, &b_bsl, &b_bex, &b_dex, &b_gexp};
    for (size_t j = 0; j < sizeof(bufs) / sizeof(bufs[0]); ++j)
        if ((rc = ensure(*bufs[j], need[j]))) return rc;
    const unsigned char *dinner[3] = {nullptr, nullptr, nullptr};
    for (int c = 0; c < 3; ++c) {
        const int BB = 16 << c;
        bool used = false;
        for (auto &M : mats) used |= (2 * M.b == BB);
        if (used && (rc = inner_table(o.inner_strategy, BB, &dinner[c]))) return rc;
    }
    BMat *dm = (BMat *)b_mats.ptr;
    BUnit *du = (BUnit *)b_units.ptr;
    long long *dstarts = (long long *)b_starts.ptr;
    int *dmisc = (int *)b_misc.ptr;
    std::vector<long long> starts(col_start);
    starts.insert(starts.end(), out_start.begin(), out_start.end());
    cudaMemcpyAsync(dm, mats.data(), sizeof(BMat) * batch, cudaMemcpyHostToDevice, stream);
    if (!units.empty()) cudaMemcpyAsync(du, units.data(), sizeof(BUnit) * units.size(), cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(b_tab.ptr, tables.data(), sizeof(int) * tables.size(), cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(dstarts, starts.data(), sizeof(long long) * 2 * batch, cudaMemcpyHostToDevice, stream);
    cudaMemsetAsync(dmisc, 0, sizeof(int) * 4, stream);
    if ((rc = sync("batched setup"))) return rc;

    BArgs ba{};
    ba.mats = dm;
    ba.units = du;
    ba.G = (double *)b_g.ptr;
    ba.V = (double *)b_v.ptr;
    ba.part = (double *)b_part.ptr;
    ba.vprime = (double *)b_vp.ptr;
    ba.vflag = (int *)b_vflag.ptr;
    ba.tables = (const int *)b_tab.ptr;
    ba.counters = (unsigned long long *)b_cnt.ptr;
    ba.stats = (BStat *)b_stat.ptr;
    ba.inner_sweeps = o.inner_sweeps;
    ba.split = split ? 1 : 0;
    ba.bsl = (uint16_t *)b_bsl.ptr;
    ba.bexp = (int *)b_bex.ptr;
    ba.dexp = (int *)b_dex.ptr;
    ba.gexp = (int *)b_gexp.ptr;

    cudaFuncSetAttribute(kb_gram<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_smem_bytes<16, double>());
    cudaFuncSetAttribute(kb_gram<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_smem_bytes<32, double>());
    cudaFuncSetAttribute(kb_gram<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_smem_bytes<64, double>());
#define JSVD_JAC_ATTR(BBV)                                                                              \
    cudaFuncSetAttribute(kb_jacobi<BBV, Cfg<BBV>::kJacThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                         (int)jacobi_smem_bytes<BBV>());                                                 \
    cudaFuncSetAttribute(kb_jacobi<BBV, 2 * Cfg<BBV>::kJacThreads>,                                      \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jacobi_smem_bytes<BBV>());
    JSVD_JAC_ATTR(16)
    JSVD_JAC_ATTR(32)
    JSVD_JAC_ATTR(64)
#undef JSVD_JAC_ATTR
#define JSVD_SPLIT_ATTR(BBV)                                                                            \
    cudaFuncSetAttribute(kb_gram_split<BBV>, cudaFuncAttributeMaxDynamicSharedMemorySize,              \
                         (int)gram_split_smem<BBV>());                                                   \
    cudaFuncSetAttribute(kb_update_split<BBV>, cudaFuncAttributeMaxDynamicSharedMemorySize,            \
                         (int)update_split_smem<BBV>());
    JSVD_SPLIT_ATTR(16)
    JSVD_SPLIT_ATTR(32)
    JSVD_SPLIT_ATTR(64)
#undef JSVD_SPLIT_ATTR
    cudaFuncSetAttribute(kb_update<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)update_smem_bytes<16, double>());
    cudaFuncSetAttribute(kb_update<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)update_smem_bytes<32, double>());
    cudaFuncSetAttribute(kb_update<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)update_smem_bytes<64, double>());

    // ---- graph: init -> while(sweep) -> finalize ----------------------------------
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return check("stream");
    int prio_least = 0, prio_greatest = 0;
    cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    cudaStream_t ms[3], vs[3];
    for (int c = 0; c < 3; ++c) {
        cudaStreamCreateWithPriority(&ms[c], cudaStreamNonBlocking, prio_greatest);
        cudaStreamCreateWithPriority(&vs[c], cudaStreamNonBlocking, prio_least);
    }
    std::vector<cudaEvent_t> gev(1 + 2 * 3 * kRing + 6);
    for (auto &e : gev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    cudaGraph_t graph = nullptr, g_init = nullptr, g_fin = nullptr;
    cudaGraphExec_t exec = nullptr;
    int status = 0;
    auto fail = [&](const char *where) {
        cudaError_t e = cudaGetLastError();
        set_error(where, e == cudaSuccess ? cudaErrorUnknown : e);
        status = JSVD_ERR_CUDA;
    };
    do {
        if (cudaGraphCreate(&graph, 0) != cudaSuccess) { fail("graph create"); break; }
        // init
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { fail("capture"); break; }
        kb_init<<<dim3(64, batch), 256, 0, cs>>>(dm, batch, A, ba.G, ba.V, ba.stats, ba.counters,
                                                 (unsigned long long *)(dmisc + 2));
        if (split)
            kb_col_maxexp<<<(unsigned)((col_tot * 32 + 255) / 256), 256, 0, cs>>>(dm, batch, dstarts, col_tot, ba.G,
                                                                                 ba.gexp);
        if (cudaStreamEndCapture(cs, &g_init) != cudaSuccess) { fail("capture init"); break; }
        cudaGraphNode_t n_init, n_while, n_fin;
        if (cudaGraphAddChildGraphNode(&n_init, graph, nullptr, 0, g_init) != cudaSuccess) { fail("child init"); break; }
        cudaGraphConditionalHandle handle;
        if (cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
            fail("conditional handle");
            break;
        }
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        if (cudaGraphAddNode(&n_while, graph, &n_init, nullptr, 1, &cp) != cudaSuccess) { fail("while node"); break; }
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
            cudaSuccess) { fail("capture body"); break; }
        // One branch per block-width class; inside it the V updates run on a
        // low-priority branch that trails the main one through a ring of V' slots.
        cudaEventRecord(gev[0], cs);
        for (int c = 0; c < 3; ++c) {
            cudaStreamWaitEvent(ms[c], gev[0], 0);
            cudaStreamWaitEvent(vs[c], gev[0], 0);
        }
        for (const Planned &p : plan) {
            const int c = p.BB == 16 ? 0 : p.BB == 32 ? 1 : 2;
            const int slot = p.step % kRing;
            BArgs a = ba;
            a.inner = dinner[c];
            a.vprime = ba.vprime + (size_t)slot * vp_tot;
            a.vflag = ba.vflag + (size_t)slot * vf_tot;
            a.bsl = ba.bsl + (size_t)slot * bsl_tot;
            a.bexp = ba.bexp + (size_t)slot * bex_tot;
            a.dexp = ba.dexp + (size_t)slot * dex_tot;
            const int off = p.l.offset, cnt = p.l.count, units_n = p.l.units;
            if (units_n <= 0) continue;
            cudaEvent_t *jac_done = &gev[1 + (c * kRing + slot) * 2];
            cudaEvent_t *v_done = jac_done + 1;
            if (p.kind == 0 && p.step >= kRing && Vo) cudaStreamWaitEvent(ms[c], *v_done, 0);
            // split contractions update V on the main branch (their update CTAs
            // slow the latency-bound Jacobi kernel when they run beside it)
            const bool vside = p.kind == 3 && !split;
            if (vside) cudaStreamWaitEvent(vs[c], *jac_done, 0);
            cudaStream_t st = vside ? vs[c] : ms[c];
            const int prio = vside ? prio_least : prio_greatest;
#define JSVD_LAUNCH_B(BBV)                                                                              \
    if (p.BB == BBV) {                                                                                  \
        if (p.kind == 0 && split)                                                                       \
            launch_prio(kb_gram_split<BBV>, units_n, SplitCfg<BBV>::kGThreads, gram_split_smem<BBV>(), st, \
                        prio, a, off, cnt, p.step);                                                     \
        else if (p.kind == 0)                                                                           \
            launch_prio(kb_gram<BBV>, units_n, Cfg<BBV>::kGramThreads, gram_smem_bytes<BBV, double>(), st, \
                        prio, a, off, cnt, p.step);                                                     \
        else if (p.kind == 1 && ba.inner_sweeps == 1)                                                   \
            launch_prio(kb_jacobi<BBV, 2 * Cfg<BBV>::kJacThreads>, units_n, 2 * Cfg<BBV>::kJacThreads,  \
                        jacobi_smem_bytes<BBV>(), st, prio, a, off, cnt, p.step);                       \
        else if (p.kind == 1)                                                                           \
            launch_prio(kb_jacobi<BBV, Cfg<BBV>::kJacThreads>, units_n, Cfg<BBV>::kJacThreads,          \
                        jacobi_smem_bytes<BBV>(), st, prio, a, off, cnt, p.step);                       \
        else if (split)                                                                                 \
            launch_prio(kb_update_split<BBV>, units_n, 32 * SplitCfg<BBV>::kUpdWarps,                   \
                        update_split_smem<BBV>(), st, prio, a, off, cnt, p.step, p.kind - 2);           \
        else                                                                                            \
            launch_prio(kb_update<BBV>, units_n, kUpdThreads, update_smem_bytes<BBV, double>(), st,     \
                        prio, a, off, cnt, p.step, p.kind - 2);                                         \
    }
            JSVD_LAUNCH_B(16)
            JSVD_LAUNCH_B(32)
            JSVD_LAUNCH_B(64)
#undef JSVD_LAUNCH_B
            if (p.kind == 1) cudaEventRecord(*jac_done, ms[c]);
            if (p.kind == 3) cudaEventRecord(*v_done, vside ? vs[c] : ms[c]);
        }
        for (int c = 0; c < 3; ++c) {
            cudaEventRecord(gev[1 + 2 * 3 * kRing + 2 * c], ms[c]);
            cudaEventRecord(gev[2 + 2 * 3 * kRing + 2 * c], vs[c]);
            cudaStreamWaitEvent(cs, gev[1 + 2 * 3 * kRing + 2 * c], 0);
            cudaStreamWaitEvent(cs, gev[2 + 2 * 3 * kRing + 2 * c], 0);
        }
        kb_sweep_end<<<1, 1024, 0, cs>>>(batch, ba.stats, ba.counters, dmisc, o.max_sweeps, handle);
        if (cudaStreamEndCapture(cs, &body) != cudaSuccess) { fail("capture body end"); break; }
        // finalize
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { fail("capture fin"); break; }
        kb_colnorms<<<(unsigned)((col_tot * 32 + 255) / 256), 256, 0, cs>>>(dm, batch, dstarts, col_tot, ba.G,
                                                                            (double *)b_sigma.ptr, (int *)b_border.ptr);
        kb_sort<<<batch, 512, 0, cs>>>(dm, dstarts, (double *)b_sigma.ptr, (int *)b_border.ptr, (int *)b_perm.ptr,
                                       o.sort);
        kb_finalize<<<(unsigned)out_tot, 128, 0, cs>>>(dm, batch, dstarts, dstarts + batch, out_tot, ba.G, ba.V,
                                                       (double *)b_sigma.ptr, (int *)b_perm.ptr, S, U, Vo);
        if (cudaStreamEndCapture(cs, &g_fin) != cudaSuccess) { fail("capture fin end"); break; }
        if (cudaGraphAddChildGraphNode(&n_fin, graph, &n_while, 1, g_fin) != cudaSuccess) { fail("child fin"); break; }
        if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) { fail("instantiate"); break; }
        // order after the caller's prior work on the context stream
        cudaEvent_t ev;
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        cudaEventRecord(ev, stream);
        cudaStreamWaitEvent(cs, ev, 0);
        if (profiling) {
            ensure_events(2);
            cudaEventRecord(events[0], cs);
        }
        if (cudaGraphLaunch(exec, cs) != cudaSuccess) { fail("graph launch"); cudaEventDestroy(ev); break; }
        if (profiling) cudaEventRecord(events[1], cs);
        cudaEventRecord(ev, cs);
        cudaStreamWaitEvent(stream, ev, 0);
        cudaEventDestroy(ev);
        if (cudaStreamSynchronize(cs) != cudaSuccess) { fail("batched run"); break; }
        if (profiling) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, events[0], events[1]);
            prof_ms[4] += ms;
        }
    } while (0);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (g_init) cudaGraphDestroy(g_init);
    if (g_fin) cudaGraphDestroy(g_fin);
    cudaStreamDestroy(cs);
    for (int c = 0; c < 3; ++c) {
        cudaStreamDestroy(ms[c]);
        cudaStreamDestroy(vs[c]);
    }
    for (auto &e : gev) cudaEventDestroy(e);
    if (status) return status;

    // ---- statistics ------------------------------------------------------------
    std::vector<BStat> st(batch);
    int misc[4];
    cudaMemcpy(st.data(), ba.stats, sizeof(BStat) * batch, cudaMemcpyDeviceToHost);
    cudaMemcpy(misc, dmisc, sizeof(int) * 4, cudaMemcpyDeviceToHost);
    if ((rc = check("batched stats"))) return rc;
    if (misc[2] || misc[3]) {
        last_error = "input holds Inf or NaN";
        return JSVD_ERR_NONFINITE;
    }
    int all_conv = 1;
    prof_launches[4] += 3 + (long long)misc[0] * ((long long)plan.size() + 1);
    for (int i = 0; i < batch; ++i) {
        const int BB = 2 * mats[i].b;
        const double bbd = BB;
        prof_flops[4] += (double)st[i].sweeps * (mats[i].nb - 1) * mats[i].npairs *
                             ((double)mats[i].m * bbd * (bbd + 1.0) + 9.0 * bbd * bbd * (bbd - 1.0) + bbd * bbd * bbd / 3.0) +
                         (double)st[i].updated * 2.0 * ((double)mats[i].m + (Vo ? (double)mats[i].n : 0.0)) * bbd * bbd;
        all_conv &= st[i].converged;
        if (infos) {
            jsvd_info &f = infos[i];
            memset(&f, 0, sizeof f);
            f.sweeps = st[i].sweeps;
            f.converged = st[i].converged;
            f.b = mats[i].b;
            f.rotations = st[i].rot;
            f.proper_rotations = st[i].proper;
            f.pairs_updated = st[i].updated;
            f.breakdowns = st[i].brk;
            f.off_norm = st[i].off;
        }
    }
    return all_conv ? JSVD_SUCCESS : JSVD_NOT_CONVERGED;
}

extern "C" int jsvd_dgesvj_batched(jsvd_ctx_t ctx, int batch, const int *m, const int *n, const int *b,
                                   const double *A, const long long *a_off, double *S, const long long *s_off,
                                   double *U, const long long *u_off, double *V, const long long *v_off,
                                   const jsvd_opts *opts, jsvd_info *infos) {
    if (!ctx) return -1;
    if (batch < 0) return -2;
    if (batch == 0) return 0;
    if (!m) return -3;
    if (!n) return -4;
    for (int i = 0; i < batch; ++i)
        if (m[i] < 1 || n[i] < 1 || m[i] < n[i]) return -3;
    if (!A || !a_off) return -6;
    if (!S || !s_off) return -8;
    if (!U || !u_off) return -10;
    if (V && !v_off) return -13;
    cudaSetDevice(ctx->device);
    if (opts && opts->preprocess)
        return ctx->solve_batched_qr(batch, m, n, b, A, a_off, S, s_off, U, u_off, V, v_off, opts, infos);
    return ctx->solve_batched(batch, m, n, b, A, a_off, S, s_off, U, u_off, V, v_off, opts, infos);
}
