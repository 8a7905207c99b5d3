// Reverse-mode derivative of the SVD (jsvd_dgesvj_backward).
//
// For A = U diag(s) V^T (U m x n with orthonormal columns, V n x n orthogonal,
// distinct positive s) and cotangents dU, ds, dV, the published SVD adjoint is
//   dA = U [ (F o (J - J^T)) S + diag(ds) + S (F o (K - K^T)) ] V^T
//        + (I - U U^T) dU S^{-1} V^T,
//   J = U^T dU,  K = V^T dV,  F_ij = 1 / (s_j^2 - s_i^2) (i != j), F_ii = 0.
// The off-diagonal entry (a s_j + c s_i) / ((s_j - s_i)(s_j + s_i)) with
// a = J_ij - J_ji, c = K_ij - K_ji is evaluated in the split form
//   (a + c) / (2 (s_j - s_i)) + (a - c) / (2 (s_j + s_i)),
// which keeps its accuracy when s_i and s_j are close.  With
//   N = [...] - J S^{-1}   and   X = U N + dU S^{-1},   dA = X V^T.
// All products are FP64 grouped GEMMs over the whole batch (three launches)
// plus two elementwise kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "driver.h"
#include "gemm_fp64.cuh"
#include "jsvd.h"

using namespace jsvd;

namespace {

struct AdjMat {
    int m, n;
    long long u_off, s_off, v_off, a_off;   // caller's packing
    long long j_off, x_off;                 // workspace: J, K, N (n x n each) and X (m x n)
};

// N = (off-diagonal split form) + diag(ds) - J S^{-1}, written over K's slot.
__global__ void k_adj_middle(const AdjMat *mats, int batch, const long long *nn_start, long long total,
                             const double *S, const double *dS, double *W) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = batch - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (nn_start[mid] <= e) lo = mid;
            else hi = mid - 1;
        }
        const AdjMat M = mats[lo];
        const int n = M.n;
        const long long f = e - nn_start[lo];
        const int i = (int)(f % n), j = (int)(f / n);
        double *J = W + M.j_off;
        const double *K = J + (size_t)n * n;
        double *N = J + 2 * (size_t)n * n;
        const double si = S[M.s_off + i], sj = S[M.s_off + j];
        double v;
        if (i == j) {
            v = dS ? dS[M.s_off + i] : 0.0;
        } else {
            const double a = J[i + (size_t)j * n] - J[j + (size_t)i * n];
            const double c = K[i + (size_t)j * n] - K[j + (size_t)i * n];
            v = 0.5 * (a + c) / (sj - si) + 0.5 * (a - c) / (sj + si);
        }
        v -= J[i + (size_t)j * n] / sj;
        N[i + (size_t)j * n] = v;
    }
}

// X = dU S^{-1} (or 0 without dU).
__global__ void k_adj_scale(const AdjMat *mats, int batch, const long long *mn_start, long long total,
                            const double *S, const double *dU, double *W) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = batch - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (mn_start[mid] <= e) lo = mid;
            else hi = mid - 1;
        }
        const AdjMat M = mats[lo];
        const long long f = e - mn_start[lo];
        const int j = (int)(f / M.m);
        W[M.x_off + f] = dU ? dU[M.u_off + f] / S[M.s_off + j] : 0.0;
    }
}

int tiles_of(int M, int N) { return ((M + kGemmTile - 1) / kGemmTile) * ((N + kGemmTile - 1) / kGemmTile); }

}  // namespace

int jsvd_ctx::backward(int batch, const int *m, const int *n, const double *U, const long long *u_off,
                       const double *S, const long long *s_off, const double *V, const long long *v_off,
                       const double *dU, const double *dS, const double *dV, double *dA, const long long *a_off) {
    int rc;
    std::vector<AdjMat> mats(batch);
    long long w_tot = 0, nn_tot = 0, mn_tot = 0;
    std::vector<long long> nn_start(batch), mn_start(batch);
    for (int i = 0; i < batch; ++i) {
        AdjMat &M = mats[i];
        M.m = m[i];
        M.n = n[i];
        M.u_off = u_off[i];
        M.s_off = s_off[i];
        M.v_off = v_off[i];
        M.a_off = a_off[i];
        M.j_off = w_tot;
        w_tot += 3LL * M.n * M.n;
        M.x_off = w_tot;
        w_tot += (long long)M.m * M.n;
        nn_start[i] = nn_tot;
        nn_tot += (long long)M.n * M.n;
        mn_start[i] = mn_tot;
        mn_tot += (long long)M.m * M.n;
    }
    if ((rc = ensure(adj_w, sizeof(double) * std::max<long long>(w_tot, 1)))) return rc;
    if ((rc = ensure(adj_meta, sizeof(AdjMat) * batch + sizeof(long long) * 2 * batch))) return rc;
    double *W = (double *)adj_w.ptr;
    AdjMat *dm = (AdjMat *)adj_meta.ptr;
    long long *dstart = (long long *)((char *)adj_meta.ptr + sizeof(AdjMat) * batch);
    std::vector<long long> starts(nn_start);
    starts.insert(starts.end(), mn_start.begin(), mn_start.end());
    cudaMemcpyAsync(dm, mats.data(), sizeof(AdjMat) * batch, cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(dstart, starts.data(), sizeof(long long) * 2 * batch, cudaMemcpyHostToDevice, stream);

    // GEMM descriptor sets: (1) J = U^T dU, K = V^T dV   (2) X = U N + X   (3) dA = X V^T
    std::vector<GemmDesc> d1, d2, d3;
    int t1 = 0, t2 = 0, t3 = 0;
    for (int i = 0; i < batch; ++i) {
        const AdjMat &M = mats[i];
        double *J = W + M.j_off, *K = J + (size_t)M.n * M.n, *N = J + 2 * (size_t)M.n * M.n, *X = W + M.x_off;
        if (dU) {
            d1.push_back(GemmDesc{M.n, M.n, M.m, U + M.u_off, M.m, dU + M.u_off, M.m, J, M.n, 1.0, 0.0, t1});
            t1 += tiles_of(M.n, M.n);
        }
        if (dV) {
            d1.push_back(GemmDesc{M.n, M.n, M.n, V + M.v_off, M.n, dV + M.v_off, M.n, K, M.n, 1.0, 0.0, t1});
            t1 += tiles_of(M.n, M.n);
        }
        d2.push_back(GemmDesc{M.m, M.n, M.n, U + M.u_off, M.m, N, M.n, X, M.m, 1.0, 1.0, t2});
        t2 += tiles_of(M.m, M.n);
        d3.push_back(GemmDesc{M.m, M.n, M.n, X, M.m, V + M.v_off, M.n, dA + M.a_off, M.m, 1.0, 0.0, t3});
        t3 += tiles_of(M.m, M.n);
    }
    const size_t nd = d1.size() + d2.size() + d3.size();
    if ((rc = ensure(adj_desc, sizeof(GemmDesc) * nd))) return rc;
    GemmDesc *dd = (GemmDesc *)adj_desc.ptr;
    std::vector<GemmDesc> all(d1);
    all.insert(all.end(), d2.begin(), d2.end());
    all.insert(all.end(), d3.begin(), d3.end());
    cudaMemcpyAsync(dd, all.data(), sizeof(GemmDesc) * nd, cudaMemcpyHostToDevice, stream);
    // J and K start at zero when their cotangent is absent
    if (!dU || !dV) cudaMemsetAsync(W, 0, sizeof(double) * w_tot, stream);
    gemm_grouped(true, false, Elt::F64, Elt::F64, dd, (int)d1.size(), t1, stream);
    const int blocks = 1024;
    k_adj_middle<<<blocks, 256, 0, stream>>>(dm, batch, dstart, nn_tot, S, dS, W);
    k_adj_scale<<<blocks, 256, 0, stream>>>(dm, batch, dstart + batch, mn_tot, S, dU, W);
    gemm_grouped(false, false, Elt::F64, Elt::F64, dd + d1.size(), (int)d2.size(), t2, stream);
    gemm_grouped(false, true, Elt::F64, Elt::F64, dd + d1.size() + d2.size(), (int)d3.size(), t3, stream);
    prof_launches[4] += (d1.empty() ? 0 : 1) + 4;
    double fl = 0.0;
    for (auto &M : mats) fl += 6.0 * M.m * (double)M.n * M.n + 2.0 * (double)M.n * M.n * M.n;
    prof_flops[4] += fl;
    if ((rc = check("adjoint"))) return rc;
    // the host descriptor vectors must outlive the async copies
    return sync("adjoint");
}

extern "C" int jsvd_dgesvj_backward(jsvd_ctx_t ctx, int batch, const int *m, const int *n, const double *U,
                                    const long long *u_off, const double *S, const long long *s_off,
                                    const double *V, const long long *v_off, const double *dU, const double *dS,
                                    const double *dV, double *dA, const long long *a_off) {
    if (!ctx) return -1;
    if (batch < 0) return -2;
    if (batch == 0) return 0;
    if (!m) return -3;
    if (!n) return -4;
    for (int i = 0; i < batch; ++i)
        if (m[i] < 1 || n[i] < 1 || m[i] < n[i]) return -3;
    if (!U || !u_off) return -5;
    if (!S || !s_off) return -7;
    if (!V || !v_off) return -9;
    if (!dA || !a_off) return -14;
    cudaSetDevice(ctx->device);
    return ctx->backward(batch, m, n, U, u_off, S, s_off, V, v_off, dU, dS, dV, dA, a_off);
}
