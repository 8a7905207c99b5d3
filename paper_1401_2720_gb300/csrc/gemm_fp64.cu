// FP64-accumulating tiled GEMM; see gemm_fp64.cuh.
#include <cuda_runtime.h>

#include "gemm_fp64.cuh"

namespace jsvd {
namespace {

constexpr int BM = kGemmTile, BN = kGemmTile, BK = 16, THREADS = 256;

template <typename T>
__device__ __forceinline__ double ld_elt(const void *p, size_t i) {
    return (double)reinterpret_cast<const T *>(p)[i];
}

// One 64x64 tile of C; thread (tm, tn) owns rows 4tm..4tm+3, cols 4tn..4tn+3.
template <bool TA, bool TB, typename EA, typename EB>
__device__ __forceinline__ void gemm_tile(const GemmDesc &d, int tile_m, int tile_n,
                                          double (*As)[BM], double (*Bs)[BN]) {
    const int t = threadIdx.x;
    const int tm = t % 16, tn = t / 16;
    const int m0 = tile_m * BM, n0 = tile_n * BN;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    for (int k0 = 0; k0 < d.K; k0 += BK) {
        // op(A)[m][k] -> As[k][m]
#pragma unroll
        for (int i = 0; i < (BM * BK) / THREADS; ++i) {
            int m, k;
            if (!TA) { m = t % BM; k = t / BM + i * (THREADS / BM); }
            else     { k = t % BK; m = t / BK + i * (THREADS / BK); }
            const int gm = m0 + m, gk = k0 + k;
            double v = 0.0;
            if (gm < d.M && gk < d.K)
                v = TA ? ld_elt<EA>(d.A, (size_t)gm * d.lda + gk) : ld_elt<EA>(d.A, (size_t)gk * d.lda + gm);
            As[k][m] = v;
        }
        // op(B)[k][n] -> Bs[k][n]
#pragma unroll
        for (int i = 0; i < (BN * BK) / THREADS; ++i) {
            int n, k;
            if (!TB) { k = t % BK; n = t / BK + i * (THREADS / BK); }
            else     { n = t % BN; k = t / BN + i * (THREADS / BN); }
            const int gn = n0 + n, gk = k0 + k;
            double v = 0.0;
            if (gn < d.N && gk < d.K)
                v = TB ? ld_elt<EB>(d.B, (size_t)gk * d.ldb + gn) : ld_elt<EB>(d.B, (size_t)gn * d.ldb + gk);
            Bs[k][n] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            const double2 a01 = reinterpret_cast<const double2 *>(&As[k][4 * tm])[0];
            const double2 a23 = reinterpret_cast<const double2 *>(&As[k][4 * tm])[1];
            const double2 b01 = reinterpret_cast<const double2 *>(&Bs[k][4 * tn])[0];
            const double2 b23 = reinterpret_cast<const double2 *>(&Bs[k][4 * tn])[1];
            const double a[4] = {a01.x, a01.y, a23.x, a23.y};
            const double b[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = __fma_rn(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int gn = n0 + 4 * tn + j;
        if (gn >= d.N) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int gm = m0 + 4 * tm + i;
            if (gm >= d.M) continue;
            double *c = d.C + (size_t)gn * d.ldc + gm;
            const double v = d.alpha * acc[i][j];
            *c = (d.beta == 0.0) ? v : __fma_rn(d.beta, *c, v);
        }
    }
}

template <bool TA, bool TB, typename EA, typename EB>
__global__ void __launch_bounds__(THREADS) k_gemm_grouped(const GemmDesc *descs, int count) {
    __shared__ __align__(16) double As[BK][BM];
    __shared__ __align__(16) double Bs[BK][BN];
    const int tile = blockIdx.x;
    // binary search for the problem that owns this tile
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (descs[mid].tile0 <= tile) lo = mid;
        else hi = mid - 1;
    }
    const GemmDesc d = descs[lo];
    const int local = tile - d.tile0;
    const int tiles_m = (d.M + BM - 1) / BM;
    const int tiles_n = (d.N + BN - 1) / BN;
    if (local >= tiles_m * tiles_n) return;
    gemm_tile<TA, TB, EA, EB>(d, local % tiles_m, local / tiles_m, As, Bs);
}

template <bool TA, bool TB, typename EA, typename EB>
__global__ void __launch_bounds__(THREADS) k_gemm_one(GemmDesc d) {
    __shared__ __align__(16) double As[BK][BM];
    __shared__ __align__(16) double Bs[BK][BN];
    gemm_tile<TA, TB, EA, EB>(d, blockIdx.x, blockIdx.y, As, Bs);
}

template <bool TA, bool TB>
void dispatch_one(Elt ea, Elt eb, const GemmDesc &d, cudaStream_t s) {
    dim3 grid((d.M + BM - 1) / BM, (d.N + BN - 1) / BN);
    if (ea == Elt::F64 && eb == Elt::F64) k_gemm_one<TA, TB, double, double><<<grid, THREADS, 0, s>>>(d);
    else if (ea == Elt::F32 && eb == Elt::F64) k_gemm_one<TA, TB, float, double><<<grid, THREADS, 0, s>>>(d);
    else if (ea == Elt::F64 && eb == Elt::F32) k_gemm_one<TA, TB, double, float><<<grid, THREADS, 0, s>>>(d);
    else k_gemm_one<TA, TB, float, float><<<grid, THREADS, 0, s>>>(d);
}

template <bool TA, bool TB>
void dispatch_grouped(Elt ea, Elt eb, const GemmDesc *d, int count, int tiles, cudaStream_t s) {
    if (ea == Elt::F64 && eb == Elt::F64) k_gemm_grouped<TA, TB, double, double><<<tiles, THREADS, 0, s>>>(d, count);
    else if (ea == Elt::F32 && eb == Elt::F64) k_gemm_grouped<TA, TB, float, double><<<tiles, THREADS, 0, s>>>(d, count);
    else if (ea == Elt::F64 && eb == Elt::F32) k_gemm_grouped<TA, TB, double, float><<<tiles, THREADS, 0, s>>>(d, count);
    else k_gemm_grouped<TA, TB, float, float><<<tiles, THREADS, 0, s>>>(d, count);
}

}  // namespace

void gemm(bool ta, bool tb, Elt ea, Elt eb, int M, int N, int K, double alpha, const void *A, int lda,
          const void *B, int ldb, double beta, double *C, int ldc, cudaStream_t s) {
    if (M <= 0 || N <= 0) return;
    GemmDesc d{M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, 0};
    if (!ta && !tb) dispatch_one<false, false>(ea, eb, d, s);
    else if (ta && !tb) dispatch_one<true, false>(ea, eb, d, s);
    else if (!ta && tb) dispatch_one<false, true>(ea, eb, d, s);
    else dispatch_one<true, true>(ea, eb, d, s);
}

void gemm_grouped(bool ta, bool tb, Elt ea, Elt eb, const GemmDesc *descs, int count, int total_tiles,
                  cudaStream_t s) {
    if (count <= 0 || total_tiles <= 0) return;
    if (!ta && !tb) dispatch_grouped<false, false>(ea, eb, descs, count, total_tiles, s);
    else if (ta && !tb) dispatch_grouped<true, false>(ea, eb, descs, count, total_tiles, s);
    else if (!ta && tb) dispatch_grouped<false, true>(ea, eb, descs, count, total_tiles, s);
    else dispatch_grouped<true, true>(ea, eb, descs, count, total_tiles, s);
}

}  // namespace jsvd
