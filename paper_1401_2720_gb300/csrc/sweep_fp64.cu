// FP64 block p-step kernels; see sweep_fp64.cuh for the decomposition.
#include <cuda_runtime.h>

#include <cstdint>

#include "rotation.cuh"
#include "sweep_fp64.cuh"

namespace jsvd {

__device__ __forceinline__ int block_col(int P, int Q, int b, int j) {
    return j < b ? P * b + j : Q * b + (j - b);
}

// Index of (i, j), i >= j, in the column-major packed lower triangle of order BB.
template <int BB>
__device__ __forceinline__ int packed_lower(int i, int j) {
    return j * BB - (j * (j - 1)) / 2 + (i - j);
}

// ---------------------------------------------------------------------------
// Gram partials: one CTA = one row chunk of one block pair.  The chunk is
// staged row-major in shared memory (row stride BB+2 doubles) so that each
// thread reads 2x2 blocks of operands with 16-byte loads; each thread owns
// 2x2 blocks (I, J), I >= J, of the lower triangle of H_pq and accumulates
// them over the chunk's rows in increasing row order.
template <int BB>
__global__ void __launch_bounds__(kGramThreads)
gram_partial(PStepArgs a) {
    using C = Cfg<BB>;
    extern __shared__ __align__(16) double smem[];
    double *X = smem;  // [kGramRows][kGramLd]
    const int pair = blockIdx.y, chunk = blockIdx.x;
    const int P = a.table[2 * (a.step * a.npairs + pair)];
    const int Q = a.table[2 * (a.step * a.npairs + pair) + 1];
    const int r0 = chunk * kGramRows;

    // coalesced column reads, transposed into the row-major tile
    for (int e = threadIdx.x; e < kGramRows * BB; e += kGramThreads) {
        const int r = e % kGramRows, j = e / kGramRows;
        const int col = block_col(P, Q, a.b, j);
        X[r * C::kGramLd + j] = a.G[(size_t)col * a.ldg + r0 + r];
    }
    __syncthreads();

    constexpr int NB = BB / 2;                  // 2x2 blocks per dimension
    constexpr int NBLK = NB * (NB + 1) / 2;     // blocks in the lower triangle
    double *out = a.part + ((size_t)pair * a.g_chunks + chunk) * C::kPacked;
    for (int blk = threadIdx.x; blk < NBLK; blk += kGramThreads) {
        // blk -> (I, J), I >= J, row-major enumeration of the lower triangle
        int I = (int)((sqrtf(8.0f * blk + 1.0f) - 1.0f) * 0.5f);
        while ((I + 1) * (I + 2) / 2 <= blk) ++I;
        while (I * (I + 1) / 2 > blk) --I;
        const int J = blk - I * (I + 1) / 2;
        double h00 = 0.0, h10 = 0.0, h01 = 0.0, h11 = 0.0;
        const double *xi = X + 2 * I, *xj = X + 2 * J;
#pragma unroll 4
        for (int r = 0; r < kGramRows; ++r) {
            const double2 u = *reinterpret_cast<const double2 *>(xi + r * C::kGramLd);
            const double2 v = *reinterpret_cast<const double2 *>(xj + r * C::kGramLd);
            h00 = __fma_rn(u.x, v.x, h00);
            h10 = __fma_rn(u.y, v.x, h10);
            h01 = __fma_rn(u.x, v.y, h01);
            h11 = __fma_rn(u.y, v.y, h11);
        }
        const int i0 = 2 * I, j0 = 2 * J;
        out[packed_lower<BB>(i0, j0)] = h00;
        out[packed_lower<BB>(i0 + 1, j0)] = h10;
        out[packed_lower<BB>(i0 + 1, j0 + 1)] = h11;
        if (I != J) out[packed_lower<BB>(i0, j0 + 1)] = h01;
    }
}

// ---------------------------------------------------------------------------
// Per-pair factorization and inner sweep.  Shared memory: A and B, each
// BB x BB column-major with ld BB+1, plus the inner table.
//   A: H (lower) -> L by Cholesky -> later V' (= I, then rotated)
//   B: R = L^T (upper), rotated in the inner sweep
// Inner p-step: pair y of the inner table is handled by the 8-lane group y;
// lane g of the group owns rows g, g+8, ... of both columns in R and V'.
template <int BB>
__global__ void __launch_bounds__(Cfg<BB>::kJacThreads)
pair_jacobi(PStepArgs a) {
    using C = Cfg<BB>;
    extern __shared__ __align__(16) double smem[];
    double *A = smem;                      // [BB][kLd]
    double *B = smem + BB * C::kLd;        // [BB][kLd]
    unsigned char *tab = reinterpret_cast<unsigned char *>(smem + 2 * BB * C::kLd);
    __shared__ double s_piv;
    __shared__ int s_brk;
    __shared__ unsigned long long s_off;
    __shared__ int s_cnt[2];

    const int tid = threadIdx.x;
    const int pair = blockIdx.x;
    const int P = a.table[2 * (a.step * a.npairs + pair)];
    const int Q = a.table[2 * (a.step * a.npairs + pair) + 1];

    for (int e = tid; e < (BB - 1) * BB; e += C::kJacThreads) tab[e] = a.inner[e];
    if (tid == 0) { s_off = 0ull; s_brk = 0; s_cnt[0] = 0; s_cnt[1] = 0; }

    // (1) H = sum of the row-chunk partials, in chunk order
    const double *part = a.part + (size_t)pair * a.g_chunks * C::kPacked;
    for (int e = tid; e < BB * BB; e += C::kJacThreads) {
        const int i = e % BB, j = e / BB;
        if (i < j) continue;
        const int k = packed_lower<BB>(i, j);
        double s = 0.0;
        for (int c = 0; c < a.g_chunks; ++c) s = __dadd_rn(s, part[(size_t)c * C::kPacked + k]);
        A[i + j * C::kLd] = s;
    }
    __syncthreads();

    // (2) normalized off-diagonal maximum of H (convergence report)
    {
        double mx = 0.0;
        for (int e = tid; e < BB * BB; e += C::kJacThreads) {
            const int i = e % BB, j = e / BB;
            if (i <= j) continue;
            const double d = A[i + i * C::kLd] * A[j + j * C::kLd];
            if (d > 0.0) mx = fmax(mx, fabs(A[i + j * C::kLd]) / sqrt(d));
        }
        atomicMax(&s_off, (unsigned long long)__double_as_longlong(mx));
    }

    // (3) Cholesky H = L L^T without pivoting (Sec. 4.1), right-looking:
    // entry (i, j) receives -L(i,k) L(j,k) for k = 0, 1, ... in order, then the
    // division by the pivot.  A non-positive pivot zeroes its column.
    for (int k = 0; k < BB; ++k) {
        if (tid == 0) {
            const double d = A[k + k * C::kLd];
            if (d > 0.0) {
                s_piv = __dsqrt_rn(d);
            } else {
                s_piv = 0.0;
                s_brk += 1;
            }
        }
        __syncthreads();
        const double piv = s_piv;
        for (int i = k + tid; i < BB; i += C::kJacThreads)
            A[i + k * C::kLd] = (piv > 0.0) ? (i == k ? piv : __ddiv_rn(A[i + k * C::kLd], piv)) : 0.0;
        __syncthreads();
        const int rem = BB - 1 - k;  // trailing order
        for (int e = tid; e < rem * rem; e += C::kJacThreads) {
            const int i = k + 1 + e % rem, j = k + 1 + e / rem;
            if (i >= j)
                A[i + j * C::kLd] = __fma_rn(-A[i + k * C::kLd], A[j + k * C::kLd], A[i + j * C::kLd]);
        }
        __syncthreads();
    }

    // (4) R = L^T into B; V' = I into A
    for (int e = tid; e < BB * BB; e += C::kJacThreads) {
        const int i = e % BB, j = e / BB;
        B[i + j * C::kLd] = (i <= j) ? A[j + i * C::kLd] : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < BB * BB; e += C::kJacThreads) {
        const int i = e % BB, j = e / BB;
        A[i + j * C::kLd] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();

    // (5) inner sweeps of the pointwise one-sided method on R (Sec. 4.3)
    const int y = tid / C::kLanesPerPair;          // inner pair of this group
    const int g = tid % C::kLanesPerPair;          // lane within the group
    const double c_eps = kEps * sqrt((double)BB);  // c(eps) = eps sqrt(nhat), nhat = BB
    int my_rot = 0, my_proper = 0, changed = 0;
    for (int sw = 0; sw < a.inner_sweeps; ++sw) {
        int sweep_rot = 0;
        for (int st = 0; st < BB - 1; ++st) {
            const int p = tab[2 * (st * (BB / 2) + y)];
            const int q = tab[2 * (st * (BB / 2) + y) + 1];
            double *rp = B + p * C::kLd, *rq = B + q * C::kLd;
            double *wp = A + p * C::kLd, *wq = A + q * C::kLd;
            double hpp = 0.0, hqq = 0.0, hpq = 0.0;
#pragma unroll
            for (int k = 0; k < C::kRowsPerLane; ++k) {
                const int r = g + k * C::kLanesPerPair;
                const double x = rp[r], z = rq[r];
                hpp = __fma_rn(x, x, hpp);
                hqq = __fma_rn(z, z, hqq);
                hpq = __fma_rn(x, z, hpq);
            }
#pragma unroll
            for (int off = C::kLanesPerPair / 2; off > 0; off >>= 1) {
                hpp = __dadd_rn(hpp, __shfl_xor_sync(0xffffffffu, hpp, off));
                hqq = __dadd_rn(hqq, __shfl_xor_sync(0xffffffffu, hqq, off));
                hpq = __dadd_rn(hpq, __shfl_xor_sync(0xffffffffu, hpq, off));
            }
            const int gp = block_col(P, Q, a.b, p), gq = block_col(P, Q, a.b, q);
            const double t = (gp < a.nplus && gq >= a.nplus) ? -1.0 : 1.0;
            const bool rho = needs_rotation(hpp, hqq, hpq, c_eps);
            Rot rot{1.0, 0.0};
            if (rho) rot = rot_params(hpp, hqq, hpq, t);
            bool swap = false;
            if (t > 0.0) {
                const double npp = rho ? __fma_rn(-rot.tn, hpq, hpp) : hpp;
                const double nqq = rho ? __fma_rn(rot.tn, hpq, hqq) : hqq;
                swap = (gq < a.nplus && npp < nqq) || (gp >= a.nplus && npp > nqq);
            }
            if (rho || swap) {
#pragma unroll
                for (int k = 0; k < C::kRowsPerLane; ++k) {
                    const int r = g + k * C::kLanesPerPair;
                    double x = rp[r], z = rq[r];
                    double u = wp[r], v = wq[r];
                    if (rho) { rot_apply(x, z, t, rot); rot_apply(u, v, t, rot); }
                    if (swap) {
                        rp[r] = z; rq[r] = x; wp[r] = v; wq[r] = u;
                    } else {
                        rp[r] = x; rq[r] = z; wp[r] = u; wq[r] = v;
                    }
                }
                changed = 1;
            }
            if (g == 0 && rho) {
                ++my_rot;
                ++sweep_rot;
                if (rot.cs != 1.0) ++my_proper;
            }
            __syncthreads();
        }
        if (a.inner_sweeps > 1 && __syncthreads_count(sweep_rot) == 0) break;
    }

    // (6) V' and its flag to global memory; counters
    const int any_change = __syncthreads_or(changed);
    double *vp = a.vprime + (size_t)pair * BB * BB;
    for (int e = tid; e < BB * BB; e += C::kJacThreads) {
        const int i = e % BB, j = e / BB;
        vp[e] = A[i + j * C::kLd];
    }
    atomicAdd(&s_cnt[0], my_rot);
    atomicAdd(&s_cnt[1], my_proper);
    __syncthreads();
    if (tid == 0) {
        a.vflag[pair] = any_change;
        atomicAdd(&a.counters[kCntRot], (unsigned long long)s_cnt[0]);
        atomicAdd(&a.counters[kCntProper], (unsigned long long)s_cnt[1]);
        if (any_change) atomicAdd(&a.counters[kCntUpdated], 1ull);
        if (s_brk) atomicAdd(&a.counters[kCntBreak], (unsigned long long)s_brk);
        atomicMax(&a.counters[kCntOff], s_off);
    }
}

// ---------------------------------------------------------------------------
// Block update [A_P A_Q] := [A_P A_Q] V' for one chunk of kUpdRows rows.
// X (chunk, column-major, ld kUpdRows) and V' (row-major by k, ld BB+2) in
// shared memory; each thread owns a 4x4 output tile and sums over k = 0..BB-1
// in increasing order.
template <int BB>
__global__ void __launch_bounds__(kUpdThreads)
block_update(PStepArgs a, int g_chunks_u) {
    using C = Cfg<BB>;
    constexpr int RU = C::kUpdRows;
    constexpr int WLD = BB + 2;
    extern __shared__ __align__(16) double smem[];
    double *X = smem;                // [BB][RU]
    double *W = smem + BB * RU;      // [BB][WLD], W[k*WLD + c] = V'(k, c)
    const int pair = blockIdx.y;
    if (!a.vflag[pair]) return;
    const int P = a.table[2 * (a.step * a.npairs + pair)];
    const int Q = a.table[2 * (a.step * a.npairs + pair) + 1];

    double *M;
    int ld, r0;
    if ((int)blockIdx.x < g_chunks_u) {
        M = a.G; ld = a.ldg; r0 = blockIdx.x * RU;
    } else {
        M = a.V; ld = a.ldv; r0 = (blockIdx.x - g_chunks_u) * RU;
    }
    const double *vp = a.vprime + (size_t)pair * BB * BB;
    for (int e = threadIdx.x; e < BB * BB; e += kUpdThreads) {
        const int k = e % BB, c = e / BB;          // vp is column-major: vp[k + c*BB]
        W[k * WLD + c] = vp[e];
    }
    for (int e = threadIdx.x; e < BB * RU / 2; e += kUpdThreads) {
        const int r2 = e % (RU / 2), j = e / (RU / 2);
        const int col = block_col(P, Q, a.b, j);
        reinterpret_cast<double2 *>(X + j * RU)[r2] =
            reinterpret_cast<const double2 *>(M + (size_t)col * ld + r0)[r2];
    }
    __syncthreads();

    const int rt = threadIdx.x % (RU / 4);     // row tile
    const int ct = threadIdx.x / (RU / 4);     // column tile (BB/4 of them)
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
#pragma unroll 4
    for (int k = 0; k < BB; ++k) {
        const double2 x01 = reinterpret_cast<const double2 *>(X + k * RU + 4 * rt)[0];
        const double2 x23 = reinterpret_cast<const double2 *>(X + k * RU + 4 * rt)[1];
        const double2 w01 = reinterpret_cast<const double2 *>(W + k * WLD + 4 * ct)[0];
        const double2 w23 = reinterpret_cast<const double2 *>(W + k * WLD + 4 * ct)[1];
        const double xv[4] = {x01.x, x01.y, x23.x, x23.y};
        const double wv[4] = {w01.x, w01.y, w23.x, w23.y};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = __fma_rn(xv[i], wv[j], acc[i][j]);
    }
    // every CTA of this pair owns disjoint rows: write in place
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int col = block_col(P, Q, a.b, 4 * ct + j);
        double2 *dst = reinterpret_cast<double2 *>(M + (size_t)col * ld + r0 + 4 * rt);
        dst[0] = make_double2(acc[0][j], acc[1][j]);
        dst[1] = make_double2(acc[2][j], acc[3][j]);
    }
}

// ---------------------------------------------------------------------------
template <int BB>
static void launch_bb(const PStepArgs &a, cudaStream_t s, cudaEvent_t *ev) {
    using C = Cfg<BB>;
    static bool configured = false;
    const size_t sm_gram = sizeof(double) * kGramRows * C::kGramLd;
    const size_t sm_jac = sizeof(double) * 2 * BB * C::kLd + (BB - 1) * BB + 16;
    const size_t sm_upd = sizeof(double) * (BB * C::kUpdRows + BB * (BB + 2));
    if (!configured) {
        cudaFuncSetAttribute(gram_partial<BB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_gram);
        cudaFuncSetAttribute(pair_jacobi<BB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_jac);
        cudaFuncSetAttribute(block_update<BB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_upd);
        configured = true;
    }
    if (ev) cudaEventRecord(ev[0], s);
    gram_partial<BB><<<dim3(a.g_chunks, a.npairs), kGramThreads, sm_gram, s>>>(a);
    if (ev) cudaEventRecord(ev[1], s);
    pair_jacobi<BB><<<a.npairs, C::kJacThreads, sm_jac, s>>>(a);
    if (ev) cudaEventRecord(ev[2], s);
    const int gu = a.g_rows / C::kUpdRows;
    const int vu = a.V ? a.v_rows / C::kUpdRows : 0;
    block_update<BB><<<dim3(gu + vu, a.npairs), kUpdThreads, sm_upd, s>>>(a, gu);
    if (ev) cudaEventRecord(ev[3], s);
}

size_t pstep_smem_jacobi(int BB) {
    return sizeof(double) * 2 * BB * (BB + 1) + (BB - 1) * BB + 16;
}

void launch_pstep_fp64(int BB, const PStepArgs &a, cudaStream_t s, cudaEvent_t *ev) {
    switch (BB) {
        case 16: launch_bb<16>(a, s, ev); break;
        case 32: launch_bb<32>(a, s, ev); break;
        case 64: launch_bb<64>(a, s, ev); break;
        default: break;
    }
}

}  // namespace jsvd
