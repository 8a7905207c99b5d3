// Tensor-core forms of the two contractions of the FP64 block p-step
// (Eq. (2.7) Gram partials, Eq. (2.9) block update) on split bf16 digits; the
// arithmetic is described in split_mma.cuh.  Launched by launch_phase when
// PStepArgs::split is set; the per-pair Cholesky and inner sweep are the FP64
// pair_jacobi kernel, whose epilogue writes the split right factors.
#include <cuda_runtime.h>

#include <cstdint>

#include "split_mma.cuh"
#include "sweep_fp64.cuh"

namespace jsvd {

template <int BB> struct SplitCfg {
    static constexpr int kTiles = (BB / 16) * (BB / 16 + 1) / 2;       // lower-triangle 16x16 tiles: 1, 3, 10
    static constexpr int kKsplit = BB == 64 ? 1 : (BB == 32 ? 2 : 4);  // K parts per tile (warps per tile)
    static constexpr int kGramWarps = kTiles * kKsplit;                // 4, 6, 10
    static constexpr int kGLd = kGramRows + split::kPad;               // digit row stride (K = rows)
    static constexpr int kGSlice = BB * kGLd;
    // update: rows per block; at BB = 64, 32 rows keep the CTA's shared memory
    // small enough for a pair_jacobi CTA to run beside it on the same SM
    static constexpr int kMB = BB == 64 ? 32 : 128;
    static constexpr int kULd = BB + split::kPad;
    static constexpr int kUSliceA = kMB * kULd;
    static constexpr int kUSliceB = BB * kULd;
    static constexpr int kUpdWarps = 8;
    static constexpr int kUpdRowsPerCta = 512;                         // rows of one update CTA
};

template <int BB>
constexpr size_t gram_split_smem() {
    using S = SplitCfg<BB>;
    return 2u * split::kSlices * S::kGSlice + sizeof(int) * BB +
           sizeof(float) * (S::kKsplit - 1) * S::kTiles * split::kLevels * 8 * 32;
}
template <int BB>
constexpr size_t update_split_smem() {
    using S = SplitCfg<BB>;
    return 2u * split::kSlices * (S::kUSliceA + S::kUSliceB) + sizeof(int) * (2 * BB + (S::kUpdWarps + 1) * S::kMB);
}

// Store the 9 digits of 4 consecutive K entries (one 8-byte store per slice).
__device__ __forceinline__ void store_digits4(uint16_t *dst, int slice_stride, const unsigned long long (&z)[4]) {
#define JSVD_D4(I)                                                                                            \
    *reinterpret_cast<uint2 *>(dst + (I) * slice_stride) =                                                    \
        make_uint2(split::pack2(split::digit_bf16<I>(z[0]), split::digit_bf16<I>(z[1])),                       \
                   split::pack2(split::digit_bf16<I>(z[2]), split::digit_bf16<I>(z[3])));
    JSVD_D4(0) JSVD_D4(1) JSVD_D4(2) JSVD_D4(3) JSVD_D4(4) JSVD_D4(5) JSVD_D4(6) JSVD_D4(7) JSVD_D4(8)
#undef JSVD_D4
}

// ---------------------------------------------------------------------------
// Gram partial of one 128-row chunk of [G_P G_Q] (lower triangle, packed),
// grid (chunks, pairs).  Column c of the chunk gets the exponent bound E_c of
// its 128 entries; H(j, k) = 2^(E_j + E_k - 40) * combine(levels).
template <int BB>
__global__ void __launch_bounds__(32 * SplitCfg<BB>::kGramWarps) gram_split(PStepArgs a) {
    using S = SplitCfg<BB>;
    constexpr int NW = S::kGramWarps;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint16_t *Dg = reinterpret_cast<uint16_t *>(smem_raw);
    int *cexp = reinterpret_cast<int *>(smem_raw + 2u * split::kSlices * S::kGSlice);
    float *red = reinterpret_cast<float *>(cexp + BB);

    const int pair = blockIdx.y, chunk = blockIdx.x;
    const int P = a.table[2 * (a.step * a.npairs + pair)];
    const int Q = a.table[2 * (a.step * a.npairs + pair) + 1];
    const double *G = reinterpret_cast<const double *>(a.G);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = chunk * kGramRows;

    // (1) one warp per column: 128 rows (4 per lane), exponent bound, digits
    for (int c = warp; c < BB; c += NW) {
        const double *col = G + (size_t)block_col(P, Q, a.b, c) * a.ldg + r0 + 4 * lane;
        const double2 x01 = *reinterpret_cast<const double2 *>(col);
        const double2 x23 = *reinterpret_cast<const double2 *>(col + 2);
        int E = max(max(split::exp_bound(x01.x, 0), split::exp_bound(x01.y, 0)),
                    max(split::exp_bound(x23.x, 0), split::exp_bound(x23.y, 0)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
        if (E == split::kNoExp) E = 0;
        const unsigned long long z[4] = {split::fixed_biased(x01.x, 0, E), split::fixed_biased(x01.y, 0, E),
                                         split::fixed_biased(x23.x, 0, E), split::fixed_biased(x23.y, 0, E)};
        store_digits4(Dg + c * S::kGLd + 4 * lane, S::kGSlice, z);
        if (lane == 0) cexp[c] = E;
    }
    __syncthreads();

    // (2) warp -> (lower tile t, K part); levels over its K range
    const int t = warp % S::kTiles, kpart = warp / S::kTiles;
    int I = 0;
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    const int J = t - I * (I + 1) / 2;
    constexpr int KSTEPS = kGramRows / 16 / S::kKsplit;
    float lev[split::kLevels][8];
    split::zero_levels(lev);
    const int k0 = kpart * 16 * KSTEPS;
    split::tile_levels<KSTEPS>(Dg + I * 16 * S::kGLd + k0, S::kGLd, S::kGSlice, Dg + J * 16 * S::kGLd + k0, S::kGLd,
                               S::kGSlice, lev);
    if (S::kKsplit > 1) {
        // the K parts' level sums are exact integers: add them in part order
        float *mine = red + (((size_t)(kpart - 1) * S::kTiles + t) * split::kLevels * 8) * 32 + lane;
        if (kpart > 0) {
#pragma unroll
            for (int L = 0; L < split::kLevels; ++L)
#pragma unroll
                for (int e = 0; e < 8; ++e) mine[(L * 8 + e) * 32] = lev[L][e];
        }
        __syncthreads();
        if (kpart == 0) {
            for (int p = 1; p < S::kKsplit; ++p) {
                const float *src = red + (((size_t)(p - 1) * S::kTiles + t) * split::kLevels * 8) * 32 + lane;
#pragma unroll
                for (int L = 0; L < split::kLevels; ++L)
#pragma unroll
                    for (int e = 0; e < 8; ++e) lev[L][e] += src[(L * 8 + e) * 32];
            }
        }
    }
    if (kpart == 0) {
        double *out = a.part + ((size_t)pair * a.g_chunks + chunk) * Cfg<BB>::kPacked;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int row = I * 16 + split::acc_row(e), col = J * 16 + split::acc_col(e);
            if (row < col) continue;
            float lv[split::kLevels];
#pragma unroll
            for (int L = 0; L < split::kLevels; ++L) lv[L] = lev[L][e];
            out[packed_lower<BB>(row, col)] = split::combine<false>(lv, cexp[row], cexp[col]);
        }
    }
}

// ---------------------------------------------------------------------------
// [X_P X_Q] := [X_P X_Q] V' on split digits, grid (units, pairs); a unit is
// kUpdRowsPerCta rows of G (blockIdx.x < g_units) or of V.  For G the A
// operand is G D^-1 (D from the pair's Gram diagonal) against the digits of
// D V'; for V it is V against those of V'.  Row r of a block gets the exponent
// bound E_r of its BB entries; X(r, k) = 2^(E_r + F_k - 40) * combine(levels).
template <int BB>
__global__ void __launch_bounds__(32 * SplitCfg<BB>::kUpdWarps) update_split(PStepArgs a, int g_units) {
    using S = SplitCfg<BB>;
    constexpr int NW = S::kUpdWarps;
    constexpr int MB = S::kMB;
    constexpr int CPW = BB / NW;          // columns per warp when loading: 8, 4, 2
    constexpr int RPL = MB / 32;          // rows per lane: 1, 4, 4
    static_assert(RPL == 1 || RPL % 2 == 0, "rows per lane");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint16_t *As = reinterpret_cast<uint16_t *>(smem_raw);
    uint16_t *Bs = As + split::kSlices * S::kUSliceA;
    int *fexp = reinterpret_cast<int *>(Bs + split::kSlices * S::kUSliceB);
    int *dexp = fexp + BB;
    int *rmax = dexp + BB;                // [NW][MB]
    int *rexp = rmax + NW * MB;           // [MB]

    const int pair = blockIdx.y;
    if (!a.vflag[pair]) return;
    const int P = a.table[2 * (a.step * a.npairs + pair)];
    const int Q = a.table[2 * (a.step * a.npairs + pair) + 1];
    const int ver = (int)blockIdx.x < g_units ? 0 : 1;
    const int unit = ver ? (int)blockIdx.x - g_units : (int)blockIdx.x;
    double *X = reinterpret_cast<double *>(ver ? a.V : a.G);
    const int ld = ver ? a.ldv : a.ldg;
    const int rows = ver ? a.v_rows : a.g_rows;
    const int rbeg = unit * S::kUpdRowsPerCta;
    const int rend = min(rows, rbeg + S::kUpdRowsPerCta);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // right factor digits and exponents of this pair and version
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.bslice + ((size_t)pair * 2 + ver) * split_b_elems<BB>());
        uint4 *dst = reinterpret_cast<uint4 *>(Bs);
        for (int e = threadIdx.x; e < split_b_elems<BB>() / 8; e += 32 * NW) dst[e] = src[e];
        for (int k = threadIdx.x; k < BB; k += 32 * NW) {
            fexp[k] = a.bexp[((size_t)pair * 2 + ver) * BB + k];
            dexp[k] = ver ? 0 : a.dexp[(size_t)pair * BB + k];
        }
    }
    __syncthreads();

    int gcol[CPW];
#pragma unroll
    for (int c = 0; c < CPW; ++c) gcol[c] = block_col(P, Q, a.b, warp * CPW + c);

    for (int rb = rbeg; rb < rend; rb += MB) {
        // (1) load: warp w takes columns [w CPW, (w+1) CPW), lane rows rb + lane RPL + q
        double x[CPW][RPL];
#pragma unroll
        for (int c = 0; c < CPW; ++c) {
            const double *src = X + (size_t)gcol[c] * ld + rb + lane * RPL;
            if constexpr (RPL == 1) {
                x[c][0] = src[0];
            } else {
#pragma unroll
                for (int q = 0; q < RPL; q += 2) {   // RPL even: 16-byte aligned pairs
                    const double2 v = *reinterpret_cast<const double2 *>(src + q);
                    x[c][q] = v.x;
                    x[c][q + 1] = v.y;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            int m = split::kNoExp;
#pragma unroll
            for (int c = 0; c < CPW; ++c) m = max(m, split::exp_bound(x[c][q], -dexp[warp * CPW + c]));
            rmax[warp * MB + lane * RPL + q] = m;
        }
        __syncthreads();
        // (2) row exponent bounds and digits of x 2^-dexp
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int r = lane * RPL + q;
            int E = split::kNoExp;
#pragma unroll
            for (int w = 0; w < NW; ++w) E = max(E, rmax[w * MB + r]);
            if (E == split::kNoExp) E = 0;
            if (warp == 0) rexp[r] = E;
            uint16_t *dst = As + r * S::kULd + warp * CPW;
            if constexpr (CPW >= 4) {
#pragma unroll
                for (int c = 0; c < CPW; c += 4) {
                    const unsigned long long z[4] = {
                        split::fixed_biased(x[c][q], -dexp[warp * CPW + c], E),
                        split::fixed_biased(x[c + 1][q], -dexp[warp * CPW + c + 1], E),
                        split::fixed_biased(x[c + 2][q], -dexp[warp * CPW + c + 2], E),
                        split::fixed_biased(x[c + 3][q], -dexp[warp * CPW + c + 3], E)};
                    store_digits4(dst + c, S::kUSliceA, z);
                }
            } else {
                static_assert(CPW == 2, "two columns per warp");
                const unsigned long long z0 = split::fixed_biased(x[0][q], -dexp[warp * CPW], E);
                const unsigned long long z1 = split::fixed_biased(x[CPW - 1][q], -dexp[warp * CPW + 1], E);
#define JSVD_D2(I) \
    *reinterpret_cast<uint32_t *>(dst + (I) * S::kUSliceA) = split::pack2(split::digit_bf16<I>(z0), split::digit_bf16<I>(z1));
                JSVD_D2(0) JSVD_D2(1) JSVD_D2(2) JSVD_D2(3) JSVD_D2(4) JSVD_D2(5) JSVD_D2(6) JSVD_D2(7) JSVD_D2(8)
#undef JSVD_D2
            }
        }
        __syncthreads();
        // (3) 16x16 output tiles over the warps; combine and store to X
        constexpr int TM = MB / 16, TN = BB / 16;
        for (int t = warp; t < TM * TN; t += NW) {
            const int tm = t / TN, tn = t % TN;
            float lev[split::kLevels][8];
            split::zero_levels(lev);
            split::tile_levels<BB / 16>(As + tm * 16 * S::kULd, S::kULd, S::kUSliceA, Bs + tn * 16 * S::kULd, S::kULd,
                                        S::kUSliceB, lev);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int row = tm * 16 + split::acc_row(e), col = tn * 16 + split::acc_col(e);
                float lv[split::kLevels];
#pragma unroll
                for (int L = 0; L < split::kLevels; ++L) lv[L] = lev[L][e];
                X[(size_t)block_col(P, Q, a.b, col) * ld + rb + row] = split::combine<true>(lv, rexp[row], fexp[col]);
            }
        }
        __syncthreads();
    }
}

template <int BB>
static void configure_split_once() {
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    cudaFuncSetAttribute(gram_split<BB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_split_smem<BB>());
    cudaFuncSetAttribute(update_split<BB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)update_split_smem<BB>());
    done[dev] = true;
}

template <int BB>
static void launch_split_bb(Phase ph, const PStepArgs &a, cudaStream_t s) {
    using S = SplitCfg<BB>;
    configure_split_once<BB>();
    if (ph == Phase::Gram) {
        gram_split<BB><<<dim3(a.g_chunks, a.npairs), 32 * S::kGramWarps, gram_split_smem<BB>(), s>>>(a);
        return;
    }
    const int gu = (ph == Phase::UpdateV) ? 0 : (a.g_rows + S::kUpdRowsPerCta - 1) / S::kUpdRowsPerCta;
    const int vu = (ph == Phase::UpdateG || !a.V) ? 0 : (a.v_rows + S::kUpdRowsPerCta - 1) / S::kUpdRowsPerCta;
    if (gu + vu > 0)
        update_split<BB><<<dim3(gu + vu, a.npairs), 32 * S::kUpdWarps, update_split_smem<BB>(), s>>>(a, gu);
}

void launch_split_phase(int BB, Phase ph, const PStepArgs &a, cudaStream_t s) {
    switch (BB) {
        case 16: launch_split_bb<16>(ph, a, s); break;
        case 32: launch_split_bb<32>(ph, a, s); break;
        case 64: launch_split_bb<64>(ph, a, s); break;
        default: break;
    }
}

}  // namespace jsvd
