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
    // update: 4 producer warps (load, exponents, digits) and 4 consumer warps
    // (one 16x16 output tile each) over double-buffered blocks of kMB rows;
    // every producer thread holds 8 entries of a block (one row, 8 columns)
    static constexpr int kCG = BB / 8;                                 // column groups of 8
    static constexpr int kMB = 128 / kCG;                              // rows per block: 16, 32, 64
    static constexpr int kULd = BB + split::kPad;
    static constexpr int kUSliceA = kMB * kULd;
    static constexpr int kUSliceB = BB * kULd;
    static constexpr int kUpdWarps = 8;
    static constexpr int kUpdRowsPerCta = 512;                         // rows of one update CTA
    static_assert((kMB / 16) * (BB / 16) == 4, "one tile per consumer warp");
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
    return 2u * split::kSlices * (2 * S::kUSliceA + S::kUSliceB) + sizeof(int) * (2 * BB + 2 * (S::kCG + 1) * S::kMB);
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
//
// Warps 0-3 produce: load block t (thread p: row p % kMB, columns
// 8 (p / kMB) .. +7), reduce the row exponents, write the digits to buffer
// t % 2, and arrive on FULL(t % 2).  Warps 4-7 consume: wait on FULL, run the
// level MMAs of their tile, read the tile rows' exponents, arrive on EMPTY
// (which the producers wait on before refilling that buffer two blocks
// later), then combine and store.  Named barriers with matched counts: every
// producer and consumer thread runs the same number of blocks.
namespace nb {
constexpr int kFull0 = 1, kEmpty0 = 3, kProd = 5;   // ids 1-2 FULL, 3-4 EMPTY, 5 producers only
}
template <int ID, int COUNT>
__device__ __forceinline__ void bar_sync() {
    asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(COUNT) : "memory");
}
template <int ID, int COUNT>
__device__ __forceinline__ void bar_arrive() {
    asm volatile("bar.arrive %0, %1;" ::"n"(ID), "n"(COUNT) : "memory");
}
// barrier of buffer buf (0 or 1) with immediate ids
template <int ID0, int COUNT>
__device__ __forceinline__ void bar_sync_buf(int buf) {
    if (buf) bar_sync<ID0 + 1, COUNT>(); else bar_sync<ID0, COUNT>();
}
template <int ID0, int COUNT>
__device__ __forceinline__ void bar_arrive_buf(int buf) {
    if (buf) bar_arrive<ID0 + 1, COUNT>(); else bar_arrive<ID0, COUNT>();
}

template <int BB>
__global__ void __launch_bounds__(32 * SplitCfg<BB>::kUpdWarps) update_split(PStepArgs a, int g_units) {
    using S = SplitCfg<BB>;
    constexpr int MB = S::kMB;
    constexpr int CG = S::kCG;
    constexpr int NT = 32 * S::kUpdWarps;             // 256
    constexpr int NP = NT / 2;                         // producer threads
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint16_t *As = reinterpret_cast<uint16_t *>(smem_raw);                 // [2][kSlices][MB][kULd]
    uint16_t *Bs = As + 2 * split::kSlices * S::kUSliceA;                   // [kSlices][BB][kULd]
    int *fexp = reinterpret_cast<int *>(Bs + split::kSlices * S::kUSliceB);
    int *dexp = fexp + BB;
    int *rmax = dexp + BB;                // [2][CG][MB]
    int *rexp = rmax + 2 * CG * MB;       // [2][MB]

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
    const int nblk = (min(rows, rbeg + S::kUpdRowsPerCta) - rbeg) / MB;   // rows is a multiple of 256

    // right factor digits and exponents of this pair and version
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.bslice + ((size_t)pair * 2 + ver) * split_b_elems<BB>());
        uint4 *dst = reinterpret_cast<uint4 *>(Bs);
        for (int e = threadIdx.x; e < split_b_elems<BB>() / 8; e += NT) dst[e] = src[e];
        for (int k = threadIdx.x; k < BB; k += NT) {
            fexp[k] = a.bexp[((size_t)pair * 2 + ver) * BB + k];
            dexp[k] = ver ? 0 : a.dexp[(size_t)pair * BB + k];
        }
    }
    __syncthreads();

    if (threadIdx.x < NP) {
        // ---------------- producers ----------------
        const int p = threadIdx.x;
        const int r = p % MB, cg = p / MB;
        const double *src0 = X + rbeg + r;
        size_t coff[8];
        int dx[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            coff[c] = (size_t)block_col(P, Q, a.b, 8 * cg + c) * ld;
            dx[c] = dexp[8 * cg + c];
        }
        double x[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) x[c] = src0[coff[c]];
        for (int t = 0; t < nblk; ++t) {
            const int buf = t & 1;
            int m = split::kNoExp;
#pragma unroll
            for (int c = 0; c < 8; ++c) m = max(m, split::exp_bound(x[c], -dx[c]));
            rmax[(buf * CG + cg) * MB + r] = m;
            bar_sync<nb::kProd, NP>();
            int E = split::kNoExp;
#pragma unroll
            for (int g = 0; g < CG; ++g) E = max(E, rmax[(buf * CG + g) * MB + r]);
            if (E == split::kNoExp) E = 0;
            unsigned long long z[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) z[c] = split::fixed_biased(x[c], -dx[c], E);
            // prefetch the next block's entries while this one is split
            if (t + 1 < nblk) {
#pragma unroll
                for (int c = 0; c < 8; ++c) x[c] = src0[coff[c] + (size_t)(t + 1) * MB];
            }
            if (t >= 2) bar_sync_buf<nb::kEmpty0, NT>(buf);   // consumers are done with block t - 2
            if (cg == 0) rexp[buf * MB + r] = E;
            uint16_t *dst = As + (size_t)buf * split::kSlices * S::kUSliceA + r * S::kULd + 8 * cg;
            const unsigned long long z0[4] = {z[0], z[1], z[2], z[3]};
            const unsigned long long z1[4] = {z[4], z[5], z[6], z[7]};
            store_digits4(dst, S::kUSliceA, z0);
            store_digits4(dst + 4, S::kUSliceA, z1);
            bar_arrive_buf<nb::kFull0, NT>(buf);
        }
    } else {
        // ---------------- consumers ----------------
        const int cw = (threadIdx.x - NP) >> 5;        // 0..3: tile
        constexpr int TN = BB / 16;
        const int tm = cw / TN, tn = cw % TN;
        int gcol[8];
        int fx[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int col = tn * 16 + split::acc_col(e);
            gcol[e] = block_col(P, Q, a.b, col);
            fx[e] = fexp[col];
        }
        for (int t = 0; t < nblk; ++t) {
            const int buf = t & 1;
            bar_sync_buf<nb::kFull0, NT>(buf);
            float lev[split::kLevels][8];
            split::zero_levels(lev);
            const uint16_t *Ab = As + (size_t)buf * split::kSlices * S::kUSliceA;
            split::tile_levels<BB / 16>(Ab + tm * 16 * S::kULd, S::kULd, S::kUSliceA, Bs + tn * 16 * S::kULd, S::kULd,
                                        S::kUSliceB, lev);
            const int r0 = tm * 16 + split::acc_row(0), r1 = tm * 16 + split::acc_row(2);
            const int e0 = rexp[buf * MB + r0], e1 = rexp[buf * MB + r1];
            if (t + 2 < nblk) bar_arrive_buf<nb::kEmpty0, NT>(buf);
            const size_t rb = (size_t)rbeg + (size_t)t * MB;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                float lv[split::kLevels];
#pragma unroll
                for (int L = 0; L < split::kLevels; ++L) lv[L] = lev[L][e];
                const int row = (e & 2) ? r1 : r0;
                X[(size_t)gcol[e] * ld + rb + row] = split::combine<true>(lv, (e & 2) ? e1 : e0, fx[e]);
            }
        }
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
