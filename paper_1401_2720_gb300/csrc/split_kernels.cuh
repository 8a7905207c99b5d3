// Tensor-core forms of the two contractions of the FP64 block p-step
// (Eq. (2.7) Gram partials, Eq. (2.9) block update) on split bf16 digits, as
// device functions over an explicit row range: the single-matrix kernels
// (sweep_split.cu) and the batched solver (batched.cu) wrap them.  The digit
// arithmetic is described in split_mma.cuh.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "split_mma.cuh"
#include "sweep_device.cuh"

namespace jsvd {

template <int BB> struct SplitCfg {
    // Gram: 2 producer warps split sub-chunks of kSub rows into a second
    // buffer while kTiles x kKsplit consumer warps accumulate the levels of
    // the lower-triangle 16x16 tiles; a tile's K range (the sub-chunks) is
    // dealt over kKsplit warps.  One partial per kGramRowsSplit rows.  At
    // most 12 warps: registers are split over the 4 SM sub-partitions.
    static constexpr int kTiles = (BB / 16) * (BB / 16 + 1) / 2;       // 1, 3, 10
    static constexpr int kKsplit = BB == 64 ? 1 : (BB == 32 ? 2 : 4);
    static constexpr int kGCons = kTiles * kKsplit;                    // consumer warps: 4, 6, 10
    static constexpr int kGThreads = 32 * (kGCons + 2);
    static constexpr int kSub = 32;
    static constexpr int kSubsPerChunk = kGramRowsSplit / kSub;        // 8
    static constexpr int kChunksPerCta = 4;
    static constexpr int kGLd = kSub + split::kPad;                    // 40
    static constexpr int kGSlice = BB * kGLd;
    static constexpr int kCPT = BB / 4;                                // columns per producer thread
    // update: 4 producer warps (load, exponents, digits) and 8 consumer warps
    // (one 16x16 output tile each, two per SM sub-partition) over
    // double-buffered blocks of kMB rows; every producer thread holds 16
    // entries of a block (one row, 16 columns)
    static constexpr int kCG = BB / 16;                                // column groups of 16
    static constexpr int kMB = 128 / kCG;                              // rows per block: 32, 64, 128
    static constexpr int kULd = BB + split::kPad;
    static constexpr int kUSliceA = kMB * kULd;
    static constexpr int kUSliceB = BB * kULd;
    static constexpr int kUpdProd = 4, kUpdCons = 8;
    static constexpr int kUpdWarps = kUpdProd + kUpdCons;
    static constexpr int kUpdRowsPerCta = 512;                         // rows of one update CTA
    static_assert((kMB / 16) * (BB / 16) == kUpdCons, "one tile per consumer warp");
};

template <int BB>
constexpr size_t gram_split_smem() {
    using S = SplitCfg<BB>;
    return 2u * 2 * split::kSlices * S::kGSlice + sizeof(int) * BB +
           sizeof(float) * (S::kKsplit - 1) * S::kTiles * split::kLevels * 8 * 32;
}
template <int BB>
constexpr size_t update_split_smem() {
    using S = SplitCfg<BB>;
    return 2u * split::kSlices * (2 * S::kUSliceA + S::kUSliceB) + sizeof(int) * (2 * BB + 2 * (S::kCG + 1) * S::kMB);
}

// Store the 9 digits of 4 consecutive K entries (one 8-byte store per slice).
static __device__ __forceinline__ void store_digits4(uint16_t *dst, int slice_stride, const unsigned long long (&z)[4]) {
#define JSVD_D4(I)                                                                                            \
    *reinterpret_cast<uint2 *>(dst + (I) * slice_stride) =                                                    \
        make_uint2(split::digit_pair<I>(z[0], z[1]), split::digit_pair<I>(z[2], z[3]));
    JSVD_D4(0) JSVD_D4(1) JSVD_D4(2) JSVD_D4(3) JSVD_D4(4) JSVD_D4(5) JSVD_D4(6) JSVD_D4(7) JSVD_D4(8)
#undef JSVD_D4
}

// Named barriers of the producer/consumer kernels (id 0 is __syncthreads).
namespace nb {
constexpr int kFull0 = 1, kEmpty0 = 3, kProd = 5, kCons = 6;   // 1-2 FULL, 3-4 EMPTY, 5 producers, 6 consumers
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

// ---------------------------------------------------------------------------
// Gram partials of rows [row0, row0 + nrows) of [G_P G_Q] (lower triangle,
// packed), one per 256 rows (the last may be shorter), written to
// part_pair[chunk0 + i]; nrows is a multiple of 32 (zero rows pad a matrix).
// Column c's scale is its exponent bound E_c = gexp_cols[c] (indexed by G's
// column); H(j, k) = 2^(E_j + E_k - 40) * combine(levels),
// the levels summed exactly over the 256 rows (each partial sum is below
// 9 * 256 * 64^2 < 2^24).
//
// Warps 0-1 produce: thread p takes rows 2 (p % 16), +1 of a 32-row
// sub-chunk and columns kCPT (p / 16) .. +kCPT-1, writes their digits to
// buffer s % 2 and arrives on FULL.  Consumer warp w owns tile w % kTiles for
// the sub-chunks s with s % kKsplit == w / kTiles; after a chunk's last
// sub-chunk the K parts are added through shared memory (consumers-only
// barrier) and part 0 combines and stores.
template <int BB>
__device__ __forceinline__ void gram_split_body(const double *__restrict__ G, int ldg, int P, int Q, int b,
                                                const int *__restrict__ gexp_cols, size_t row0, int nrows,
                                                double *__restrict__ part_pair, int chunk0,
                                                unsigned char *smem_raw) {
    using S = SplitCfg<BB>;
    constexpr int NT = S::kGThreads;
    constexpr int NP = 64;
    constexpr int NC = NT - NP;
    constexpr int CPT = S::kCPT;
    uint16_t *Dg = reinterpret_cast<uint16_t *>(smem_raw);                       // [2][kSlices][BB][kGLd]
    int *cexp = reinterpret_cast<int *>(Dg + 2 * split::kSlices * S::kGSlice);
    float *red = reinterpret_cast<float *>(cexp + BB);

    const int nsub = nrows / S::kSub;

    for (int c = threadIdx.x; c < BB; c += NT) {
        const int e = gexp_cols[block_col(P, Q, b, c)];
        cexp[c] = e == split::kNoExp ? 0 : e;
    }
    __syncthreads();

    if (threadIdx.x < NP) {
        // ---------------- producers ----------------
        const int p = threadIdx.x;
        const int rp = p & 15, cg = p >> 4;
        const double *src[CPT];
        int E[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            src[c] = G + (size_t)block_col(P, Q, b, cg * CPT + c) * ldg + row0 + 2 * rp;
            E[c] = cexp[cg * CPT + c];
        }
        double2 x[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) x[c] = *reinterpret_cast<const double2 *>(src[c]);
        for (int t = 0; t < nsub; ++t) {
            const int buf = t & 1;
            if (t >= 2) bar_sync_buf<nb::kEmpty0, NT>(buf);
            uint16_t *dst = Dg + (size_t)buf * split::kSlices * S::kGSlice + (cg * CPT) * S::kGLd + 2 * rp;
            // column by column: digits of this sub-chunk, then the next
            // sub-chunk's entries of the column are requested
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const unsigned long long z0 = split::fixed_biased(x[c].x, 0, E[c]);
                const unsigned long long z1 = split::fixed_biased(x[c].y, 0, E[c]);
                if (t + 1 < nsub) x[c] = *reinterpret_cast<const double2 *>(src[c] + (size_t)(t + 1) * S::kSub);
#define JSVD_G2(I)                                                                                  \
    *reinterpret_cast<uint32_t *>(dst + (I) * S::kGSlice + c * S::kGLd) =                           \
        split::digit_pair<I>(z0, z1);
                JSVD_G2(0) JSVD_G2(1) JSVD_G2(2) JSVD_G2(3) JSVD_G2(4) JSVD_G2(5) JSVD_G2(6) JSVD_G2(7) JSVD_G2(8)
#undef JSVD_G2
            }
            bar_arrive_buf<nb::kFull0, NT>(buf);
        }
    } else {
        // ---------------- consumers ----------------
        const int w = (threadIdx.x - NP) >> 5;
        const int lane = threadIdx.x & 31;
        const int t_ = w % S::kTiles, kpart = w / S::kTiles;
        int I = 0;
        while ((I + 1) * (I + 2) / 2 <= t_) ++I;
        const int J = t_ - I * (I + 1) / 2;
        float lev[split::kLevels][8];
        split::zero_levels(lev);
        for (int t = 0; t < nsub; ++t) {
            const int buf = t & 1;
            const int sub = t % S::kSubsPerChunk;
            bar_sync_buf<nb::kFull0, NT>(buf);
            if (sub % S::kKsplit == kpart) {
                const uint16_t *D = Dg + (size_t)buf * split::kSlices * S::kGSlice;
                split::tile_levels<S::kSub / 16>(D + I * 16 * S::kGLd, S::kGLd, S::kGSlice, D + J * 16 * S::kGLd,
                                                 S::kGLd, S::kGSlice, lev);
            }
            if (t + 2 < nsub) bar_arrive_buf<nb::kEmpty0, NT>(buf);
            if (sub == S::kSubsPerChunk - 1 || t == nsub - 1) {
                if constexpr (S::kKsplit > 1) {
                    // the K parts' level sums are exact integers: add them in part order
                    if (kpart > 0) {
                        float *mine = red + (((size_t)(kpart - 1) * S::kTiles + t_) * split::kLevels * 8) * 32 + lane;
#pragma unroll
                        for (int L = 0; L < split::kLevels; ++L)
#pragma unroll
                            for (int e = 0; e < 8; ++e) mine[(L * 8 + e) * 32] = lev[L][e];
                    }
                    bar_sync<nb::kCons, NC>();
                    if (kpart == 0) {
                        for (int q = 1; q < S::kKsplit; ++q) {
                            const float *src2 = red + (((size_t)(q - 1) * S::kTiles + t_) * split::kLevels * 8) * 32 + lane;
#pragma unroll
                            for (int L = 0; L < split::kLevels; ++L)
#pragma unroll
                                for (int e = 0; e < 8; ++e) lev[L][e] += src2[(L * 8 + e) * 32];
                        }
                    }
                    bar_sync<nb::kCons, NC>();
                }
                if (kpart == 0) {
                    const int chunk = chunk0 + t / S::kSubsPerChunk;
                    double *out = part_pair + (size_t)chunk * Cfg<BB>::kPacked;
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
                split::zero_levels(lev);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Rows [rbeg, rbeg + nrows) of [X_P X_Q] := [X_P X_Q] V' on split digits.
// With kRagged the last row block may be partial (its missing rows are read as
// zero and not written); without it nrows is a multiple of kMB.  For G the A operand is G D^-1 (D = 2^dexp_src, from the
// pair's Gram diagonal) against the digits of D V'; for V (dexp_src = null)
// it is V against those of V'.  bsl_pv, fexp_src: the right factor's digits
// and column exponents.  Row r of a block gets the exponent bound E_r of its
// BB entries; X(r, k) = 2^(E_r + F_k - 40) * combine(levels).  With
// gexp_cols != null the exponent bounds of the written values are max-reduced
// into gexp_cols[column of X].
//
// Warps 0-3 produce: load block t (thread p: row p % kMB, columns
// 16 (p / kMB) .. +15), reduce the row exponents, write the digits to buffer
// t % 2, and arrive on FULL(t % 2).  Warps 4-11 consume: wait on FULL, run
// the level MMAs of their tile, read the tile rows' exponents, arrive on
// EMPTY (which the producers wait on before refilling that buffer two blocks
// later), then combine and store.  Named barriers with matched counts: every
// producer and consumer thread runs the same number of blocks.
template <int BB, bool kRagged>
__device__ __forceinline__ void update_split_body(double *__restrict__ X, int ld, size_t rbeg, int nrows, int P,
                                                  int Q, int b, const uint16_t *__restrict__ bsl_pv,
                                                  const int *__restrict__ fexp_src,
                                                  const int *__restrict__ dexp_src, int *__restrict__ gexp_cols,
                                                  unsigned char *smem_raw) {
    using S = SplitCfg<BB>;
    constexpr int MB = S::kMB;
    constexpr int CG = S::kCG;
    constexpr int NT = 32 * S::kUpdWarps;             // 384
    constexpr int NP = 32 * S::kUpdProd;               // producer threads
    uint16_t *As = reinterpret_cast<uint16_t *>(smem_raw);                 // [2][kSlices][MB][kULd]
    uint16_t *Bs = As + 2 * split::kSlices * S::kUSliceA;                   // [kSlices][BB][kULd]
    int *fexp = reinterpret_cast<int *>(Bs + split::kSlices * S::kUSliceB);
    int *dexp = fexp + BB;
    int *rmax = dexp + BB;                // [2][CG][MB]
    int *rexp = rmax + 2 * CG * MB;       // [2][MB]

    const int nblk = (nrows + MB - 1) / MB;

    // right factor digits and exponents of this pair and version
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(bsl_pv);
        uint4 *dst = reinterpret_cast<uint4 *>(Bs);
        for (int e = threadIdx.x; e < split_b_elems<BB>() / 8; e += NT) dst[e] = src[e];
        for (int k = threadIdx.x; k < BB; k += NT) {
            fexp[k] = fexp_src[k];
            dexp[k] = dexp_src ? dexp_src[k] : 0;
        }
    }
    __syncthreads();

    if (threadIdx.x < NP) {
        // ---------------- producers ----------------
        const int p = threadIdx.x;
        const int r = p % MB, cg = p / MB;
        const double *src0 = X + rbeg + r;
        size_t coff[16];
        int dx[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            coff[c] = (size_t)block_col(P, Q, b, 16 * cg + c) * ld;
            dx[c] = dexp[16 * cg + c];
        }
        double x[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) x[c] = (!kRagged || r < nrows) ? src0[coff[c]] : 0.0;
        for (int t = 0; t < nblk; ++t) {
            const int buf = t & 1;
            int m = split::kNoExp;
#pragma unroll
            for (int c = 0; c < 16; ++c) m = max(m, split::exp_bound(x[c], -dx[c]));
            rmax[(buf * CG + cg) * MB + r] = m;
            bar_sync<nb::kProd, NP>();
            int E = split::kNoExp;
#pragma unroll
            for (int g = 0; g < CG; ++g) E = max(E, rmax[(buf * CG + g) * MB + r]);
            if (E == split::kNoExp) E = 0;
            if (t >= 2) bar_sync_buf<nb::kEmpty0, NT>(buf);   // consumers are done with block t - 2
            if (cg == 0) rexp[buf * MB + r] = E;
            uint16_t *dst = As + (size_t)buf * split::kSlices * S::kUSliceA + r * S::kULd + 16 * cg;
            // four columns at a time: digits of this block, then the next
            // block's entries of those columns are requested
#pragma unroll
            for (int c = 0; c < 16; c += 4) {
                const unsigned long long z[4] = {split::fixed_biased(x[c], -dx[c], E),
                                                 split::fixed_biased(x[c + 1], -dx[c + 1], E),
                                                 split::fixed_biased(x[c + 2], -dx[c + 2], E),
                                                 split::fixed_biased(x[c + 3], -dx[c + 3], E)};
                if (t + 1 < nblk) {
                    const bool in = !kRagged || (t + 1) * MB + r < nrows;
#pragma unroll
                    for (int u = 0; u < 4; ++u) x[c + u] = in ? src0[coff[c + u] + (size_t)(t + 1) * MB] : 0.0;
                }
                store_digits4(dst + c, S::kUSliceA, z);
            }
            bar_arrive_buf<nb::kFull0, NT>(buf);
        }
    } else {
        // ---------------- consumers ----------------
        const int cw = (threadIdx.x - NP) >> 5;        // 0..7: tile
        constexpr int TN = BB / 16;
        const int tm = cw / TN, tn = cw % TN;
        int gcol[8];
        int fx[8];
        // exponent bounds of the written values per column (G only): columns
        // of accumulators e = 0, 1, 4, 5
        const bool track = gexp_cols != nullptr;
        int cm[4] = {split::kNoExp, split::kNoExp, split::kNoExp, split::kNoExp};
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int col = tn * 16 + split::acc_col(e);
            gcol[e] = block_col(P, Q, b, col);
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
                if (kRagged && t * MB + row >= nrows) continue;
                const double y = split::combine<true>(lv, (e & 2) ? e1 : e0, fx[e]);
                X[(size_t)gcol[e] * ld + rb + row] = y;
                if (track) {
                    const int ci = (e & 1) + ((e & 4) >> 1);
                    cm[ci] = max(cm[ci], split::exp_bound(y, 0));
                }
            }
        }
        if (track) {
            // lanes with the same lane % 4 hold the same columns
#pragma unroll
            for (int ci = 0; ci < 4; ++ci)
#pragma unroll
                for (int o = 4; o < 32; o <<= 1) cm[ci] = max(cm[ci], __shfl_xor_sync(0xffffffffu, cm[ci], o));
            if ((threadIdx.x & 31) < 4) {
                atomicMax(&gexp_cols[gcol[0]], cm[0]);
                atomicMax(&gexp_cols[gcol[1]], cm[1]);
                atomicMax(&gexp_cols[gcol[4]], cm[2]);
                atomicMax(&gexp_cols[gcol[5]], cm[3]);
            }
        }
    }
}

}  // namespace jsvd
