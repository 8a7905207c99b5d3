// Device-side building blocks of one block p-step (Sec. 2, Sec. 4 of the
// paper), shared by the single-matrix kernels (sweep_fp64.cu) and the batched
// kernels (batched.cu).  Each function is executed by a whole CTA and handles
// one unit of work:
//   gram_unit    the lower triangle of [G_P G_Q]^T [G_P G_Q] over one chunk
//                of rows (Eq. (2.7), split over rows)
//   jacobi_unit  sum of the chunk partials, Cholesky (Sec. 4.1), M_s inner
//                sweeps (Sec. 4.3) accumulated into V' (one sweep: R side and
//                V' side on separate thread groups), counters, and for the
//                tensor-core contractions the split right factors
//   update_unit  one chunk of rows of [A_P A_Q] := [A_P A_Q] V' (Eq. (2.9))
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "cluster_sync.cuh"
#include "rotation.cuh"
#include "split8.cuh"
#include "split_mma.cuh"

namespace jsvd {

enum {
    kCntRot = 0,       // rotations (rho = 1)
    kCntProper = 1,    // proper rotations (cs != 1)
    kCntUpdated = 2,   // block pairs with V' != I
    kCntBreak = 3,     // Cholesky breakdowns
    kCntOff = 4,       // max normalized off-diagonal |h_ij|/sqrt(h_ii h_jj), double bits
    kCntErr = 5,       // device-side error flags
    kCntInner = 6,     // inner sweeps performed, summed over the pivot pairs
    kCntNormExp = 7,   // at set-up: max over the columns of the DRDSSQ exponent + 8192
    kCntSize = 8
};

constexpr int kGramRows = 128;     // rows of [G_P G_Q] per Gram unit
constexpr int kGramRowsSplit = 256;   // rows per Gram partial of the split form
constexpr int kUpdThreads = 256;   // 4x4 output tiles per thread

template <int BB> struct Cfg {
    static constexpr int kPairsInner = BB / 2;
    // 128 threads for every BB: one warp per SM sub-partition (each has its
    // own FP64 unit), with the fewest lanes per inner pair that fill them
    static constexpr int kLanesPerPair = 256 / BB;
    static constexpr int kJacThreads = kPairsInner * kLanesPerPair;   // 128
    static constexpr int kRowsPerLane = BB / kLanesPerPair;
    static constexpr int kLd = BB + 1;                                // smem ld for R, V'
    static constexpr int kPacked = BB * (BB + 1) / 2;
    static constexpr int kUpdRows = 4096 / BB;                        // rows per update unit
    static constexpr int kGramLd = BB + 2;                            // smem row stride
    // Gram: NBLK 2x2 blocks of the lower triangle; each block's rows are split
    // over kGramSplit thread groups so that every thread has a block
    static constexpr int kGramBlocks = (BB / 2) * (BB / 2 + 1) / 2;   // 36, 136, 528
    static constexpr int kGramSplit = BB == 16 ? 7 : (BB == 32 ? 2 : 1);
    static constexpr int kGramThreads = BB == 32 ? 288 : 256;
};

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

template <int BB, typename T>
constexpr size_t gram_smem_bytes() {
    return sizeof(T) * kGramRows * Cfg<BB>::kGramLd +
           (Cfg<BB>::kGramSplit > 1 ? sizeof(T) * 4 * Cfg<BB>::kGramSplit * Cfg<BB>::kGramBlocks : 0);
}
template <int BB>
constexpr size_t jacobi_smem_bytes() {
    // A, B; the Gram diagonal; the column-scale exponents; the inner table
    return sizeof(double) * (2 * BB * Cfg<BB>::kLd + BB) + sizeof(int) * BB + (BB - 1) * BB + 16;
}

// Shared-memory / global image of the split digits of a BB x BB right factor
// (one version): [kSlices][BB rows n][BB + kPad] bf16, K contiguous.
template <int BB>
constexpr int split_b_elems() { return split::kSlices * BB * (BB + split::kPad); }
template <int BB, typename T>
constexpr size_t update_smem_bytes() { return sizeof(T) * (BB * Cfg<BB>::kUpdRows + BB * (BB + 2)); }

__device__ __forceinline__ int block_col(int P, int Q, int b, int j) {
    return j < b ? P * b + j : Q * b + (j - b);
}

// Index of (i, j), i >= j, in the column-major packed lower triangle of order BB.
template <int BB>
__device__ __forceinline__ int packed_lower(int i, int j) {
    return j * BB - (j * (j - 1)) / 2 + (i - j);
}

// ---------------------------------------------------------------------------
// Gram partial of rows [r0, r0 + valid) (valid <= kGramRows).  The chunk is
// staged row-major in shared memory (row stride BB+2) so that every thread
// reads 2x2 operand blocks with vector loads.  The 2x2 blocks (I, J), I >= J,
// of the lower triangle are spread over the threads; with kGramSplit > 1 the
// rows of a block are split over that many thread groups (group g takes rows
// g, g + split, ...) and the group sums are added in group order.  Each
// partial sum runs over its rows in increasing order.  The result (double)
// goes to out[packed index].
template <int BB, typename T>
__device__ __forceinline__ void gram_unit(const T *__restrict__ G, int ldg, int r0, int valid, int P,
                                          int Q, int b, double *__restrict__ out, T *X) {
    using C = Cfg<BB>;
    using T2 = typename Vec2<T>::type;
    constexpr int NBLK = C::kGramBlocks;
    constexpr int SPLIT = C::kGramSplit;
    for (int e = threadIdx.x; e < kGramRows * BB; e += C::kGramThreads) {
        const int r = e % kGramRows, j = e / kGramRows;
        if (r < valid) X[r * C::kGramLd + j] = G[(size_t)block_col(P, Q, b, j) * ldg + r0 + r];
    }
    __syncthreads();
    T *red = X + kGramRows * C::kGramLd;   // [SPLIT][NBLK][4] when SPLIT > 1
    for (int task = threadIdx.x; task < NBLK * SPLIT; task += C::kGramThreads) {
        const int blk = task % NBLK, grp = task / NBLK;
        int I = (int)((sqrtf(8.0f * blk + 1.0f) - 1.0f) * 0.5f);
        while ((I + 1) * (I + 2) / 2 <= blk) ++I;
        while (I * (I + 1) / 2 > blk) --I;
        const int J = blk - I * (I + 1) / 2;
        T h00 = 0, h10 = 0, h01 = 0, h11 = 0;
        const T *xi = X + 2 * I, *xj = X + 2 * J;
#pragma unroll 4
        for (int r = grp; r < valid; r += SPLIT) {
            const T2 u = *reinterpret_cast<const T2 *>(xi + r * C::kGramLd);
            const T2 v = *reinterpret_cast<const T2 *>(xj + r * C::kGramLd);
            h00 = fma(u.x, v.x, h00);
            h10 = fma(u.y, v.x, h10);
            h01 = fma(u.x, v.y, h01);
            h11 = fma(u.y, v.y, h11);
        }
        if (SPLIT > 1) {
            T *dst = red + 4 * (grp * NBLK + blk);
            dst[0] = h00; dst[1] = h10; dst[2] = h01; dst[3] = h11;
        } else {
            const int i0 = 2 * I, j0 = 2 * J;
            out[packed_lower<BB>(i0, j0)] = (double)h00;
            out[packed_lower<BB>(i0 + 1, j0)] = (double)h10;
            out[packed_lower<BB>(i0 + 1, j0 + 1)] = (double)h11;
            if (I != J) out[packed_lower<BB>(i0, j0 + 1)] = (double)h01;
        }
    }
    if (SPLIT > 1) {
        __syncthreads();
        for (int t = threadIdx.x; t < NBLK * 4; t += C::kGramThreads) {
            const int blk = t / 4, c = t % 4;
            T acc = red[4 * blk + c];
            for (int g = 1; g < SPLIT; ++g) acc += red[4 * (g * NBLK + blk) + c];
            int I = (int)((sqrtf(8.0f * blk + 1.0f) - 1.0f) * 0.5f);
            while ((I + 1) * (I + 2) / 2 <= blk) ++I;
            while (I * (I + 1) / 2 > blk) --I;
            const int J = blk - I * (I + 1) / 2;
            const int i = 2 * I + (c & 1), j = 2 * J + (c >> 1);
            if (i >= j) out[packed_lower<BB>(i, j)] = (double)acc;
        }
    }
}

// ---------------------------------------------------------------------------
// Split digits of the right factors of one pivot pair for the tensor-core
// update (see split_mma.cuh): version 0 = D V' for [G_P G_Q] with
// D = diag(2^dexp[j]), 2^dexp[j] ~ sqrt(h_jj) (exact powers of two, so
// G V' = (G D^-1)(D V')), version 1 = V' for [V_P V_Q].  W is V' in shared
// memory (column-major, ld BB+1).  Column k of a version gets the exponent
// bound F_k of its entries and the digits of trunc(x 2^(62-F_k)), stored as
// out[slice][k][j] (K = j contiguous, row stride BB + kPad).
//
// With tc the images are those of the tcgen05 update instead: 8 balanced
// 8-bit digits in its operand layout (split8::right_factor_image).
template <int BB, int NT = Cfg<BB>::kJacThreads>
__device__ __forceinline__ void split_right_factor(const double *W, const double *hdiag, int *dx,
                                                   uint16_t *__restrict__ out, int *__restrict__ bexp,
                                                   int *__restrict__ dexp, bool tc = false) {
    using C = Cfg<BB>;
    constexpr int LD = BB + split::kPad;
    for (int j = threadIdx.x; j < BB; j += NT) {
        const double h = hdiag[j];
        const int d = h > 0.0 ? (split::exp_of(h) >> 1) : 0;
        dx[j] = d;
        dexp[j] = d;
    }
    __syncthreads();
    if (tc) {
        split8::right_factor_image<BB, NT>(W, C::kLd, dx, out, bexp);
        return;
    }
    for (int t = threadIdx.x; t < 2 * BB; t += NT) {
        const int ver = t / BB, k = t % BB;
        const double *w = W + k * C::kLd;
        int F = split::kNoExp;
        for (int j = 0; j < BB; ++j) F = max(F, split::exp_bound(w[j], ver ? 0 : dx[j]));
        if (F == split::kNoExp) F = 0;
        bexp[ver * BB + k] = F;
        uint16_t *o = out + (size_t)ver * split_b_elems<BB>() + k * LD;
        for (int j = 0; j < BB; j += 2) {
            const unsigned long long z0 = split::fixed_biased(w[j], ver ? 0 : dx[j], F);
            const unsigned long long z1 = split::fixed_biased(w[j + 1], ver ? 0 : dx[j + 1], F);
#define JSVD_SPLIT_STORE(I) \
    *reinterpret_cast<uint32_t *>(o + (I) * BB * LD + j) = \
        split::digit_pair<I>(z0, z1);
            JSVD_SPLIT_STORE(0) JSVD_SPLIT_STORE(1) JSVD_SPLIT_STORE(2) JSVD_SPLIT_STORE(3) JSVD_SPLIT_STORE(4)
            JSVD_SPLIT_STORE(5) JSVD_SPLIT_STORE(6) JSVD_SPLIT_STORE(7) JSVD_SPLIT_STORE(8)
#undef JSVD_SPLIT_STORE
        }
    }
}

// ---------------------------------------------------------------------------
// One inner sweep (block-oriented variant) with 2 kJacThreads threads: the
// first half (R side) forms each inner p-step's dot products on R, the
// relative test, the rotations (Eqs. (4.3)-(4.6)) and the P2 sort decision,
// publishes them in one of two parameter slots and rotates R; the second half
// (V' side) rotates V' with the published parameters one step behind (V'
// does not feed the next dot products).  Both halves do each element's
// arithmetic exactly as the single-group sweep does, so R and V' are the
// same bit for bit; the V' side's FP64 work fills the FP64 pipe while the R
// side waits on its latency chains.  Named barriers: FULL (slot filled,
// R side arrives, V' side waits), EMPTY (slot read, V' side arrives, R side
// waits before refilling it two steps later), one per side per step.
namespace jb {
constexpr int kFull0 = 1, kEmpty0 = 3, kRSide = 5, kVSide = 6;
}
template <int ID, int COUNT>
__device__ __forceinline__ void nbar_sync() {
    asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(COUNT) : "memory");
}
template <int ID, int COUNT>
__device__ __forceinline__ void nbar_arrive() {
    asm volatile("bar.arrive %0, %1;" ::"n"(ID), "n"(COUNT) : "memory");
}

// Element arithmetic of the inner sweep in the type RT of R and V': FP64, or
// FP32 in the first stage of the mixed solver, whose rotations (Eqs.
// (4.3)-(4.6), relative test with eps = 2^-24) are then FP32 as well.
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double add_t(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_t(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double mul_t(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_t(float a, float b) { return __fmul_rn(a, b); }

// Eq. (4.1) / (4.2) on one row in RT: the FMA form of rot_apply with cs, tn
// given in RT; `proper` is cs != 1 of the FP64 parameters.
template <typename RT>
__device__ __forceinline__ void rot_apply_t(RT &x, RT &y, bool hyperbolic, RT cs, RT tn, bool proper) {
    const RT xn = fma_t(hyperbolic ? tn : -tn, y, x);
    const RT yn = fma_t(tn, x, y);
    if (proper) {
        x = mul_t(cs, xn);
        y = mul_t(cs, yn);
    } else {
        x = xn;
        y = yn;
    }
}

//
// CLUSTER: the CTA of rank 0 of a 2-CTA cluster runs the R side, the CTA of
// rank 1 (another SM) the V' side (without: both sides in this CTA): the
// R side stores each step's parameters into the peer's slots (distributed
// shared memory) and arrives on the peer's mbarrier full[slot]; the V' side
// waits on it and, once it has read the slot, arrives on the R side's
// empty[slot].  Same arithmetic, so the same R and V' bit for bit.  Waits are
// bounded (~2 s); one that gives up raises the error flag in *err.
template <int BB, typename RT = double, bool CLUSTER = false>
__device__ __forceinline__ void jacobi_sweep_pipelined(RT *A, RT *B, const unsigned char *tab, int P, int Q,
                                                       int b, int nplus, int bord_lo, int bord_hi, double c_eps,
                                                       double c_eps2,
                                                       int &my_rot, int &my_proper, int &changed,
                                                       uint64_t *full = nullptr, uint64_t *empty = nullptr,
                                                       unsigned long long *err = nullptr) {
    using C = Cfg<BB>;
    constexpr int NH = C::kJacThreads;        // threads per side
    constexpr int NT = 2 * NH;
    constexpr int NP = BB / 2;                // pairs per inner step
    __shared__ double s_cs[2][NP], s_tn[2][NP];
    __shared__ int s_fl[2][NP];               // bit 0: rotate, 1: swap, 2: hyperbolic, 3: cs != 1
    const int tid = threadIdx.x;
    const int role = CLUSTER ? (int)cl::rank() : -1;
    bool dead = false;
    auto cwait = [&](uint64_t *bar, uint32_t parity) {
        if (dead) return;
        if (!cl::wait_parity(bar, parity, 2048)) {
            dead = true;
            atomicOr(err, 4ull);
        }
    };
    if (tid < NH && role != 1) {
        // ---------------- R side ----------------
        const int y = tid / C::kLanesPerPair;
        const int g = tid % C::kLanesPerPair;
        for (int st = 0; st < BB - 1; ++st) {
            const int slot = st & 1;
            const int p = tab[2 * (st * (BB / 2) + y)];
            const int q = tab[2 * (st * (BB / 2) + y) + 1];
            RT *rp = B + p * C::kLd, *rq = B + q * C::kLd;
            RT tpp = 0, tqq = 0, tpq = 0;
#pragma unroll
            for (int k = 0; k < C::kRowsPerLane; ++k) {
                const int r = g + k * C::kLanesPerPair;
                const RT x = rp[r], z = rq[r];
                tpp = fma_t(x, x, tpp);
                tqq = fma_t(z, z, tqq);
                tpq = fma_t(x, z, tpq);
            }
#pragma unroll
            for (int off = C::kLanesPerPair / 2; off > 0; off >>= 1) {
                tpp = add_t(tpp, __shfl_xor_sync(0xffffffffu, tpp, off));
                tqq = add_t(tqq, __shfl_xor_sync(0xffffffffu, tqq, off));
                tpq = add_t(tpq, __shfl_xor_sync(0xffffffffu, tpq, off));
            }
            const int gp = block_col(P, Q, b, p), gq = block_col(P, Q, b, q);
            const bool hyp = gp < nplus && gq >= nplus;
            const bool border = (gp >= bord_lo && gp < bord_hi) || (gq >= bord_lo && gq < bord_hi);
            bool rho, swap = false, proper;
            RT cs_t, tn_t;
            Rot rot{1.0, 0.0};
            if constexpr (sizeof(RT) == sizeof(double)) {
                const double hpp = tpp, hqq = tqq, hpq = tpq;
                rho = !border && needs_rotation(hpp, hqq, hpq, c_eps, c_eps2);
                if (rho) rot = rot_params(hpp, hqq, hpq, hyp);
                if (!hyp && !border) {
                    const double npp = rho ? __fma_rn(-rot.tn, hpq, hpp) : hpp;
                    const double nqq = rho ? __fma_rn(rot.tn, hpq, hqq) : hqq;
                    swap = (gq < nplus && npp < nqq) || (gp >= nplus && npp > nqq);
                }
                cs_t = (RT)rot.cs;
                tn_t = (RT)rot.tn;
                proper = is_proper(rot);
            } else {
                // FP32 sweeps: the rotation itself in FP32 (rotation.cuh)
                RotF rf{1.0f, 0.0f};
                rho = !border && needs_rotation_f(tpp, tqq, tpq, (float)c_eps);
                if (rho) rf = rot_params_f(tpp, tqq, tpq, hyp);
                if (!hyp && !border) {
                    const float npp = rho ? __fmaf_rn(-rf.tn, tpq, tpp) : tpp;
                    const float nqq = rho ? __fmaf_rn(rf.tn, tpq, tqq) : tqq;
                    swap = (gq < nplus && npp < nqq) || (gp >= nplus && npp > nqq);
                }
                cs_t = rf.cs;
                tn_t = rf.tn;
                proper = rf.cs != 1.0f;
                rot = Rot{(double)rf.cs, (double)rf.tn};
            }
            const int flags = (rho ? 1 : 0) | (swap ? 2 : 0) | (hyp ? 4 : 0) | (proper ? 8 : 0);
            if constexpr (!CLUSTER) {
                if (st >= 2) {
                    if (slot) nbar_sync<jb::kEmpty0 + 1, NT>(); else nbar_sync<jb::kEmpty0, NT>();
                }
                if (g == 0) {
                    s_cs[slot][y] = rot.cs;
                    s_tn[slot][y] = rot.tn;
                    s_fl[slot][y] = flags;
                }
                if (slot) nbar_arrive<jb::kFull0 + 1, NT>(); else nbar_arrive<jb::kFull0, NT>();
            } else {
                if (st >= 2) cwait(&empty[slot], (uint32_t)(((st >> 1) - 1) & 1));
                if (g == 0 && !dead) {
                    cl::st_f64(cl::peer_addr(&s_cs[slot][y], 1), rot.cs);
                    cl::st_f64(cl::peer_addr(&s_tn[slot][y], 1), rot.tn);
                    cl::st_s32(cl::peer_addr(&s_fl[slot][y], 1), flags);
                    cl::arrive_remote(cl::peer_addr(&full[slot], 1));
                }
            }
            if (rho || swap) {
#pragma unroll
                for (int k = 0; k < C::kRowsPerLane; ++k) {
                    const int r = g + k * C::kLanesPerPair;
                    RT x = rp[r], z = rq[r];
                    if (rho) rot_apply_t(x, z, hyp, cs_t, tn_t, proper);
                    if (swap) {
                        rp[r] = z; rq[r] = x;
                    } else {
                        rp[r] = x; rq[r] = z;
                    }
                }
                changed = 1;
            }
            if (g == 0 && rho) {
                ++my_rot;
                if (proper) ++my_proper;
            }
            nbar_sync<jb::kRSide, NH>();
        }
    } else if (tid >= NH && role != 0) {
        // ---------------- V' side ----------------
        const int v = tid - NH;
        const int y = v / C::kLanesPerPair;
        const int g = v % C::kLanesPerPair;
        for (int st = 0; st < BB - 1; ++st) {
            const int slot = st & 1;
            const int p = tab[2 * (st * (BB / 2) + y)];
            const int q = tab[2 * (st * (BB / 2) + y) + 1];
            if constexpr (!CLUSTER) {
                if (slot) nbar_sync<jb::kFull0 + 1, NT>(); else nbar_sync<jb::kFull0, NT>();
            } else {
                cwait(&full[slot], (uint32_t)((st >> 1) & 1));
            }
            const double cs = s_cs[slot][y], tn = s_tn[slot][y];
            const int fl = dead ? 0 : s_fl[slot][y];
            if (st + 2 < BB - 1) {
                if constexpr (!CLUSTER) {
                    if (slot) nbar_arrive<jb::kEmpty0 + 1, NT>(); else nbar_arrive<jb::kEmpty0, NT>();
                } else {
                    __syncwarp();
                    if ((tid & 31) == 0 && !dead) cl::arrive_remote(cl::peer_addr(&empty[slot], 0));
                }
            }
            const bool rho = fl & 1, swap = fl & 2, hyp = fl & 4, proper = fl & 8;
            if (role == 1 && (rho || swap)) changed = 1;
            const RT cs_t = (RT)cs, tn_t = (RT)tn;
            RT *wp = A + p * C::kLd, *wq = A + q * C::kLd;
            if (rho || swap) {
#pragma unroll
                for (int k = 0; k < C::kRowsPerLane; ++k) {
                    const int r = g + k * C::kLanesPerPair;
                    RT u = wp[r], w = wq[r];
                    if (rho) rot_apply_t(u, w, hyp, cs_t, tn_t, proper);
                    if (swap) {
                        wp[r] = w; wq[r] = u;
                    } else {
                        wp[r] = u; wq[r] = w;
                    }
                }
            }
            nbar_sync<jb::kVSide, NH>();
        }
    }
}

// ---------------------------------------------------------------------------
// Per-pair factorization and inner sweeps; executed by Cfg<BB>::kJacThreads
// threads.  smem: A and B, each BB x BB column-major with ld BB+1, then the
// inner table ((BB-1) x BB/2 pairs of bytes).
//   A: H (lower) -> L by Cholesky -> V' (= I, then rotated)
//   B: R = L^T (upper), rotated in the inner sweeps
// Inner p-step: pair y of the inner table is handled by the lane group y
// (256/BB lanes); lane g of the group owns rows g, g + 256/BB, ... of both
// columns in R and V'.
// Writes V' (column-major, BB x BB) to vp and "V' != I" to *vflag; adds the
// rotation counts to counters[].  With bsl != null (tensor-core contractions)
// it also writes, for the update of G, the column scales D = 2^dexp[j] with
// 2^dexp[j] ~ ||g_j|| (from the Gram diagonal) and the split digits of D V',
// and for the update of V those of V' (bsl + split_b_elems, bexp + BB); bexp
// holds each column's exponent bound.  With gexp != null the exponent bounds
// of the pair's columns of G are reset (the split update recomputes them).  Global columns in [bord_lo, bord_hi) are the
// identity border: they are exactly orthogonal to everything, and they are
// neither rotated nor swapped, so they keep their positions.
template <int BB, int NT = Cfg<BB>::kJacThreads, typename RT = double, bool CLUSTER = false>
__device__ __forceinline__ void jacobi_unit(const double *__restrict__ part, int chunks,
                                            const unsigned char *__restrict__ inner, int P, int Q, int b,
                                            int nplus, int bord_lo, int bord_hi, int inner_sweeps, double eps,
                                            double *__restrict__ vp,
                                            int *__restrict__ vflag, unsigned long long *__restrict__ counters,
                                            double *smem, uint16_t *__restrict__ bsl = nullptr,
                                            int *__restrict__ bexp = nullptr, int *__restrict__ dexp = nullptr,
                                            int *__restrict__ gexp = nullptr, bool tc = false) {
    using C = Cfg<BB>;
    double *A = smem;
    double *B = smem + BB * C::kLd;
    double *hdiag = smem + 2 * BB * C::kLd;
    int *dx = reinterpret_cast<int *>(hdiag + BB);
    unsigned char *tab = reinterpret_cast<unsigned char *>(dx + BB);
    __shared__ double s_piv;
    __shared__ int s_brk;
    __shared__ unsigned long long s_off;
    __shared__ int s_cnt[2];

    const int tid = threadIdx.x;
    for (int e = tid; e < (BB - 1) * BB; e += NT) tab[e] = inner[e];
    if (tid == 0) { s_off = 0ull; s_brk = 0; s_cnt[0] = 0; s_cnt[1] = 0; }
    // CLUSTER: a 2-CTA cluster per pivot pair, CTA 0 the factorization and
    // the R side of the inner sweep, CTA 1 the V' side and the V' outputs
    const int role = CLUSTER ? (int)cl::rank() : -1;
    __shared__ uint64_t s_full[2], s_empty[2];
    if constexpr (CLUSTER) {
        if (tid == 0) {
            for (int i = 0; i < 2; ++i) {
                tc::mbar_init(&s_full[i], BB / 2);
                tc::mbar_init(&s_empty[i], C::kJacThreads / 32);
            }
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        cl::sync();
    }

    if (role != 1) {
        // (1) H = sum of the row-chunk partials in a fixed order: chunk c goes to
        // accumulator c mod 8 (in increasing c), then the 8 accumulators are added
        // pairwise; short dependency chains keep the FP64 latency off the path
        for (int e = tid; e < BB * BB; e += NT) {
            const int i = e % BB, j = e / BB;
            if (i < j) continue;
            const int k = packed_lower<BB>(i, j);
            double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            int c = 0;
            for (; c + 8 <= chunks; c += 8) {
    #pragma unroll
                for (int u = 0; u < 8; ++u) acc[u] = __dadd_rn(acc[u], part[(size_t)(c + u) * C::kPacked + k]);
            }
    #pragma unroll
            for (int u = 0; u < 8; ++u)
                if (c + u < chunks) acc[u] = __dadd_rn(acc[u], part[(size_t)(c + u) * C::kPacked + k]);
            A[i + j * C::kLd] = __dadd_rn(__dadd_rn(__dadd_rn(acc[0], acc[1]), __dadd_rn(acc[2], acc[3])),
                                          __dadd_rn(__dadd_rn(acc[4], acc[5]), __dadd_rn(acc[6], acc[7])));
        }
        __syncthreads();

        // (2) normalized off-diagonal maximum of H, max |h_ij| / sqrt(h_ii h_jj)
        // (reported only): B[j] = 1/sqrt(h_jj) first, then two products per entry
        for (int j = tid; j < BB; j += NT) {
            const double d = A[j + j * C::kLd];
            B[j] = d > 0.0 ? rsqrt(d) : 0.0;
            hdiag[j] = d;
            if (role == 0) cl::st_f64(cl::peer_addr(&hdiag[j], 1), d);
        }
        __syncthreads();
        {
            double mx = 0.0;
            for (int e = tid; e < BB * BB; e += NT) {
                const int i = e % BB, j = e / BB;
                if (i <= j) continue;
                mx = fmax(mx, fabs(A[i + j * C::kLd]) * B[i] * B[j]);
            }
            atomicMax(&s_off, (unsigned long long)__double_as_longlong(mx));
        }

        // (3) Cholesky H = L L^T without pivoting (Sec. 4.1), right-looking:
        // entry (i, j) receives -L(i,k) L(j,k) for k = 0, 1, ... in order, then the
        // division by the pivot.  A non-positive pivot zeroes its column.  The
        // pivot of column k + 1 is taken by thread 0, which performs that entry's
        // last update itself (e = 0 of the trailing update), right after it.
        auto pivot = [&](int k) {
            const double d = A[k + k * C::kLd];
            if (d > 0.0) {
                s_piv = __dsqrt_rn(d);
            } else {
                s_piv = 0.0;
                s_brk += 1;
            }
        };
        if (tid == 0) pivot(0);
        __syncthreads();
        for (int k = 0; k < BB; ++k) {
            const double piv = s_piv;
            for (int i = k + tid; i < BB; i += NT)
                A[i + k * C::kLd] = (piv > 0.0) ? (i == k ? piv : __ddiv_rn(A[i + k * C::kLd], piv)) : 0.0;
            __syncthreads();
            const int rem = BB - 1 - k;
            for (int e = tid; e < rem * rem; e += NT) {
                const int i = k + 1 + e % rem, j = k + 1 + e / rem;
                if (i >= j)
                    A[i + j * C::kLd] = __fma_rn(-A[i + k * C::kLd], A[j + k * C::kLd], A[i + j * C::kLd]);
            }
            if (tid == 0 && k + 1 < BB) pivot(k + 1);
            __syncthreads();
        }

    }
    // (4) R = L^T into B; V' = I into A (both in RT from here on)
    RT *Rt = reinterpret_cast<RT *>(B);
    RT *Vt = reinterpret_cast<RT *>(A);
    if (role != 1) {
        for (int e = tid; e < BB * BB; e += NT) {
            const int i = e % BB, j = e / BB;
            Rt[i + j * C::kLd] = (i <= j) ? (RT)A[j + i * C::kLd] : (RT)0;
        }
    }
    __syncthreads();
    for (int e = tid; e < BB * BB; e += NT) {
        const int i = e % BB, j = e / BB;
        Vt[i + j * C::kLd] = (i == j) ? (RT)1 : (RT)0;
    }
    __syncthreads();

    // (5) inner sweeps of the pointwise one-sided method on R (Sec. 4.3)
    const double c_eps = eps * sqrt((double)BB);   // c(eps) = eps sqrt(nhat), nhat = BB
    const double c_eps2 = __dmul_rn(c_eps, c_eps);
    int my_rot = 0, my_proper = 0, changed = 0, sweeps_done = 0;
    if constexpr (NT == 2 * C::kJacThreads) {
        // one inner sweep, V' rotated one step behind R by the second half of
        // the threads
        jacobi_sweep_pipelined<BB, RT, CLUSTER>(Vt, Rt, tab, P, Q, b, nplus, bord_lo, bord_hi, c_eps, c_eps2, my_rot,
                                             my_proper,
                                       changed, s_full, s_empty, &counters[kCntErr]);
        sweeps_done = 1;
    } else {
    static_assert(NT == C::kJacThreads && sizeof(RT) == sizeof(double), "thread count, FP64 inner sweep");
    const int y = tid / C::kLanesPerPair;
    const int g = tid % C::kLanesPerPair;
    for (int sw = 0; sw < inner_sweeps; ++sw) {
        int sweep_rot = 0;
        ++sweeps_done;
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
            const int gp = block_col(P, Q, b, p), gq = block_col(P, Q, b, q);
            const bool hyp = gp < nplus && gq >= nplus;
            const bool border = (gp >= bord_lo && gp < bord_hi) || (gq >= bord_lo && gq < bord_hi);
            const bool rho = !border && needs_rotation(hpp, hqq, hpq, c_eps, c_eps2);
            Rot rot{1.0, 0.0};
            if (rho) rot = rot_params(hpp, hqq, hpq, hyp);
            bool swap = false;
            if (!hyp && !border) {
                const double npp = rho ? __fma_rn(-rot.tn, hpq, hpp) : hpp;
                const double nqq = rho ? __fma_rn(rot.tn, hpq, hqq) : hqq;
                swap = (gq < nplus && npp < nqq) || (gp >= nplus && npp > nqq);
            }
            if (rho || swap) {
#pragma unroll
                for (int k = 0; k < C::kRowsPerLane; ++k) {
                    const int r = g + k * C::kLanesPerPair;
                    double x = rp[r], z = rq[r];
                    double u = wp[r], v = wq[r];
                    if (rho) { rot_apply(x, z, hyp, rot); rot_apply(u, v, hyp, rot); }
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
                if (is_proper(rot)) ++my_proper;
            }
            __syncthreads();
        }
        if (inner_sweeps > 1 && __syncthreads_count(sweep_rot) == 0) break;
    }
    }

    // (6) V' and its flag to global memory; counters (in a cluster: the V'
    // outputs from CTA 1, the rotation counters from CTA 0)
    const int any_change = __syncthreads_or(changed);
    if (role != 0) {
        for (int e = tid; e < BB * BB; e += NT) {
            const int i = e % BB, j = e / BB;
            vp[e] = (double)Vt[i + j * C::kLd];
        }
        if constexpr (sizeof(RT) == sizeof(double))
            if (bsl && any_change) split_right_factor<BB, NT>(A, hdiag, dx, bsl, bexp, dexp, tc);
        // the update of G rewrites these columns and max-reduces their new bounds
        if (gexp && any_change)
            for (int k = tid; k < BB; k += NT) gexp[block_col(P, Q, b, k)] = split::kNoExp;
    }
    atomicAdd(&s_cnt[0], my_rot);
    atomicAdd(&s_cnt[1], my_proper);
    __syncthreads();
    if (tid == 0) {
        if (role != 0) {
            *vflag = any_change;
            if (any_change) atomicAdd(&counters[kCntUpdated], 1ull);
        }
        if (role != 1) {
            atomicAdd(&counters[kCntRot], (unsigned long long)s_cnt[0]);
            atomicAdd(&counters[kCntProper], (unsigned long long)s_cnt[1]);
            atomicAdd(&counters[kCntInner], (unsigned long long)sweeps_done);
            if (s_brk) atomicAdd(&counters[kCntBreak], (unsigned long long)s_brk);
            atomicMax(&counters[kCntOff], s_off);
        }
    }
    // no CTA of the cluster may exit while its peer can still reach its shared memory
    if constexpr (CLUSTER) cl::sync();
}

// ---------------------------------------------------------------------------
// Rows [r0, r0 + valid) of [A_P A_Q] := [A_P A_Q] V' (valid <= kUpdRows, a
// multiple of 4).  X (column-major, ld kUpdRows) and V' (row-major by k,
// ld BB+2) in shared memory; thread (rt, ct) owns a 4x4 output tile and sums
// over k = 0..BB-1 in increasing order.  Units of one pair own disjoint rows,
// so the result is written in place.
template <int BB, typename T>
__device__ __forceinline__ void update_unit(T *__restrict__ M, int ld, int r0, int valid, int P, int Q,
                                            int b, const double *__restrict__ vp, T *X) {
    using C = Cfg<BB>;
    using T2 = typename Vec2<T>::type;
    constexpr int RU = C::kUpdRows;
    constexpr int WLD = BB + 2;
    T *W = X + BB * RU;
    for (int e = threadIdx.x; e < BB * BB; e += kUpdThreads) {
        const int k = e % BB, c = e / BB;
        W[k * WLD + c] = (T)vp[e];
    }
    for (int e = threadIdx.x; e < BB * RU / 2; e += kUpdThreads) {
        const int r2 = e % (RU / 2), j = e / (RU / 2);
        if (2 * r2 < valid)
            reinterpret_cast<T2 *>(X + j * RU)[r2] =
                reinterpret_cast<const T2 *>(M + (size_t)block_col(P, Q, b, j) * ld + r0)[r2];
    }
    __syncthreads();
    const int rt = threadIdx.x % (RU / 4);
    const int ct = threadIdx.x / (RU / 4);
    if (4 * rt >= valid) return;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0;
#pragma unroll 4
    for (int k = 0; k < BB; ++k) {
        const T2 x01 = reinterpret_cast<const T2 *>(X + k * RU + 4 * rt)[0];
        const T2 x23 = reinterpret_cast<const T2 *>(X + k * RU + 4 * rt)[1];
        const T2 w01 = reinterpret_cast<const T2 *>(W + k * WLD + 4 * ct)[0];
        const T2 w23 = reinterpret_cast<const T2 *>(W + k * WLD + 4 * ct)[1];
        const T xv[4] = {x01.x, x01.y, x23.x, x23.y};
        const T wv[4] = {w01.x, w01.y, w23.x, w23.y};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(xv[i], wv[j], acc[i][j]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        T2 *dst = reinterpret_cast<T2 *>(M + (size_t)block_col(P, Q, b, 4 * ct + j) * ld + r0 + 4 * rt);
        T2 lo, hi;
        lo.x = acc[0][j]; lo.y = acc[1][j];
        hi.x = acc[2][j]; hi.y = acc[3][j];
        dst[0] = lo;
        dst[1] = hi;
    }
}

}  // namespace jsvd
