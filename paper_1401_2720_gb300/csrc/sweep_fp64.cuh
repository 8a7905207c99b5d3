// FP64 block p-step of the block-oriented one-sided Jacobi (H)SVD (Sec. 2, 4).
//
// One p-step is three launches over the n_b/2 disjoint block pairs (P, Q)
// of the step's row of the block p-strategy table:
//
//   gram_partial<BB>   H_pq partial sums (lower triangle) of one row chunk of
//                      [G_P G_Q] per CTA: grid (row chunks, pairs).
//                      Eq. (2.7) / Alg. 4.1 split over rows so every SM works.
//   pair_jacobi<BB>    per pair: fixed-order sum of the partials, Cholesky
//                      H = L L^T, R = L^T (Sec. 4.1), V' = I, M_s inner sweeps
//                      of the pointwise method on R (Sec. 4.3), V' to global
//                      memory with a flag "V' != I", rotation counters.
//   block_update<BB>   [A_P A_Q] := [A_P A_Q] V' for A = G and A = V,
//                      one row chunk per CTA (Eq. (2.9) / Alg. 4.2).
//
// BB = 2b is the order of the pivot block.  All arithmetic is FP64; the
// FP64 pipe is the bound on this GPU, so every FMA that is issued does useful
// work: the Gram kernel computes only the lower triangle, the update skips
// pairs whose V' is the identity.
#pragma once
#include <cstdint>

namespace jsvd {

struct PStepArgs {
    double *G;              // m_pad x n_pad, column-major, ld = ldg
    int ldg;
    int g_rows;             // rows of G processed (multiple of 256)
    double *V;              // v_rows x n_pad, ld = ldv (may be null)
    int ldv;
    int v_rows;             // rows of V processed (multiple of 256)
    const int *table;       // outer table: [steps][npairs][2]
    int npairs;             // n_b / 2
    int step;               // p-step index into the table
    const unsigned char *inner;  // inner table: [BB-1][BB/2][2]
    int b;                  // block width
    int nplus;              // workspace columns < nplus are J = +1
    int inner_sweeps;       // M_s
    double *part;           // Gram partials [npairs][g_chunks][BB*(BB+1)/2]
    int g_chunks;           // g_rows / kGramRows
    double *vprime;         // V' [npairs][BB*BB], column-major
    int *vflag;             // [npairs]: 1 if V' != I
    unsigned long long *counters;  // see kCnt* below
};

enum {
    kCntRot = 0,       // rotations (rho = 1)
    kCntProper = 1,    // proper rotations (cs != 1)
    kCntUpdated = 2,   // block pairs with V' != I
    kCntBreak = 3,     // Cholesky breakdowns
    kCntOff = 4,       // max normalized off-diagonal |h_ij|/sqrt(h_ii h_jj), double bits
    kCntErr = 5,       // device-side error flags
    kCntSize = 8
};

constexpr int kGramRows = 128;     // rows of [G_P G_Q] per Gram CTA
constexpr int kGramThreads = 256;
constexpr int kUpdThreads = 256;   // 4x4 output tiles per thread
constexpr int kRowAlign = 256;     // g_rows, v_rows are multiples of this

template <int BB> struct Cfg {
    static constexpr int kPairsInner = BB / 2;
    static constexpr int kLanesPerPair = 8;
    static constexpr int kJacThreads = kPairsInner * kLanesPerPair;   // 4*BB
    static constexpr int kRowsPerLane = BB / kLanesPerPair;
    static constexpr int kLd = BB + 1;                                // smem ld for R, V'
    static constexpr int kPacked = BB * (BB + 1) / 2;
    static constexpr int kUpdRows = 4096 / BB;                        // rows per update CTA
    static constexpr int kGramLd = BB + 2;                            // smem row stride
};

// Launches the three kernels of one p-step on stream s.  If ev is not null,
// ev[0..3] are recorded before the Gram, Jacobi and update launches and
// after the update launch.
void launch_pstep_fp64(int BB, const PStepArgs &a, cudaStream_t s, cudaEvent_t *ev);
size_t pstep_smem_jacobi(int BB);

}  // namespace jsvd
