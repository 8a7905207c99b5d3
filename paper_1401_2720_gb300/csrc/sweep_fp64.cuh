// Block p-step of the block-oriented one-sided Jacobi (H)SVD on one matrix
// (Sec. 2, 4 of the paper).  One p-step is three launches over the n_b/2
// disjoint block pairs (P, Q) of the step's row of the block p-strategy table:
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
// BB = 2b is the order of the pivot block.  With PStepArgs::split (the
// default for the FP64 sweeps) the Gram and update launches are tensor-core
// kernels -- with PStepArgs::tc (the default) gram_tc / update_tc on tcgen05
// (gram_tc.cu, update_tc.cu), else gram_split / update_split on mma.sync
// (sweep_split.cu, split_kernels.cuh) -- and pair_jacobi also writes the
// split right factors.
// In the FP64 FMA form all arithmetic is FP64 and the FP64 pipe is the bound,
// so every FMA that is issued does useful work: the Gram kernel computes only
// the lower triangle, the update skips pairs whose V' is the identity.  In the
// FP32 form (the first stage of the mixed-precision solver) G and V are float,
// the Gram's per-chunk sums, the update and the inner sweep's dots and
// rotations run in FP32, and the chunk sums, Cholesky factor, rotation
// parameters (Eqs. (4.3)-(4.6)) and counters stay FP64.
#pragma once
#include <cstdint>

#include "sweep_device.cuh"

namespace jsvd {

struct PStepArgs {
    void *G;                // g_rows x n_pad, column-major, ld = ldg (double, or float if fp32)
    int ldg;
    int g_rows;             // rows of G processed (multiple of kRowAlign)
    void *V;                // v_rows x n_pad, ld = ldv (may be null), same type as G
    int ldv;
    int v_rows;             // rows of V processed (multiple of kRowAlign)
    const int *table;       // outer table: [steps][npairs][2]
    int npairs;             // n_b / 2
    int step;               // p-step index into the table
    const unsigned char *inner;  // inner table: [BB-1][BB/2][2]
    int b;                  // block width
    int nplus;              // workspace columns < nplus are J = +1
    int bord_lo, bord_hi;   // workspace columns of the identity border (never rotated or swapped)
    int inner_sweeps;       // M_s
    int fp32;               // 1: G, V are float; Gram sums and update in FP32
    double eps;             // unit roundoff of the relative test: 2^-53, or 2^-24 in FP32 sweeps
    double *part;           // Gram partials [npairs][g_chunks][BB*(BB+1)/2]
    int g_chunks;           // g_rows / kGramRows (kGramRowsSplit for the split forms)
    int g_parts;            // partial slots per pair the Jacobi kernel sums: g_chunks, or fewer when the
                            // tcgen05 Gram adds up each CTA's consecutive chunks of a pair
    double *vprime;         // V' [npairs][BB*BB], column-major
    int *vflag;             // [npairs]: 1 if V' != I
    unsigned long long *counters;  // kCnt* slots
    // tensor-core contractions (FP64 sweeps only): the Jacobi kernel writes the
    // split right factors, the Gram and update kernels are the split forms
    int split;
    uint16_t *bslice;       // [npairs][2][split_b_elems<BB>] digits (G version, V version)
    int *bexp;              // [npairs][2][BB] column exponent bounds of the right factors
    int *dexp;              // [npairs][BB] column scales of [G_P G_Q]
    int *gexp;              // [n_pad] exponent bound of every column of G: |g_ij| < 2^gexp[j]
    int tc;                 // 1: the Gram and the update run on tcgen05 (gram_tc.cu, update_tc.cu);
                            // bslice then holds the 8-bit images [npairs][2][split8::image_elems<BB>]
};


constexpr int kRowAlign = 256;     // g_rows, v_rows are multiples of this

// One kernel of a p-step on stream s: the Gram partials, the per-pair
// Cholesky + inner sweep, or the update of G, of V, or of both.
enum class Phase { Gram, Jacobi, UpdateG, UpdateV, UpdateGV };
void launch_phase(int BB, Phase ph, const PStepArgs &a, cudaStream_t s);
// The tensor-core forms of the Gram and update phases (sweep_split.cu).
void launch_split_phase(int BB, Phase ph, const PStepArgs &a, cudaStream_t s);
// The tcgen05 block update (update_tc.cu): G and V of every pair with V' != I.
void launch_update_tc(int BB, const PStepArgs &a, cudaStream_t s);
// The Gram partials on tcgen05 (gram_tc.cu), when PStepArgs::tc is set.
void launch_gram_tc(int BB, const PStepArgs &a, cudaStream_t s);
// Partial slots per pair the tcgen05 Gram writes for these arguments (g_parts).
int gram_tc_parts(const PStepArgs &a);
// gexp[j] = exponent bound of column j of G (rows [0, rows)), one CTA per column.
void launch_col_maxexp(const double *G, int ldg, int rows, int ncols, int *gexp, cudaStream_t s);

}  // namespace jsvd
