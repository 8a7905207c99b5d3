// Dense FP64-accumulating GEMM used around the sweep (mixed-precision
// re-orthonormalization, G = A Q) and by the SVD adjoint:
//   C = alpha * op(A) * op(B) + beta * C,   op(X) = X or X^T,
// column-major, A and B stored as float or double (converted to double on
// load), FP64 FMA accumulation in increasing k.  A group of independent
// problems of different shapes is one launch (grouped GEMM).
#pragma once
#include <cuda_runtime.h>

namespace jsvd {

struct GemmDesc {
    int M, N, K;
    const void *A;
    int lda;
    const void *B;
    int ldb;
    double *C;
    int ldc;
    double alpha, beta;
    int tile0;   // first tile index of this problem in the launch
};

enum class Elt { F32, F64 };

// One problem (batch = 1): all pointers device, C not aliased with A or B.
void gemm(bool ta, bool tb, Elt ea, Elt eb, int M, int N, int K, double alpha, const void *A, int lda,
          const void *B, int ldb, double beta, double *C, int ldc, cudaStream_t s);

// Grouped launch over `count` descriptors in device memory; tile0 of each
// descriptor must be the running sum of ceil(M/64)*ceil(N/64) of the ones
// before it, and total_tiles their sum.  All problems share ta, tb, ea, eb.
void gemm_grouped(bool ta, bool tb, Elt ea, Elt eb, const GemmDesc *descs, int count, int total_tiles,
                  cudaStream_t s);

constexpr int kGemmTile = 64;

}  // namespace jsvd
