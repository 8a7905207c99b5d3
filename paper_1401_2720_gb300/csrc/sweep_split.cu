// Tensor-core forms of the two contractions of the FP64 block p-step for one
// matrix (Eq. (2.7) Gram partials, Eq. (2.9) block update); the pipelines are
// in split_kernels.cuh.  Launched by launch_phase when PStepArgs::split is set;
// the per-pair Cholesky and inner sweep are the FP64 pair_jacobi kernel, whose
// epilogue writes the split right factors.
#include <cuda_runtime.h>

#include <cstdint>

#include "split_kernels.cuh"
#include "sweep_fp64.cuh"

namespace jsvd {

// ---------------------------------------------------------------------------
// Exponent bound of every column of G: gexp[j] = max_i exp_bound(G(i, j)),
// one CTA per column.  Seeds the bounds at the start of the FP64 sweeps; the
// split update keeps them current afterwards.
__global__ void k_col_maxexp(const double *__restrict__ G, int ldg, int rows, int *__restrict__ gexp) {
    __shared__ int red[32];
    const double *col = G + (size_t)blockIdx.x * ldg;
    int m = split::kNoExp;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) m = max(m, split::exp_bound(col[r], 0));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : split::kNoExp;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) gexp[blockIdx.x] = m;
    }
}

void launch_col_maxexp(const double *G, int ldg, int rows, int ncols, int *gexp, cudaStream_t s) {
    k_col_maxexp<<<ncols, 256, 0, s>>>(G, ldg, rows, gexp);
}

// ---------------------------------------------------------------------------
// Single-matrix kernels: Gram grid (ceil(chunks / kChunksPerCta), pairs);
// update grid (units, pairs), a unit being kUpdRowsPerCta rows of G
// (blockIdx.x < g_units) or of V.
template <int BB>
__global__ void __launch_bounds__(SplitCfg<BB>::kGThreads, 1) gram_split(PStepArgs a) {
    using S = SplitCfg<BB>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int pair = blockIdx.y;
    const int P = a.table[2 * (a.step * a.npairs + pair)];
    const int Q = a.table[2 * (a.step * a.npairs + pair) + 1];
    const int chunk0 = blockIdx.x * S::kChunksPerCta;
    const int nchunks = min(S::kChunksPerCta, a.g_chunks - chunk0);
    gram_split_body<BB>(reinterpret_cast<const double *>(a.G), a.ldg, P, Q, a.b, a.gexp,
                        (size_t)chunk0 * kGramRowsSplit, nchunks * kGramRowsSplit,
                        a.part + (size_t)pair * a.g_chunks * Cfg<BB>::kPacked, chunk0, smem_raw);
}

template <int BB>
__global__ void __launch_bounds__(32 * SplitCfg<BB>::kUpdWarps) update_split(PStepArgs a, int g_units) {
    using S = SplitCfg<BB>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
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
    const int nrows = min(rows, rbeg + S::kUpdRowsPerCta) - rbeg;
    update_split_body<BB, false>(X, ld, (size_t)rbeg, nrows, P, Q, a.b,
                          a.bslice + ((size_t)pair * 2 + ver) * split_b_elems<BB>(),
                          a.bexp + ((size_t)pair * 2 + ver) * BB, ver ? nullptr : a.dexp + (size_t)pair * BB,
                          ver == 0 ? a.gexp : nullptr, smem_raw);
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
        if (a.tc) {
            launch_gram_tc(BB, a, s);
            return;
        }
        const int ctas = (a.g_chunks + S::kChunksPerCta - 1) / S::kChunksPerCta;
        gram_split<BB><<<dim3(ctas, a.npairs), S::kGThreads, gram_split_smem<BB>(), s>>>(a);
        return;
    }
    if (a.tc) {
        // G and V in one persistent tcgen05 launch
        launch_update_tc(BB, a, s);
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
