// Single-matrix block p-step kernels; see sweep_fp64.cuh.
#include <cuda_runtime.h>

#include <cstdint>

#include "sweep_fp64.cuh"

namespace jsvd {

template <int BB, typename T>
__global__ void __launch_bounds__(kGramThreads) gram_partial(PStepArgs a) {
    extern __shared__ __align__(16) double smem[];
    const int pair = blockIdx.y, chunk = blockIdx.x;
    const int P = a.table[2 * (a.step * a.npairs + pair)];
    const int Q = a.table[2 * (a.step * a.npairs + pair) + 1];
    double *out = a.part + ((size_t)pair * a.g_chunks + chunk) * Cfg<BB>::kPacked;
    gram_unit<BB, T>(reinterpret_cast<const T *>(a.G), a.ldg, chunk * kGramRows, kGramRows, P, Q, a.b, out,
                     reinterpret_cast<T *>(smem));
}

template <int BB>
__global__ void __launch_bounds__(Cfg<BB>::kJacThreads) pair_jacobi(PStepArgs a) {
    extern __shared__ __align__(16) double smem[];
    const int pair = blockIdx.x;
    const int P = a.table[2 * (a.step * a.npairs + pair)];
    const int Q = a.table[2 * (a.step * a.npairs + pair) + 1];
    jacobi_unit<BB>(a.part + (size_t)pair * a.g_chunks * Cfg<BB>::kPacked, a.g_chunks, a.inner, P, Q, a.b,
                    a.nplus, a.bord_lo, a.bord_hi, a.inner_sweeps, a.eps, a.vprime + (size_t)pair * BB * BB, a.vflag + pair,
                    a.counters, smem);
}

template <int BB, typename T>
__global__ void __launch_bounds__(kUpdThreads) block_update(PStepArgs a, int g_chunks_u) {
    constexpr int RU = Cfg<BB>::kUpdRows;
    extern __shared__ __align__(16) double smem[];
    const int pair = blockIdx.y;
    if (!a.vflag[pair]) return;
    const int P = a.table[2 * (a.step * a.npairs + pair)];
    const int Q = a.table[2 * (a.step * a.npairs + pair) + 1];
    T *M;
    int ld, r0;
    if ((int)blockIdx.x < g_chunks_u) {
        M = reinterpret_cast<T *>(a.G); ld = a.ldg; r0 = blockIdx.x * RU;
    } else {
        M = reinterpret_cast<T *>(a.V); ld = a.ldv; r0 = (blockIdx.x - g_chunks_u) * RU;
    }
    update_unit<BB, T>(M, ld, r0, RU, P, Q, a.b, a.vprime + (size_t)pair * BB * BB, reinterpret_cast<T *>(smem));
}

template <int BB, typename T>
static void launch_bb(const PStepArgs &a, cudaStream_t s, cudaEvent_t *ev) {
    using C = Cfg<BB>;
    const size_t sm_gram = gram_smem_bytes<BB, T>();
    const size_t sm_jac = jacobi_smem_bytes<BB>();
    const size_t sm_upd = update_smem_bytes<BB, T>();
    cudaFuncSetAttribute(gram_partial<BB, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_gram);
    cudaFuncSetAttribute(pair_jacobi<BB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_jac);
    cudaFuncSetAttribute(block_update<BB, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_upd);
    if (ev) cudaEventRecord(ev[0], s);
    gram_partial<BB, T><<<dim3(a.g_chunks, a.npairs), kGramThreads, sm_gram, s>>>(a);
    if (ev) cudaEventRecord(ev[1], s);
    pair_jacobi<BB><<<a.npairs, C::kJacThreads, sm_jac, s>>>(a);
    if (ev) cudaEventRecord(ev[2], s);
    const int gu = a.g_rows / C::kUpdRows;
    const int vu = a.V ? a.v_rows / C::kUpdRows : 0;
    block_update<BB, T><<<dim3(gu + vu, a.npairs), kUpdThreads, sm_upd, s>>>(a, gu);
    if (ev) cudaEventRecord(ev[3], s);
}

void launch_pstep_fp64(int BB, const PStepArgs &a, cudaStream_t s, cudaEvent_t *ev) {
    if (a.fp32) {
        switch (BB) {
            case 16: launch_bb<16, float>(a, s, ev); break;
            case 32: launch_bb<32, float>(a, s, ev); break;
            case 64: launch_bb<64, float>(a, s, ev); break;
            default: break;
        }
    } else {
        switch (BB) {
            case 16: launch_bb<16, double>(a, s, ev); break;
            case 32: launch_bb<32, double>(a, s, ev); break;
            case 64: launch_bb<64, double>(a, s, ev); break;
            default: break;
        }
    }
}

}  // namespace jsvd
