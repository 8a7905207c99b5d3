// Single-matrix block p-step kernels; see sweep_fp64.cuh.
#include <cuda_runtime.h>

#include <cstdint>

#include "sweep_fp64.cuh"

namespace jsvd {

// The pipelined variant on a 2-CTA cluster per pivot pair (one SM for the
// factorization and the R side, another for the V' side and the V' outputs),
// used when the p-step has at most half as many pairs as the GPU has SMs: the
// R side then has its SM's FP64 pipe to itself.  Same results bit for bit.
template <int BB, typename RT = double>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(2 * Cfg<BB>::kJacThreads)
    pair_jacobi_cl(PStepArgs a) {
    extern __shared__ __align__(16) double smem[];
    const int pair = blockIdx.x >> 1;
    const int P = a.table[2 * (a.step * a.npairs + pair)];
    const int Q = a.table[2 * (a.step * a.npairs + pair) + 1];
    const double *part = a.part + (size_t)pair * a.g_parts * Cfg<BB>::kPacked;
    uint16_t *bsl = a.split ? a.bslice + (size_t)pair * 2 * split_b_elems<BB>() : nullptr;
    int *bexp = a.split ? a.bexp + (size_t)pair * 2 * BB : nullptr;
    int *dexp = a.split ? a.dexp + (size_t)pair * BB : nullptr;
    int *gexp = a.split ? a.gexp : nullptr;
    jacobi_unit<BB, 2 * Cfg<BB>::kJacThreads, RT, true>(part, a.g_parts, a.inner, P, Q, a.b, a.nplus, a.bord_lo,
                                                         a.bord_hi, 1, a.eps, a.vprime + (size_t)pair * BB * BB,
                                                         a.vflag + pair, a.counters, smem, bsl, bexp, dexp, gexp,
                                                         a.tc != 0);
}

// The cluster kernel requests enough shared memory that no two of its CTAs
// share an SM (the point is a second FP64 pipe for the V' side).
template <int BB>
constexpr size_t jacobi_cl_smem_bytes() {
    return jacobi_smem_bytes<BB>() > 120 * 1024 ? jacobi_smem_bytes<BB>() : 120 * 1024;
}

// SMs of the current device (cached per device).
static int sm_count() {
    static int nsm[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 148;
    if (nsm[dev] == 0) cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev);
    return nsm[dev];
}

template <int BB, typename T>
__global__ void __launch_bounds__(Cfg<BB>::kGramThreads) gram_partial(PStepArgs a) {
    extern __shared__ __align__(16) double smem[];
    const int pair = blockIdx.y, chunk = blockIdx.x;
    const int P = a.table[2 * (a.step * a.npairs + pair)];
    const int Q = a.table[2 * (a.step * a.npairs + pair) + 1];
    double *out = a.part + ((size_t)pair * a.g_chunks + chunk) * Cfg<BB>::kPacked;
    gram_unit<BB, T>(reinterpret_cast<const T *>(a.G), a.ldg, chunk * kGramRows, kGramRows, P, Q, a.b, out,
                     reinterpret_cast<T *>(smem));
}

// NT = kJacThreads: any number of inner sweeps; NT = 2 kJacThreads: one inner
// sweep with V' rotated by a second thread group (jacobi_sweep_pipelined),
// R and V' held in RT (float in the FP32 sweeps of the mixed solver, whose
// rotations are then FP32 too; the sum of the Gram partials and the Cholesky
// stay FP64).
template <int BB, int NT, typename RT = double>
__global__ void __launch_bounds__(NT) pair_jacobi(PStepArgs a) {
    extern __shared__ __align__(16) double smem[];
    const int pair = blockIdx.x;
    const int P = a.table[2 * (a.step * a.npairs + pair)];
    const int Q = a.table[2 * (a.step * a.npairs + pair) + 1];
    jacobi_unit<BB, NT, RT>(a.part + (size_t)pair * a.g_parts * Cfg<BB>::kPacked, a.g_parts, a.inner, P, Q, a.b,
                    a.nplus, a.bord_lo, a.bord_hi, a.inner_sweeps, a.eps, a.vprime + (size_t)pair * BB * BB, a.vflag + pair,
                    a.counters, smem, a.split ? a.bslice + (size_t)pair * 2 * split_b_elems<BB>() : nullptr,
                    a.split ? a.bexp + (size_t)pair * 2 * BB : nullptr, a.split ? a.dexp + (size_t)pair * BB : nullptr,
                    a.split ? a.gexp : nullptr, a.tc != 0);
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

// The dynamic shared memory limit of each kernel is raised once per device.
template <int BB, typename T>
static void configure_once() {
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    cudaFuncSetAttribute(gram_partial<BB, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)gram_smem_bytes<BB, T>());
    cudaFuncSetAttribute(pair_jacobi<BB, Cfg<BB>::kJacThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)jacobi_smem_bytes<BB>());
    cudaFuncSetAttribute(pair_jacobi<BB, 2 * Cfg<BB>::kJacThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)jacobi_smem_bytes<BB>());
    cudaFuncSetAttribute(pair_jacobi<BB, 2 * Cfg<BB>::kJacThreads, float>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jacobi_smem_bytes<BB>());
    cudaFuncSetAttribute(pair_jacobi_cl<BB, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)jacobi_cl_smem_bytes<BB>());
    cudaFuncSetAttribute(pair_jacobi_cl<BB, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)jacobi_cl_smem_bytes<BB>());
    cudaFuncSetAttribute(block_update<BB, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)update_smem_bytes<BB, T>());
    done[dev] = true;
}

template <int BB, typename T>
static void launch_bb(Phase ph, const PStepArgs &a, cudaStream_t s) {
    using C = Cfg<BB>;
    configure_once<BB, T>();
    switch (ph) {
        case Phase::Gram: {
            const size_t sm = gram_smem_bytes<BB, T>();
            gram_partial<BB, T><<<dim3(a.g_chunks, a.npairs), C::kGramThreads, sm, s>>>(a);
            break;
        }
        case Phase::Jacobi: {
            const size_t sm = jacobi_smem_bytes<BB>();
            const bool cluster = a.inner_sweeps == 1 && 2 * a.npairs <= sm_count();
            if (cluster && a.fp32)
                pair_jacobi_cl<BB, float><<<2 * a.npairs, 2 * C::kJacThreads, jacobi_cl_smem_bytes<BB>(), s>>>(a);
            else if (cluster)
                pair_jacobi_cl<BB, double><<<2 * a.npairs, 2 * C::kJacThreads, jacobi_cl_smem_bytes<BB>(), s>>>(a);
            else if (a.inner_sweeps == 1 && a.fp32)
                pair_jacobi<BB, 2 * C::kJacThreads, float><<<a.npairs, 2 * C::kJacThreads, sm, s>>>(a);
            else if (a.inner_sweeps == 1)
                pair_jacobi<BB, 2 * C::kJacThreads><<<a.npairs, 2 * C::kJacThreads, sm, s>>>(a);
            else
                pair_jacobi<BB, C::kJacThreads><<<a.npairs, C::kJacThreads, sm, s>>>(a);
            break;
        }
        default: {
            const size_t sm = update_smem_bytes<BB, T>();
            const int gu = (ph == Phase::UpdateV) ? 0 : a.g_rows / C::kUpdRows;
            const int vu = (ph == Phase::UpdateG || !a.V) ? 0 : a.v_rows / C::kUpdRows;
            if (gu + vu > 0) block_update<BB, T><<<dim3(gu + vu, a.npairs), kUpdThreads, sm, s>>>(a, gu);
            break;
        }
    }
}

void launch_phase(int BB, Phase ph, const PStepArgs &a, cudaStream_t s) {
    if (a.split && !a.fp32 && ph != Phase::Jacobi) {
        launch_split_phase(BB, ph, a, s);
        return;
    }
    if (a.fp32) {
        switch (BB) {
            case 16: launch_bb<16, float>(ph, a, s); break;
            case 32: launch_bb<32, float>(ph, a, s); break;
            case 64: launch_bb<64, float>(ph, a, s); break;
            default: break;
        }
    } else {
        switch (BB) {
            case 16: launch_bb<16, double>(ph, a, s); break;
            case 32: launch_bb<32, double>(ph, a, s); break;
            case 64: launch_bb<64, double>(ph, a, s); break;
            default: break;
        }
    }
}

}  // namespace jsvd
