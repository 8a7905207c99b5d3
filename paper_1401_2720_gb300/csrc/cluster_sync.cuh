// Thread-block-cluster primitives as inline PTX (sm_90 and later): the CTA's
// rank in its cluster, distributed shared memory (a peer CTA's shared-memory
// address, stores into it), mbarrier arrivals on a peer's barrier with
// release semantics at cluster scope, bounded waits with acquire semantics at
// cluster scope, and the cluster-wide barrier.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace jsvd {
namespace cl {

__device__ __forceinline__ uint32_t rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// The address of `p` (this CTA's shared memory) in the shared memory of CTA
// `peer` of the cluster.
__device__ __forceinline__ uint32_t peer_addr(const void *p, uint32_t peer) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(peer));
    return r;
}

__device__ __forceinline__ void st_f64(uint32_t addr, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ void st_s32(uint32_t addr, int v) {
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// One arrival on the mbarrier at cluster shared-memory address `addr`
// (possibly a peer's), releasing this thread's prior writes at cluster scope.
__device__ __forceinline__ void arrive_remote(uint32_t addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(addr) : "memory");
}

// Wait for the phase with the given parity of a local mbarrier, acquiring at
// cluster scope; false after `limit` suspended polls of ~1 ms each.
__device__ __forceinline__ bool wait_parity(uint64_t *bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity), "r"(1000000u)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Every thread of every CTA of the cluster (warp-uniform).
__device__ __forceinline__ void sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

}  // namespace cl
}  // namespace jsvd
