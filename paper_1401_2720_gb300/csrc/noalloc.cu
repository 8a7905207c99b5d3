// jsvd_dgesvj_noalloc: the FP64 SVD for callers that cannot allocate device
// memory -- code inside a framework whose memory pool owns every device byte,
// or a process under a cap on cudaMalloc.  The paper has no counterpart; this
// only changes where the solver's scratch lives.  Like jsvd_dgesvj it
// synchronises its stream (once per block sweep, to read the rotation
// counters, and once at the end).
//
// All scratch (the bordered working copy of G, V, the Gram partials, V', the
// counters, the pivot tables, the singular-value workspace) is carved from
// one file-scope __device__ array of kScratchBytes; nothing here calls
// cudaMalloc, cudaMallocHost, cudaFree or an allocating library routine.
// The kernels are the ones jsvd_dgesvj launches.
#include <cuda_runtime.h>

#include <mutex>

#include "driver.h"
#include "jsvd.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB, held by every GPU that loads the library
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device addresses of the array, looked up once per device.  In host code the
// name g_noalloc_scratch is only a host-side stand-in, never a device address.
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// A context whose workspace requests are bump-allocated from the array.
struct NoallocCtx : jsvd_ctx {
    unsigned char *base;
    size_t used = 0;
    unsigned long long counters_host[8] = {};   // pageable: no cudaMallocHost

    // one stream, no events: nothing is created
    explicit NoallocCtx(void *b) : base(static_cast<unsigned char *>(b)) {
        host_counters = counters_host;
        side_streams = false;
        owns_memory = false;   // every Buffer points into the static array
    }

    int ensure(Buffer &buf, size_t bytes) override {
        if (buf.bytes >= bytes) return 0;
        const size_t off = (used + 255) & ~size_t(255);
        if (off > kScratchBytes || bytes > kScratchBytes - off) {
            last_error = "the problem needs more scratch than the static array holds";
            return JSVD_ERR_TOO_LARGE;
        }
        buf.ptr = base + off;
        buf.bytes = bytes;
        used = off + bytes;
        return 0;
    }
};

}  // namespace

extern "C" int jsvd_dgesvj_noalloc(int m, int n, const double *A, int lda, double *S, double *U, int ldu,
                                   double *V, int ldv, const jsvd_opts *opts, jsvd_info *info, void *stream) {
    if (m < 1 || m < n) return -1;
    if (n < 1) return -2;
    if (!A) return -3;
    if (lda < m) return -4;
    if (!S) return -5;
    if (!U) return -6;
    if (ldu < m) return -7;
    if (V && ldv < n) return -9;
    if (opts && opts->precision != JSVD_PREC_FP64) return JSVD_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return JSVD_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return JSVD_ERR_UNSUPPORTED;
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_addr[dev]) {
            // first call on this device (its device is current here)
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return JSVD_ERR_CUDA;
            }
            g_scratch_addr[dev] = p;
        }
        base = g_scratch_addr[dev];
    }
    NoallocCtx ctx(base);
    ctx.device = dev;
    ctx.stream = static_cast<cudaStream_t>(stream);
    return ctx.solve(m, n, n, A, lda, S, U, ldu, V, ldv, opts, info, false);
}
