// jsvd_dgesvj_noalloc: the FP64 SVD for callers that cannot allocate device
// memory -- code running while a CUDA graph is being captured, inside a
// framework whose memory pool owns every device byte, or under a cap on
// cudaMalloc.  The paper has no counterpart; this only changes where the
// solver's scratch lives.
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

    ~NoallocCtx() override {
        // nothing was allocated: detach the carved buffers so that the base
        // destructor frees nothing
        for (Buffer *b : {&g, &v, &part, &vprime, &vflag, &counters, &sigma, &border, &perm, &bslice, &bexp, &dexp, &gexp,
                          &g32, &v32, &tmp_a,
                          &tmp_b, &tmp_g, &b_mats, &b_units, &b_g, &b_v, &b_part, &b_vp, &b_vflag, &b_tab, &b_cnt,
                          &b_stat, &b_starts, &b_sigma, &b_border, &b_perm, &b_misc, &b_bsl, &b_bex, &b_dex,
                          &b_gexp, &adj_w, &adj_meta,
                          &adj_desc}) {
            b->ptr = nullptr;
            b->bytes = 0;
        }
        tables.clear();
        host_counters = nullptr;
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
