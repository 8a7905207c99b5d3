// Throughput probes for the rooflines the benchmark reports.  FP64: two
// kernels keep every SM's FP64 pipe busy for a requested time, one with
// independent DFMA chains and one with FP64 mma.sync (m8n8k4) accumulations.
// bf16: the mma.sync m16n8k16 instruction that the split contractions issue,
// 8 independent accumulators per warp.  Each is timed with CUDA events on the
// context's stream after a warm-up of the same length (so the SM clock has
// settled).  Nothing here is on the SVD path.
#include <cuda_runtime.h>

#include "driver.h"
#include "jsvd.h"

namespace {

constexpr int kMma = 8;       // independent mma accumulators per warp

// GEMM-shaped: a 4x4 register tile of accumulators, each FMA depending on the
// previous one through its addend, the operands taken from two register
// vectors (as in the update kernel's inner loop, minus its loads).
__global__ void probe_dfma(double *out, int iters) {
    double x[4], y[4], acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        x[i] = 1e-3 * threadIdx.x + i;
        y[i] = 0.5 - 1e-9 * i;
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = __fma_rn(x[i], y[(j + r) & 3], acc[i][j]);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) s += acc[i][j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void probe_dmma(double *out, int iters) {
    double av[kMma], bv[kMma];
#pragma unroll
    for (int j = 0; j < kMma; ++j) {
        av[j] = 1e-3 * ((threadIdx.x + j) & 7);
        bv[j] = 0.5 - 1e-3 * j;
    }
    double c[kMma][2];
#pragma unroll
    for (int j = 0; j < kMma; ++j) c[j][0] = c[j][1] = 0.0;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kMma; ++j)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                         : "+d"(c[j][0]), "+d"(c[j][1])
                         : "d"(av[j]), "d"(bv[(j + 3) % kMma]));
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kMma; ++j) s += c[j][0] + c[j][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void probe_bf16(double *out, int iters) {
    const unsigned a0 = 0x3f803f80u ^ (threadIdx.x & 7u), b0 = 0x3f003f00u;   // small bf16 pairs
    float c[kMma][4];
#pragma unroll
    for (int j = 0; j < kMma; ++j) c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kMma; ++j)
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+f"(c[j][0]), "+f"(c[j][1]), "+f"(c[j][2]), "+f"(c[j][3])
                : "r"(a0), "r"(a0 + j), "r"(a0), "r"(a0 + 1), "r"(b0), "r"(b0 + j));
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kMma; ++j) s += c[j][0] + c[j][1] + c[j][2] + c[j][3];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Calibrate the iteration count of probe `kind` to about `seconds`, warm up,
// time; returns TFLOP/s or a negative status.
double run_probe(jsvd_ctx_t ctx, int kind, double seconds, double *buf, int blocks, int threads, int *rc) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int iters = 64;
    float ms = 0.f;
    for (int pass = 0; pass < 3; ++pass) {
        cudaEventRecord(e0, ctx->stream);
        if (kind == 0) probe_dfma<<<blocks, threads, 0, ctx->stream>>>(buf, iters);
        else if (kind == 1) probe_dmma<<<blocks, threads, 0, ctx->stream>>>(buf, iters);
        else probe_bf16<<<blocks, threads, 0, ctx->stream>>>(buf, iters);
        cudaEventRecord(e1, ctx->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) { *rc = ctx->check("probe"); break; }
        cudaEventElapsedTime(&ms, e0, e1);
        if (pass < 2) {
            double scale = (seconds * 1e3) / (ms > 1e-3 ? ms : 1e-3);
            double next = iters * scale;
            iters = next > 2e9 ? 2000000000 : (next < 1 ? 1 : (int)next);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double warps = (double)blocks * (threads / 32);
    const double fl = kind == 0 ? 2.0 * 64 * (double)iters * blocks * threads
                    : kind == 1 ? 2.0 * 8 * 8 * 4 * kMma * (double)iters * warps
                                : 2.0 * 16 * 8 * 16 * kMma * (double)iters * warps;
    return fl / (ms * 1e-3) / 1e12;
}

}  // namespace

extern "C" int jsvd_bf16_mma_peak(jsvd_ctx_t ctx, double seconds, double *tflops) {
    if (!ctx) return -1;
    if (!(seconds > 0.0) || seconds > 60.0) return -2;
    cudaSetDevice(ctx->device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const int blocks = sms * 2, threads = 256;
    double *buf = nullptr;
    if (cudaMalloc(&buf, sizeof(double) * blocks * threads) != cudaSuccess) return ctx->check("probe alloc");
    int rc = 0;
    const double tf = run_probe(ctx, 2, seconds, buf, blocks, threads, &rc);
    cudaFree(buf);
    if (!rc) rc = ctx->check("probe");
    if (!rc && tflops) *tflops = tf;
    return rc;
}

extern "C" int jsvd_fp64_peak(jsvd_ctx_t ctx, double seconds, double *dfma_tflops, double *dmma_tflops) {
    if (!ctx) return -1;
    if (!(seconds > 0.0) || seconds > 60.0) return -2;
    cudaSetDevice(ctx->device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const int blocks = sms * 8, threads = 256;
    double *buf = nullptr;
    if (cudaMalloc(&buf, sizeof(double) * blocks * threads) != cudaSuccess) return ctx->check("probe alloc");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = 0;
    for (int kind = 0; kind < 2 && !rc; ++kind) {
        // calibrate the iteration count on a short launch, then warm up and time
        int iters = 64;
        float ms = 0.f;
        for (int pass = 0; pass < 3; ++pass) {
            cudaEventRecord(e0, ctx->stream);
            if (kind == 0) probe_dfma<<<blocks, threads, 0, ctx->stream>>>(buf, iters);
            else probe_dmma<<<blocks, threads, 0, ctx->stream>>>(buf, iters);
            cudaEventRecord(e1, ctx->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = ctx->check("probe"); break; }
            cudaEventElapsedTime(&ms, e0, e1);
            if (pass < 2) {
                double scale = (seconds * 1e3) / (ms > 1e-3 ? ms : 1e-3);
                double next = iters * scale;
                iters = next > 2e9 ? 2000000000 : (next < 1 ? 1 : (int)next);
            }
        }
        if (rc) break;
        const double fl = kind == 0 ? 2.0 * 64 * (double)iters * blocks * threads
                                    : 2.0 * 8 * 8 * 4 * kMma * (double)iters * blocks * (threads / 32);
        const double tf = fl / (ms * 1e-3) / 1e12;
        if (kind == 0 && dfma_tflops) *dfma_tflops = tf;
        if (kind == 1 && dmma_tflops) *dmma_tflops = tf;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (!rc) rc = ctx->check("probe");
    return rc;
}
