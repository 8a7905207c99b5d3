// The Gram partials of one p-step, H = [G_P G_Q]^T [G_P G_Q] over 256-row
// chunks (Eq. (2.7)), on the 5th-generation tensor cores (tcgen05.mma
// kind::f16, accumulators in tensor memory), FP64-accurate through the 8-bit
// digit form of split8.cuh: every column c of the pair gets its exponent bound
// E_c (from the column bounds G carries), every entry the digits d_0..d_7 of
// Y = trunc(x 2^(62 - E_c)), and H(c, n) = 2^(E_c + E_n - 68) T with
// T = sum_{L<=7} lev_L 256^(7-L), lev_L = sum_{i+l=L} sum_rows d_i(c) d_l(n).
//
// The A operand of an MMA is 128 rows: SF = 128 / BB digit slices of the
// pair's BB columns stacked (slice i = g SF + s in rows s BB .. s BB + BB - 1),
// the B operand the slices 0 .. 7 - g SF of the output columns of one half
// (NC = 32 or 16 columns each), so one MMA per group g and half writes
//   lanes s BB + c, column block j (NC columns):  sum_rows d_{g SF + s}(c) d_{j - g SF}(n)
// at column block g SF .. 7: lane s BB + c and block j hold a part of level
// j + s.  For BB = 64 this is 4 MMAs per K-step and half (N = 256, 192, 128,
// 64: 11 % more digit products than the 36 needed, at the full M = 128 rate).
// Every TMEM column accumulates at most 8 / SF slices over 256 rows, so its
// sums are integers below 2^24 and exact in FP32.  The epilogue converts
// them to ints and adds the parts of every level of the lower triangle into
// integer level sums in shared memory, which then hold the exact level sums
// of all the CTA's consecutive chunks of the pair; it recombines them
// (split8::combine_levels, one rounding) once per such run and writes the
// run's partial (layout [pair][slot][packed lower]; a slot per CTA holding
// chunks of the pair).
//
// One persistent CTA per SM walks a contiguous range of the (pair, chunk)
// units.  Warp roles, synchronised through shared-memory mbarriers:
//   warps 0-15  epilogue (TMEM lane quadrant w % 4, every fourth 16-column
//               load from w / 4 in the drain; outputs tid, tid + 512, ... in
//               the recombination);
//   warps 16-23 producers: thread (column c, 8-row octet o; lanes along c) splits 8 entries
//               of each round (2048 / BB rows) into digits and stores them in
//               both operand layouts (the B layout is the A layout's rows
//               regrouped by output-column half);
//   warp 24     allocates TMEM; its lane 0 issues the MMAs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "split8.cuh"
#include "sweep_fp64.cuh"
#include "tc_umma.cuh"

namespace jsvd {

namespace {

constexpr int kEpiW = 16, kProdW0 = 16, kProdW = 8, kMmaW = 24;
constexpr int kGThreadsTc = 32 * (kEpiW + kProdW + 1);  // 800
constexpr int kBarEpiG = 3;                            // named barrier of the epilogue warps
constexpr int kStageBytesTotal = 128 * 1024;           // operand stages
constexpr int kMaxRun = 32;                            // chunks whose level sums stay below 2^30

template <int BB> struct GramCfg {
    static constexpr int kSF = 128 / BB;               // slices stacked along M: 2, 4, 8
    static constexpr int kGroups = 8 / kSF;            // MMAs per K-step and half: 4, 2, 1
    static constexpr int kNH = BB == 64 ? 2 : 1;       // output-column halves
    static constexpr int kNC = BB / kNH;               // columns per half: 32, 32, 16
    static constexpr int kHalfCols = 8 * kNC;          // TMEM columns of a half
    static constexpr int kTmemCols = kNH * kHalfCols;  // 512, 256, 128
    static constexpr int kABytes = kGroups * 4096;     // A operand of a K-step
    static constexpr int kBHalf = 8 * kNC * 32;        // B operand of a K-step and half
    static constexpr int kStage = kABytes + kNH * kBHalf;             // 32, 16, 8 KB
    static constexpr int kSlots = kStageBytesTotal / kStage;          // 4, 8, 16 K-steps
    static constexpr int kKSteps = kGramRowsSplit / 16;               // 16 per unit
    static constexpr int kOct = 256 / BB;              // 8-row octets per producer round: 4, 8, 16
    static constexpr int kRoundRows = 8 * kOct;        // 32, 64, 128
    static constexpr int kRoundKS = kRoundRows / 16;   // 2, 4, 8
    static constexpr int kRounds = kGramRowsSplit / kRoundRows;       // 8, 4, 2
    static constexpr int kPk = BB * (BB + 1) / 2;      // outputs (packed lower triangle)
    static constexpr int kTmemChunks = kTmemCols / 16; // 16-column TMEM loads of a unit: 32, 16, 8
    static constexpr int kOffLev = kStageBytesTotal;   // int [8][kPk]: the run's level sums
    static constexpr int kOffE = kOffLev + 8 * kPk * 4;    // int [BB]: the unit's column exponents (epilogue)
    static constexpr int kOffAcc = kOffE + BB * 4;     // double [kPk]: the run's sum over its flushes
    static constexpr int kOffBar = kOffAcc + kPk * 8;  // a_full[kSlots], a_empty[kSlots], d_full, d_empty, done
    static constexpr int kNumBars = 2 * kSlots + 3;
    static constexpr int kOffMisc = kOffBar + 8 * kNumBars;           // tmem base, abort flag
    static constexpr int kSmem = kOffMisc + 16;
    static_assert(kSlots % kRoundKS == 0, "a round's K-steps must not wrap the stage ring");
    static_assert(kSmem <= 227 * 1024, "shared memory");
};

__device__ __forceinline__ int gcol(int P, int Q, int b, int k) { return k < b ? P * b + k : Q * b + (k - b); }

// Bounded wait (the same contract as the update kernel's): a thread whose
// wait gives up, or that finds the CTA's abort flag set, becomes dead and
// skips all further waits and work, but still takes every named barrier.
struct GWaiter {
    volatile int *abort_flag;
    bool dead = false;
    __device__ __forceinline__ bool operator()(uint64_t *bar, uint32_t parity) {
        if (dead) return false;
        for (int round = 0; round < 64; ++round) {
            if (tc::mbar_wait(bar, parity, 32, 1000000)) return true;
            if (*abort_flag) break;
        }
        *abort_flag = 1;
        dead = true;
        return false;
    }
};


__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void bar_epi() {
    asm volatile("bar.sync %0, %1;" ::"n"(kBarEpiG), "n"(32 * kEpiW) : "memory");
}

// One slice of 8 K entries in both operand layouts.
#define JSVD_GSTORE(I)                                                                                   \
    {                                                                                                    \
        const uint4 d = make_uint4(split8::digit_pair<I>(z[0], z[1]), split8::digit_pair<I>(z[2], z[3]), \
                                   split8::digit_pair<I>(z[4], z[5]), split8::digit_pair<I>(z[6], z[7])); \
        *reinterpret_cast<uint4 *>(st + offA + (I) * (BB * 32)) = d;                                     \
        *reinterpret_cast<uint4 *>(st + offB + (I) * (C::kNC * 32)) = d;                                 \
    }

template <int BB>
__global__ void __launch_bounds__(kGThreadsTc, 1) gram_tc(PStepArgs a) {
    using C = GramCfg<BB>;
    extern __shared__ __align__(1024) unsigned char sm[];
    int *lev = reinterpret_cast<int *>(sm + C::kOffLev);
    int *ecx = reinterpret_cast<int *>(sm + C::kOffE);
    double *accp = reinterpret_cast<double *>(sm + C::kOffAcc);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + C::kOffBar);
    uint64_t *a_full = bars, *a_empty = bars + C::kSlots;
    uint64_t *d_full = bars + 2 * C::kSlots, *d_empty = d_full + 1, *done = d_full + 2;
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(sm + C::kOffMisc);
    volatile int *s_abort = reinterpret_cast<volatile int *>(sm + C::kOffMisc + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // ---- set-up ---------------------------------------------------------------
    if (warp == kMmaW) tc::tmem_alloc(s_tmem, C::kTmemCols);
    if (tid == 0) {
        for (int i = 0; i < C::kSlots; ++i) {
            tc::mbar_init(&a_full[i], kProdW / C::kRoundKS);   // the warps that write one K-step
            tc::mbar_init(&a_empty[i], 1);
        }
        tc::mbar_init(d_full, 1);
        tc::mbar_init(d_empty, kEpiW);
        tc::mbar_init(done, 1);
        *s_abort = 0;
        mbar_init_fence();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *s_tmem;

    const long long units = (long long)a.npairs * a.g_chunks;
    const long long u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
    const double *G = reinterpret_cast<const double *>(a.G);

    if (warp == kMmaW) {
        // ---------------- MMA issue (one thread) ----------------------------------
        if (lane == 0) {
            GWaiter wait{s_abort};
            bool issued = false;
            for (long long u = u0; u < u1; ++u) {
                const int ju = (int)(u - u0);
                if (ju >= 1) wait(d_empty, (uint32_t)((ju - 1) & 1));
                for (int ks = 0; ks < C::kKSteps; ++ks) {
                    const int s = ju * C::kKSteps + ks, slot = s % C::kSlots, use = s / C::kSlots;
                    wait(&a_full[slot], (uint32_t)(use & 1));
                    if (wait.dead) continue;
                    tc::fence_after_sync();
                    const uint32_t sa = tc::smem_addr(sm + slot * C::kStage);
#pragma unroll
                    for (int h = 0; h < C::kNH; ++h)
#pragma unroll
                        for (int g = 0; g < C::kGroups; ++g)
                            tc::mma_bf16(tbase + (uint32_t)(h * C::kHalfCols + C::kNC * g * C::kSF),
                                         tc::smem_desc(sa + 4096u * g),
                                         tc::smem_desc(sa + (uint32_t)(C::kABytes + h * C::kBHalf)),
                                         tc::idesc_bf16(128, C::kNC * (8 - g * C::kSF)), ks > 0 || g > 0);
                    issued = true;
                    tc::mma_commit(&a_empty[slot]);
                }
                if (!wait.dead) tc::mma_commit(d_full);
            }
            if (issued) {
                // nothing may still write TMEM when it is freed (<= ~2 s)
                tc::mma_commit(done);
                tc::mbar_wait(done, 0, 2048, 1000000);
            }
        }
        __syncwarp();
    } else if (warp >= kProdW0) {
        // ---------------- producers ----------------------------------------------
        const int pt = tid - 32 * kProdW0;
        // consecutive lanes take consecutive columns of one octet, so the 8 lanes
        // of a 16-byte store phase fill one 128-byte row chunk (no bank conflicts)
        const int c = pt % BB, o = pt / BB;
        const int ksr = o >> 1, kk = (o & 1) * 8;
        const uint32_t offA = (uint32_t)(ksr * C::kStage) + tc::op_offset(c, kk);
        const uint32_t offB = (uint32_t)(ksr * C::kStage + C::kABytes + (c / C::kNC) * C::kBHalf) +
                              tc::op_offset(c % C::kNC, kk);
        GWaiter wait{s_abort};
        // the 8 entries of this thread in round rd of unit u
        auto src_of = [&](long long u, int rd) {
            const int uu = (int)u, pair = uu / a.g_chunks, chunk = uu - pair * a.g_chunks;
            const int P = a.table[2 * (a.step * a.npairs + pair)];
            const int Q = a.table[2 * (a.step * a.npairs + pair) + 1];
            return G + (size_t)gcol(P, Q, a.b, c) * a.ldg + (size_t)chunk * kGramRowsSplit +
                   (size_t)rd * C::kRoundRows + 8 * o;
        };
        double2 cur[4], nxt[4];
        if (u0 < u1) {
            const double *p = src_of(u0, 0);
#pragma unroll
            for (int v = 0; v < 4; ++v) cur[v] = *reinterpret_cast<const double2 *>(p + 2 * v);
        }
        for (long long u = u0; u < u1; ++u) {
            const int ju = (int)(u - u0);
            int E;
            {
                const int pair = (int)(u / a.g_chunks);
                const int P = a.table[2 * (a.step * a.npairs + pair)];
                const int Q = a.table[2 * (a.step * a.npairs + pair) + 1];
                E = a.gexp[gcol(P, Q, a.b, c)];
                if (E == split::kNoExp) E = 0;
            }
            for (int rd = 0; rd < C::kRounds; ++rd) {
                // the next round's entries into registers, the one after into L2
                const bool more = rd + 1 < C::kRounds || u + 1 < u1;
                if (more) {
                    const double *p = rd + 1 < C::kRounds ? src_of(u, rd + 1) : src_of(u + 1, 0);
#pragma unroll
                    for (int v = 0; v < 4; ++v) nxt[v] = *reinterpret_cast<const double2 *>(p + 2 * v);
                }
                // two rounds ahead into L2, across the unit boundary as well
                if (rd + 2 < C::kRounds)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(src_of(u, rd + 2)));
                else if (u + 1 < u1)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(src_of(u + 1, rd + 2 - C::kRounds)));
                const int s0 = ju * C::kKSteps + rd * C::kRoundKS;
                const int slot0 = s0 % C::kSlots, use = s0 / C::kSlots;
                if (use >= 1) wait(&a_empty[slot0 + ksr], (uint32_t)((use - 1) & 1));
                if (!wait.dead) {
                    unsigned long long z[8];
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        z[2 * v] = split8::fixed_biased(cur[v].x, 0, E);
                        z[2 * v + 1] = split8::fixed_biased(cur[v].y, 0, E);
                    }
                    unsigned char *st = sm + slot0 * C::kStage;
                    JSVD_GSTORE(0) JSVD_GSTORE(1) JSVD_GSTORE(2) JSVD_GSTORE(3)
                    JSVD_GSTORE(4) JSVD_GSTORE(5) JSVD_GSTORE(6) JSVD_GSTORE(7)
                    tc::fence_proxy_async();
                }
                __syncwarp();
                // a warp's lanes share one octet pair, hence one K-step of the round
                if (lane == 0 && !wait.dead) tc::mbar_arrive(&a_full[slot0 + ksr]);
                if (more) {
#pragma unroll
                    for (int v = 0; v < 4; ++v) cur[v] = nxt[v];
                }
            }
        }
    } else {
        // ---------------- epilogue (warps 0-15) -----------------------------------
        // Every chunk of a pair has the same column scales, so the level sums
        // of a CTA's consecutive chunks of one pair add up exactly as
        // integers: the drain adds each unit's TMEM parts into lev (shared
        // memory) and frees the accumulators at once; the recombination runs
        // once per run of chunks (at most kMaxRun: per unit |lev_L| <=
        // 7 * 2^22, as only 6 of a level's 8 digit products reach 2^14 per
        // row, so kMaxRun units stay below 2^30, combine_levels' range).
        const int q = warp & 3, cg = warp >> 2;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        const int ln = 32 * q + lane, s_ln = ln / BB, c_ln = ln % BB;
        // warp-uniform bounds of the lanes' stack slice and column
        const int s_min = (32 * q) / BB, c_max = BB >= 32 ? (32 * q) % BB + 31 : BB - 1;
        GWaiter wait{s_abort};
        for (int k = tid; k < C::kPk; k += 32 * kEpiW) accp[k] = 0.0;
        for (int k = tid; k < 8 * C::kPk; k += 32 * kEpiW) lev[k] = 0;
        int run_len = 0;
        for (long long u = u0; u < u1; ++u) {
            const int ju = (int)(u - u0);
            const int pair = (int)(u / a.g_chunks);
            const int P = a.table[2 * (a.step * a.npairs + pair)];
            const int Q = a.table[2 * (a.step * a.npairs + pair) + 1];
            bar_epi();      // the previous flush has read ecx and cleared lev
            for (int k = tid; k < BB; k += 32 * kEpiW) {
                const int e = a.gexp[gcol(P, Q, a.b, k)];
                ecx[k] = e == split::kNoExp ? 0 : e;
            }
            wait(d_full, (uint32_t)(ju & 1));
            tc::fence_after_sync();
            if (!wait.dead) {
                // drain: 16-column loads cg, cg + 4, ... of this quadrant's lanes;
                // lane (s, c) and column (half h, block j, n') hold a part of
                // level j + s of output (c, h NC + n'), kept for c >= n, level <= 7
#pragma unroll 1
                for (int k16 = cg; k16 < C::kTmemChunks; k16 += 4) {
                    const int col0 = 16 * k16;
                    const int h = col0 / C::kHalfCols, j = (col0 % C::kHalfCols) / C::kNC;
                    const int n_lo = h * C::kNC + col0 % C::kNC;
                    if (s_min + j > 7 || c_max < n_lo) continue;      // nothing kept (warp-uniform)
                    uint32_t v[16];
                    tc::tmem_ld16(tbase + lane_base + (uint32_t)col0, v);
                    tc::tmem_ld_wait();
                    const int L = j + s_ln, c = c_ln;
                    if (L <= 7) {
                        int *lv = lev + L * C::kPk;
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int n = n_lo + e;
                            if (c >= n) atomicAdd(lv + packed_lower<BB>(c, n), __float2int_rn(__uint_as_float(v[e])));
                        }
                    }
                }
            }
            // every TMEM read of this unit is done: the next unit's MMAs may start
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0 && !wait.dead) tc::mbar_arrive(d_empty);
            ++run_len;
            // the last of this CTA's consecutive chunks of the pair: write the
            // run's sum to the pair's slot (blockIdx.x minus the first CTA that
            // holds a chunk of the pair); the CTA holding the pair's last chunk
            // also zeroes the slots no CTA writes
            const bool run_end = u + 1 == u1 || (int)((u + 1) / a.g_chunks) != pair;
            if (run_end || run_len == kMaxRun) {
                bar_epi();      // every level addition of the drain is done
                const long long G = gridDim.x, first_u = (long long)pair * a.g_chunks;
                const int b0 = (int)(((first_u + 1) * G + units - 1) / units) - 1;
                const int slot = (int)blockIdx.x - b0;
                double *out = a.part + ((size_t)pair * a.g_parts + slot) * Cfg<BB>::kPacked;
                for (int k = tid; k < C::kPk; k += 32 * kEpiW) {
                    int n = 0, off = 0;     // (cc, n) of packed index k
                    while (k >= off + BB - n) {
                        off += BB - n;
                        ++n;
                    }
                    const int cc = n + (k - off);
                    int l[split8::kSlices];
#pragma unroll
                    for (int L = 0; L < split8::kSlices; ++L) {
                        l[L] = lev[L * C::kPk + k];
                        lev[L * C::kPk + k] = 0;
                    }
                    const double v = wait.dead ? 0.0 : __dadd_rn(accp[k], split8::combine_levels(l, ecx[cc] + ecx[n]));
                    if (run_end) {
                        out[k] = v;
                        accp[k] = 0.0;
                    } else {
                        accp[k] = v;
                    }
                }
                if (run_end && u == first_u + a.g_chunks - 1)
                    for (int k = tid; k < (a.g_parts - slot - 1) * C::kPk; k += 32 * kEpiW) out[C::kPk + k] = 0.0;
                run_len = 0;
            }
        }
    }

    // ---- teardown -------------------------------------------------------------
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0 && *s_abort) atomicOr(&a.counters[kCntErr], 4ull);
    if (warp == kMmaW) tc::tmem_dealloc(tbase, C::kTmemCols);
}
#undef JSVD_GSTORE

int grid_for(long long units) {
    static int nsm[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && nsm[dev] == 0) cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev);
    const int g = (dev >= 0 && dev < 64 && nsm[dev] > 0) ? nsm[dev] : 148;
    return units < g ? (int)units : g;
}

template <int BB>
void launch_gram_tc_bb(const PStepArgs &a, cudaStream_t s) {
    static int nsm[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && nsm[dev] == 0) {
        cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(gram_tc<BB>, cudaFuncAttributeMaxDynamicSharedMemorySize, GramCfg<BB>::kSmem);
    }
    const long long units = (long long)a.npairs * a.g_chunks;
    if (units <= 0) return;
    gram_tc<BB><<<grid_for(units), kGThreadsTc, GramCfg<BB>::kSmem, s>>>(a);
}

}  // namespace

int gram_tc_parts(const PStepArgs &a) {
    // CTA b holds units [units b / G, units (b + 1) / G); the CTA holding unit
    // x is ceil((x + 1) G / units) - 1
    const long long units = (long long)a.npairs * a.g_chunks;
    if (units <= 0) return a.g_chunks;
    const long long G = grid_for(units);
    int parts = 1;
    for (int p = 0; p < a.npairs; ++p) {
        const long long f = (long long)p * a.g_chunks, l = f + a.g_chunks - 1;
        const long long bf = ((f + 1) * G + units - 1) / units - 1, bl = ((l + 1) * G + units - 1) / units - 1;
        parts = (int)std::max<long long>(parts, bl - bf + 1);
    }
    return parts;
}

void launch_gram_tc(int BB, const PStepArgs &a, cudaStream_t s) {
    switch (BB) {
        case 16: launch_gram_tc_bb<16>(a, s); break;
        case 32: launch_gram_tc_bb<32>(a, s); break;
        case 64: launch_gram_tc_bb<64>(a, s); break;
        default: break;
    }
}

}  // namespace jsvd
