// The block update of one p-step, [X_P X_Q] := [X_P X_Q] V' (Eq. (2.9)) for
// X = G and X = V, on the 5th-generation tensor cores (tcgen05.mma kind::f16,
// accumulators in tensor memory), FP64-accurate through the 8-bit digit form
// of split8.cuh.
//
// One persistent CTA per SM walks a contiguous range of the p-step's 128-row
// tiles (pairs with V' != I only; for each pair the tiles of G, then those of
// V).  Warp roles, synchronised only through shared-memory mbarriers:
//   warps 0-15  epilogue: warp w reads TMEM lanes 32(w%4)..+31 (= the tile's
//               rows) for a quarter of the output columns of a half (w/4),
//               recombines the 8 level sums of each output into one FP64 value
//               (32-bit integer arithmetic without data-dependent branches, one
//               rounding), stores it and tracks the exponent bounds of G's new
//               columns.  The recombination (~100 instructions per output) is
//               the kernel's largest cost, so it gets most of the warps;
//   warps 16-23 producers: thread (row r, column half) makes two passes over
//               its row's entries (L1/L2 resident after the first): the row's
//               exponent bound (max over the row, through shared memory), then
//               the 8 digit slices of its K-steps, 8 entries at a time.  The
//               first pass needs no stage, so it overlaps the MMAs still
//               reading the previous tile's stages;
//   warp 24     allocates TMEM; its lane 0 copies the pair's right-factor
//               image into shared memory (cp.async.bulk, when the pair
//               changes) and issues every tile's MMAs as its stages fill.
// Per tile and output-column half h (BB = 64: two halves of 32 columns;
// BB <= 32: one), for every K-step of 16 and slice i = 0..7 one MMA
//   D[32 (8 levels) ... ] += A_i (128 x 16) x [B_0 .. B_{7-i}]^T
// with N = NC (8 - i), written at TMEM column NC i, so level L = i + l lands
// in the columns NC L .. NC L + NC - 1.  Two accumulator sets alternate, so
// the epilogue of one half-tile overlaps the MMAs of the next.
#include <cuda_runtime.h>

#include <cstdint>

#include "split8.cuh"
#include "sweep_fp64.cuh"
#include "tc_umma.cuh"

namespace jsvd {

namespace {

constexpr int kEpiWarps = 16, kProdWarp0 = 16, kProdWarps = 8, kMmaWarp = kProdWarp0 + kProdWarps;
constexpr int kTcThreads = 32 * (kEpiWarps + kProdWarps + 1);    // 800
constexpr int kTileRows = 128;
constexpr int kBarProd = 1, kBarEpi = 2;                         // named barriers

template <int BB> struct UpdTc {
    using C = split8::TcCfg<BB>;
    static constexpr int kASlots = C::kNH == 2 ? C::kKS : 2 * C::kKS;
    static constexpr int kASlotBytes = split8::kSlices * 4096;   // 8 slices of 128 x 16 bf16
    static constexpr int kCPT = BB / 2;                          // columns per producer thread
    static constexpr int kAFullCount = BB == 16 ? 8 : 4;         // producer warps writing one slot
    static constexpr int kOffB = kASlots * kASlotBytes;
    static constexpr int kOffRexp = kOffB + C::kBBytes;          // int [2][128]
    static constexpr int kOffRmax = kOffRexp + 2 * 128 * 4;      // int [2][2][128]
    static constexpr int kOffFexp = kOffRmax + 4 * 128 * 4;      // int [BB]
    static constexpr int kOffCmax = kOffFexp + BB * 4;           // int [BB]
    static constexpr int kOffDx = kOffCmax + BB * 4;             // int [2][BB]: producers' column scales
    static constexpr int kOffBar = kOffDx + 2 * BB * 4;          // mbarriers (8-byte aligned)
    // a_full[kASlots], a_empty[kASlots], d_full[2], d_empty[2], r_full[2], r_empty[2], b_full, b_free
    static constexpr int kNumBars = 2 * kASlots + 10;
    static constexpr int kOffMisc = kOffBar + 8 * kNumBars;      // tmem base, abort flag, active count
    static constexpr int kOffPairs = kOffMisc + 16;              // int [npairs]
    static constexpr int kFixed = kOffPairs;
};

// At most one CTA per SM (the tensor memory of two would not fit for BB >= 32):
// the dynamic shared memory request is at least this.
constexpr int kMinSmem = 120 * 1024;

struct Bars {
    uint64_t *a_full, *a_empty, *d_full, *d_empty, *r_full, *r_empty, *b_full, *b_free;
};

__device__ __forceinline__ int tcol(int P, int Q, int b, int k) { return k < b ? P * b + k : Q * b + (k - b); }

// Bounded wait.  A thread whose wait gives up (or that finds the CTA's abort
// flag set) becomes dead: it skips all further waits and work but still runs
// every loop iteration and named barrier, so no thread is left waiting on it.
struct Waiter {
    volatile int *abort_flag;
    bool dead = false;
    __device__ __forceinline__ bool operator()(uint64_t *bar, uint32_t parity) {
        if (dead) return false;
        // up to ~2 s in suspended polls of at most 1 ms
        for (int round = 0; round < 64; ++round) {
            if (tc::mbar_wait(bar, parity, 32, 1000000)) return true;
            if (*abort_flag) break;
        }
        *abort_flag = 1;
        dead = true;
        return false;
    }
};

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            tc::smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(tc::smem_addr(bar))
        : "memory");
}

template <int BB>
__global__ void __launch_bounds__(kTcThreads, 1) update_tc(PStepArgs a) {
    using U = UpdTc<BB>;
    using C = split8::TcCfg<BB>;
    constexpr int KS = C::kKS, NH = C::kNH, NC = C::kNC, DW = C::kDW;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *As = sm;
    unsigned char *Bs = sm + U::kOffB;
    int *rexp = reinterpret_cast<int *>(sm + U::kOffRexp);
    int *rmax = reinterpret_cast<int *>(sm + U::kOffRmax);
    int *fexp = reinterpret_cast<int *>(sm + U::kOffFexp);
    int *cmax = reinterpret_cast<int *>(sm + U::kOffCmax);
    int *dxs = reinterpret_cast<int *>(sm + U::kOffDx);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + U::kOffBar);
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(sm + U::kOffMisc);
    volatile int *s_abort = reinterpret_cast<volatile int *>(sm + U::kOffMisc + 4);
    int *s_active = reinterpret_cast<int *>(sm + U::kOffMisc + 8);
    int *s_pairs = reinterpret_cast<int *>(sm + U::kOffPairs);
    Bars B{bars, bars + U::kASlots, bars + 2 * U::kASlots, bars + 2 * U::kASlots + 2, bars + 2 * U::kASlots + 4,
           bars + 2 * U::kASlots + 6, bars + 2 * U::kASlots + 8, bars + 2 * U::kASlots + 9};

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // ---- set-up ---------------------------------------------------------------
    if (warp == kMmaWarp) tc::tmem_alloc(s_tmem, C::kTmemCols);
    if (tid == 0) {
        for (int i = 0; i < U::kASlots; ++i) {
            tc::mbar_init(&B.a_full[i], U::kAFullCount);
            tc::mbar_init(&B.a_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&B.d_full[i], 1);
            tc::mbar_init(&B.d_empty[i], kEpiWarps);
            tc::mbar_init(&B.r_full[i], 4);     // the 4 producer warps of column half 0
            tc::mbar_init(&B.r_empty[i], kEpiWarps);
        }
        tc::mbar_init(B.b_full, 1);
        tc::mbar_init(B.b_free, 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        // the active pairs (V' != I) in pair order
        int cnt = 0;
        for (int base = 0; base < a.npairs; base += 32) {
            const int p = base + lane;
            const bool act = p < a.npairs && a.vflag[p] != 0;
            const unsigned m = __ballot_sync(0xffffffffu, act);
            if (act) s_pairs[cnt + __popc(m & ((1u << lane) - 1u))] = p;
            cnt += __popc(m);
        }
        if (lane == 0) *s_active = cnt;
    }
    for (int k = tid; k < BB; k += kTcThreads) cmax[k] = split::kNoExp;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *s_tmem;

    const int tG = a.g_rows / kTileRows;
    const int tV = a.V ? a.v_rows / kTileRows : 0;
    const int tpp = tG + tV;
    const long long total = (long long)(*s_active) * tpp;
    const long long t0 = total * blockIdx.x / gridDim.x, t1 = total * (blockIdx.x + 1) / gridDim.x;

    if (warp >= kProdWarp0) {
        // ---------------- producers and the MMA warp -----------------------------
        const int pt = tid - 32 * kProdWarp0;    // producers: 0 .. 255
        const int r = pt & 127, ch = pt >> 7;
        const int c0 = ch * U::kCPT;
        Waiter wait{s_abort};
        // tile t -> (pair, version, first row); X, ld of that version
        auto locate = [&](long long t, int &pair, int &ver, size_t &row0) {
            const int ord = (int)(t / tpp), rem = (int)(t % tpp);
            ver = rem >= tG ? 1 : 0;
            pair = s_pairs[ord];
            row0 = (size_t)(ver ? rem - tG : rem) * kTileRows;
        };
        // this thread's kCPT = b columns are one block-column (P for the first
        // half of the pivot block, Q for the second): consecutive, ld apart
        const double *src = nullptr;
        size_t ldx = 0;
        auto locate_src = [&](long long t) {
            int pair, ver;
            size_t row0;
            locate(t, pair, ver, row0);
            const int blk = a.table[2 * (a.step * a.npairs + pair) + ch];
            const double *X = reinterpret_cast<const double *>(ver ? a.V : a.G);
            ldx = (size_t)(ver ? a.ldv : a.ldg);
            src = X + (size_t)blk * U::kCPT * ldx + row0 + r;
        };
        // MMA issue state (lane 0 of warp kMmaWarp only)
        const bool issuer = warp == kMmaWarp && lane == 0;
        int m_cur = -1, m_loads = 0, m_frees = 0;
        bool m_issued = false;
        auto issue_tile = [&](long long t) {
            const int j = (int)(t - t0);
            const int ord = (int)(t / tpp), rem = (int)(t % tpp);
            const int ver = rem >= tG ? 1 : 0;
            const int item = 2 * ord + ver;
            if (item != m_cur) {
                if (m_cur >= 0) {
                    // every MMA reading the previous image has completed
                    tc::mma_commit(B.b_free);
                    wait(B.b_free, (uint32_t)(m_frees & 1));
                    ++m_frees;
                }
                if (!wait.dead) {
                    // the pair's images sit at the pair stride of the 7-bit layout
                    // (2 split_b_elems), version 1 after version 0
                    const uint16_t *src = a.bslice + (size_t)s_pairs[ord] * 2 * split_b_elems<BB>() +
                                          (size_t)ver * split8::image_elems<BB>();
                    mbar_expect_tx(B.b_full, C::kBBytes);
                    bulk_g2s(Bs, src, C::kBBytes, B.b_full);
                    wait(B.b_full, (uint32_t)(m_loads & 1));
                    ++m_loads;
                }
                m_cur = item;
            }
            for (int h = 0; h < NH; ++h) {
                const int u = j * NH + h, buf = u & 1;
                if (u >= 2) wait(&B.d_empty[buf], (uint32_t)(((u >> 1) - 1) & 1));
                tc::fence_after_sync();
                for (int ks = 0; ks < KS; ++ks) {
                    const int s = j * KS + ks, slot = s % U::kASlots, use = s / U::kASlots;
                    if (h == 0) wait(&B.a_full[slot], (uint32_t)(use & 1));
                    if (wait.dead) continue;
                    tc::fence_after_sync();
                    const uint32_t a0 = tc::smem_addr(As + slot * U::kASlotBytes);
                    const uint32_t b0 = tc::smem_addr(Bs + (ks * NH + h) * C::kBBlock);
                    const uint32_t d0 = tbase + (uint32_t)(buf * DW);
#pragma unroll
                    for (int i = 0; i < split8::kSlices; ++i)
                        tc::mma_bf16(d0 + (uint32_t)(NC * i), tc::smem_desc(a0 + 4096u * i), tc::smem_desc(b0),
                                     tc::idesc_bf16(128, NC * (split8::kSlices - i)), ks > 0 || i > 0);
                    m_issued = true;
                    if (h == NH - 1) tc::mma_commit(&B.a_empty[slot]);
                }
                if (!wait.dead) tc::mma_commit(&B.d_full[buf]);
            }
        };
        if (warp == kMmaWarp) {
            if (issuer) {
                for (long long t = t0; t < t1; ++t) issue_tile(t);
                if (m_issued) {
                    // drain: nothing may still write TMEM when it is freed (<= ~2 s)
                    tc::mma_commit(B.b_free);
                    tc::mbar_wait(B.b_free, (uint32_t)(m_frees & 1), 2048, 1000000);
                }
            }
            __syncwarp();
        } else for (long long t = t0; t < t1; ++t) {
            const int j = (int)(t - t0);
            int pair, ver;
            size_t row0;
            locate(t, pair, ver, row0);
            locate_src(t);
            // the column scales of this tile's version (0 for V)
            int *dx = dxs + (j & 1) * BB;
            for (int k = pt; k < BB; k += 32 * kProdWarps) dx[k] = ver ? 0 : a.dexp[(size_t)pair * BB + k];
            asm volatile("bar.sync %0, %1;" ::"n"(kBarProd), "n"(32 * kProdWarps) : "memory");
            // the next tile's entries of this thread into L2, so that neither
            // of its passes waits on HBM
            if (t + 1 < t1) {
                const double *cur = src;
                const size_t ldc = ldx;
                locate_src(t + 1);
#pragma unroll
                for (int c = 0; c < U::kCPT; ++c) asm volatile("prefetch.global.L2 [%0];" ::"l"(src + c * ldx));
                src = cur;
                ldx = ldc;
            }
            // first pass: the row's exponent bound over this thread's entries,
            // 16 loads in flight at a time
            int m = split::kNoExp;
            if (j == 0) {
#pragma unroll
                for (int c = 16; c < U::kCPT; ++c)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(src + c * ldx));
            }
#pragma unroll 1
            for (int c1 = 0; c1 < U::kCPT; c1 += 16) {
                constexpr int NG = U::kCPT < 16 ? U::kCPT : 16;
                double v[NG];
#pragma unroll
                for (int c = 0; c < NG; ++c) v[c] = src[(c1 + c) * ldx];
#pragma unroll
                for (int c = 0; c < NG; ++c) m = max(m, split::exp_bound(v[c], -dx[c0 + c1 + c]));
            }
            rmax[((j & 1) * 2 + ch) * 128 + r] = m;
            asm volatile("bar.sync %0, %1;" ::"n"(kBarProd), "n"(32 * kProdWarps) : "memory");
            int E = max(rmax[((j & 1) * 2) * 128 + r], rmax[((j & 1) * 2 + 1) * 128 + r]);
            if (E == split::kNoExp) E = 0;
            if (ch == 0) {
                if (j >= 2) wait(&B.r_empty[j & 1], (uint32_t)(((j >> 1) - 1) & 1));
                if (!wait.dead) {
                    rexp[(j & 1) * 128 + r] = E;
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&B.r_full[j & 1]);
                }
            }
            // the stages this thread writes must be free (the MMAs of the
            // previous tile read them while the first pass ran)
#pragma unroll
            for (int g = 0; g < U::kCPT / 8; ++g) {
                const int col = c0 + 8 * g;
                const int s = j * KS + col / 16, slot = s % U::kASlots, use = s / U::kASlots;
                if ((col % 16 == 0 || g == 0) && use >= 1) wait(&B.a_empty[slot], (uint32_t)((use - 1) & 1));
            }
            // second pass, 8 entries at a time; the next 8 are loaded before
            // this group's digits are stored (and its stage published)
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = src[u * ldx];
#pragma unroll
            for (int g = 0; g < U::kCPT / 8; ++g) {
                const int col = c0 + 8 * g;
                const int ks = col / 16, kk = col % 16;
                const int slot = (j * KS + ks) % U::kASlots;
                const bool last = kk == 8 || 8 * g + 8 == U::kCPT;
                unsigned long long z[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) z[u] = split8::fixed_biased(v[u], -dx[col + u], E);
                if (8 * g + 8 < U::kCPT) {
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[u] = src[(8 * g + 8 + u) * ldx];
                }
                if (wait.dead) continue;
                split8::store_digits8(As + slot * U::kASlotBytes + tc::op_offset(r, kk), 4096, z);
                if (last) {
                    tc::fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&B.a_full[slot]);
                }
            }
            __syncwarp();
        }
    } else {
        // ---------------- epilogue (warps 0-15: TMEM lane quadrant w % 4, column quarter w / 4) ----
        const int q = warp & 3, cg = warp >> 2;
        const int r = 32 * q + lane;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        constexpr int CW = NC / 4;              // columns of a half-tile per warp: 8, 8, 4
        int cur = -1, P = 0, Q = 0, ver = 0;
        double *X = nullptr;
        int ld = 0;
        Waiter wait{s_abort};
        auto flush = [&](int Pp, int Qp) {
            // the exponent bounds of the columns of G just written
            asm volatile("bar.sync %0, %1;" ::"n"(kBarEpi), "n"(32 * kEpiWarps) : "memory");
            for (int k = tid; k < BB; k += 32 * kEpiWarps) {
                if (cmax[k] != split::kNoExp) atomicMax(&a.gexp[tcol(Pp, Qp, a.b, k)], cmax[k]);
                cmax[k] = split::kNoExp;
            }
        };
        for (long long t = t0; t < t1; ++t) {
            const int j = (int)(t - t0);
            const int ord = (int)(t / tpp), rem = (int)(t % tpp);
            const int vnew = rem >= tG ? 1 : 0;
            const int tile = vnew ? rem - tG : rem;
            const int item = 2 * ord + vnew;
            if (item != cur) {
                if (cur >= 0 && ver == 0) flush(P, Q);
                const int pair = s_pairs[ord];
                ver = vnew;
                P = a.table[2 * (a.step * a.npairs + pair)];
                Q = a.table[2 * (a.step * a.npairs + pair) + 1];
                X = reinterpret_cast<double *>(ver ? a.V : a.G);
                ld = ver ? a.ldv : a.ldg;
                asm volatile("bar.sync %0, %1;" ::"n"(kBarEpi), "n"(32 * kEpiWarps) : "memory");
                for (int k = tid; k < BB; k += 32 * kEpiWarps) fexp[k] = a.bexp[((size_t)pair * 2 + ver) * BB + k];
                asm volatile("bar.sync %0, %1;" ::"n"(kBarEpi), "n"(32 * kEpiWarps) : "memory");
                cur = item;
            }
            wait(&B.r_full[j & 1], (uint32_t)((j >> 1) & 1));
            const int E = rexp[(j & 1) * 128 + r];
            __syncwarp();
            if (lane == 0 && !wait.dead) tc::mbar_arrive(&B.r_empty[j & 1]);
            const size_t row = (size_t)tile * kTileRows + r;
            for (int h = 0; h < NH; ++h) {
                const int u = j * NH + h, buf = u & 1;
                wait(&B.d_full[buf], (uint32_t)((u >> 1) & 1));
                if (wait.dead) continue;
                tc::fence_after_sync();
#pragma unroll 1
                for (int cc = cg * CW; cc < (cg + 1) * CW; cc += 2) {
                    uint32_t lv[split8::kSlices][2];
#pragma unroll
                    for (int L = 0; L < split8::kSlices; ++L)
                        tc::tmem_ld2(tbase + lane_base + (uint32_t)(buf * DW + NC * L + cc), lv[L]);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const int k = h * NC + cc + c;
                        float f[split8::kSlices];
#pragma unroll
                        for (int L = 0; L < split8::kSlices; ++L) f[L] = __uint_as_float(lv[L][c]);
                        const double y = split8::combine32(f, E + fexp[k]);
                        X[(size_t)tcol(P, Q, a.b, k) * ld + row] = y;
                        if (ver == 0) {
                            const int mx = __reduce_max_sync(0xffffffffu, split::exp_bound(y, 0));
                            if (lane == 0 && mx != split::kNoExp) atomicMax(&cmax[k], mx);
                        }
                    }
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&B.d_empty[buf]);
            }
        }
        if (cur >= 0 && ver == 0) flush(P, Q);
    }

    // ---- teardown -------------------------------------------------------------
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0 && *s_abort) atomicOr(&a.counters[kCntErr], 4ull);
    if (warp == kMmaWarp) tc::tmem_dealloc(tbase, C::kTmemCols);
}

template <int BB>
size_t update_tc_smem(int npairs) {
    const size_t s = (size_t)UpdTc<BB>::kFixed + 4 * (size_t)npairs;
    return s < (size_t)kMinSmem ? (size_t)kMinSmem : s;
}

template <int BB>
void launch_update_tc_bb(const PStepArgs &a, cudaStream_t s) {
    static int nsm[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const size_t smem = update_tc_smem<BB>(a.npairs);
    if (dev >= 0 && dev < 64 && nsm[dev] == 0) {
        cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(update_tc<BB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    }
    const int grid = (dev >= 0 && dev < 64 && nsm[dev] > 0) ? nsm[dev] : 148;
    update_tc<BB><<<grid, kTcThreads, smem, s>>>(a);
}

}  // namespace

size_t update_tc_smem_bytes(int BB, int npairs) {
    switch (BB) {
        case 16: return update_tc_smem<16>(npairs);
        case 32: return update_tc_smem<32>(npairs);
        default: return update_tc_smem<64>(npairs);
    }
}

void launch_update_tc(int BB, const PStepArgs &a, cudaStream_t s) {
    switch (BB) {
        case 16: launch_update_tc_bb<16>(a, s); break;
        case 32: launch_update_tc_bb<32>(a, s); break;
        case 64: launch_update_tc_bb<64>(a, s); break;
        default: break;
    }
}

}  // namespace jsvd
