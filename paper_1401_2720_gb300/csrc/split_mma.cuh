// FP64-accurate contractions on the bf16 tensor cores (mma.sync m16n8k16).
//
// The block p-step's two dense contractions -- the Gram matrix of a pivot
// block-column pair (Eq. (2.7)) and the block update [A_P A_Q] V' (Eq. (2.9))
// -- are FP64 products.  This GPU issues one FP64 warp instruction per 64
// cycles per SM sub-partition, while its bf16 tensor cores multiply ~500x
// faster, so the products are formed exactly from small integer pieces:
//
//  * Fixed point.  Every operand row of A (resp. column of B) along the
//    contraction gets a power-of-two scale 2^E with |x| < 2^E, and each entry
//    becomes the integer Y = trunc(x 2^(62-E)), |Y| < 2^62 (integer shifts of
//    the significand; no rounding other than the truncation).
//  * Digits.  Y is written in balanced base 128 with kSlices = 9 digits
//    d_0..d_8, d_i in [-64, 64], Y = sum_i d_i 128^(8-i): add the bias
//    sum_k 64*128^k and read 7-bit fields.  Every digit is an exact bf16.
//  * Levels.  sum_j Y_A Y_B = sum_{i,l} (sum_j a_i b_l) 128^(16-i-l).  The
//    terms with i + l = L are accumulated by the tensor cores into one FP32
//    accumulator per level L <= 8; every partial sum is an integer below
//    9 * 128 * 64^2 < 2^23, so FP32 accumulation is exact.  Terms with
//    i + l > 8 are below 2^-54 of the scale and are dropped.
//  * Recombination.  The 9 exact level values are combined in 64-bit
//    integers (hi = levels 0..4, lo = levels 5..8) and turned into one FP64
//    number with a single rounding, then scaled by 2^(E_A + E_B - 40).
//
// The result's error is at most a few units in the last place of the scale
// product |row max| |column max|; with the column scaling D applied by the
// callers (powers of two, exact) this is at or below the rounding error of an
// FP64 FMA contraction of the same length.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace jsvd {
namespace split {

constexpr int kSlices = 9;                  // digits per value
constexpr int kLevels = kSlices;            // levels kept: i + l <= 8
constexpr int kPad = 8;                     // bf16 row padding in shared memory (16 B)
// sum_{k=0}^{8} 64 * 128^k: adding it makes every base-128 digit non-negative
constexpr unsigned long long bias_of(int k) { return k < 0 ? 0ull : (64ull << (7 * k)) + bias_of(k - 1); }
constexpr unsigned long long kBias = bias_of(kSlices - 1);
static_assert(kBias == 0x4081020408102040ull, "digit bias");
constexpr int kNoExp = -4096;               // exponent bound of an all-zero row or column

// Unbiased exponent ex and 53-bit significand of a finite double:
// |x| = mant * 2^(ex - 52).
__device__ __forceinline__ int exp_of(double x) {
    const long long bits = __double_as_longlong(x);
    const int ef = (int)((bits >> 52) & 0x7ff);
    return ef ? ef - 1023 : -1022;
}

// Exponent bound used for the scale: |x * 2^off| < 2^(result), or kNoExp for x = 0.
__device__ __forceinline__ int exp_bound(double x, int off) {
    const long long bits = __double_as_longlong(x) & 0x7fffffffffffffffll;
    if (bits == 0) return kNoExp;
    return exp_of(x) + off + 1;
}

// The biased fixed-point value Z = kBias + trunc(x 2^(off + 62 - E)) of x,
// given |x 2^off| < 2^E.  0 <= Z < 2^64.
__device__ __forceinline__ unsigned long long fixed_biased(double x, int off, int E) {
    const long long bits = __double_as_longlong(x);
    const int ef = (int)((bits >> 52) & 0x7ff);
    unsigned long long mant = (unsigned long long)bits & 0x000fffffffffffffull;
    int ex = -1022;
    if (ef) {
        mant |= 0x0010000000000000ull;
        ex = ef - 1023;
    }
    const int sh = ex + off - E + 10;    // <= 9 because |x 2^off| < 2^E
    unsigned long long y;
    if (sh >= 0)
        y = mant << sh;
    else
        y = sh > -64 ? (mant >> (-sh)) : 0ull;
    return bits < 0 ? kBias - y : kBias + y;
}

// The biased digit u_i of Z: u_0 = Z >> 56 in [0, 128], u_i = bits [56-7i,
// 63-7i) in [0, 127]; the digit is u_i - 64.
template <int I>
__device__ __forceinline__ uint32_t digit_field(unsigned long long z) {
    return I == 0 ? (uint32_t)(z >> 56) : (uint32_t)((z >> (56 - 7 * I)) & 127ull);
}

// Digit I of z0 (low half) and of z1 (high half) as two exact bf16 values in
// one 32-bit word: 0x4300 | u is the bf16 pattern of 128 + u for u in
// [0, 128] (u = 128 carries into the exponent: 0x4380 = 256), and one
// bf16x2 FMA subtracts 192 from both halves exactly.
template <int I>
__device__ __forceinline__ uint32_t digit_pair(unsigned long long z0, unsigned long long z1) {
    const uint32_t biased = __byte_perm(digit_field<I>(z0), digit_field<I>(z1), 0x5410) | 0x43004300u;
    uint32_t d;
    asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(biased), "r"(0x3F803F80u), "r"(0xC340C340u));
    return d;
}

// ---------------------------------------------------------------------------
// Warp-level tile: lev[L][e] += sum over K of the level-L digit products for a
// 16 x 16 output tile (two n8 halves, 4 accumulators each, mma layout).
//   As: digits of A, slice i at As + i * a_slice, row r (M) at + r * a_ld, K contiguous
//   Bs: digits of B, slice l at Bs + l * b_slice, row n (N) at + n * b_ld, K contiguous
// Both pointers are already offset to the tile's first row and first k.
// KSTEPS k16 steps starting at k = 0.
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int KSTEPS>
__device__ __forceinline__ void tile_levels(const uint16_t *As, int a_ld, int a_slice, const uint16_t *Bs, int b_ld,
                                            int b_slice, float (&lev)[kLevels][8]) {
    const int lane = threadIdx.x & 31;
    // ldmatrix row addresses: A tile rows lane%16, k offset 8*(lane/16);
    // B: n = lane%8 + 8*(lane/16), k offset 8*((lane/8)%2)
    const uint32_t a0 = smem_u32(As + (lane & 15) * a_ld + 8 * (lane >> 4));
    const uint32_t b0 = smem_u32(Bs + ((lane & 7) + 8 * (lane >> 4)) * b_ld + 8 * ((lane >> 3) & 1));
#pragma unroll 1
    for (int ks = 0; ks < KSTEPS; ++ks) {
        uint32_t bf[kSlices][4];
#pragma unroll
        for (int l = 0; l < kSlices; ++l)
            ldsm_x4(b0 + 2u * (uint32_t)(l * b_slice + 16 * ks), bf[l][0], bf[l][1], bf[l][2], bf[l][3]);
        // A digit fragments double-buffered: slice i + 1 is requested before the
        // MMAs of slice i are issued
        uint32_t af[2][4];
        ldsm_x4(a0 + 2u * (uint32_t)(16 * ks), af[0][0], af[0][1], af[0][2], af[0][3]);
#pragma unroll
        for (int i = 0; i < kSlices; ++i) {
            if (i + 1 < kSlices)
                ldsm_x4(a0 + 2u * (uint32_t)((i + 1) * a_slice + 16 * ks), af[(i + 1) & 1][0], af[(i + 1) & 1][1],
                        af[(i + 1) & 1][2], af[(i + 1) & 1][3]);
#pragma unroll
            for (int l = 0; l < kSlices - i; ++l) {
                float(&d0)[4] = *reinterpret_cast<float(*)[4]>(&lev[i + l][0]);
                float(&d1)[4] = *reinterpret_cast<float(*)[4]>(&lev[i + l][4]);
                mma_bf16(d0, af[i & 1], bf[l][0], bf[l][1]);
                mma_bf16(d1, af[i & 1], bf[l][2], bf[l][3]);
            }
        }
    }
}

__device__ __forceinline__ void zero_levels(float (&lev)[kLevels][8]) {
#pragma unroll
    for (int L = 0; L < kLevels; ++L)
#pragma unroll
        for (int e = 0; e < 8; ++e) lev[L][e] = 0.0f;
}

// Output coordinates of accumulator e of this lane within the 16 x 16 tile.
__device__ __forceinline__ int acc_row(int e) { return ((threadIdx.x & 31) >> 2) + ((e & 2) ? 8 : 0); }
__device__ __forceinline__ int acc_col(int e) { return 2 * (threadIdx.x & 3) + (e & 1) + ((e & 4) ? 8 : 0); }

// r * 2^s for any s in [-2200, 2200], r finite (the rare path: r = 0, or a
// result outside the normal range).
static __device__ __noinline__ double scale_slow(double r, int s) {
    const int s1 = s / 2, s2 = s - s1;
    if (s1 < -1022 || s2 < -1022) return __dmul_rn(r, 0.0);
    return __dmul_rn(__dmul_rn(r, __longlong_as_double((long long)(s1 + 1023) << 52)),
                     __longlong_as_double((long long)(s2 + 1023) << 52));
}

// The FP64 value 2^(ea + eb - 40) * sum_L lev[L] 128^(4-L), rounded once.
// Level values are exact integers with |lev| < 2^23; with kSmall they are
// below 2^22 (contraction length <= 64), and the float -> int conversion is
// one FP32 add of 1.5 * 2^23 (the integer lands in the low significand bits)
// instead of a quarter-rate conversion instruction.
template <bool kSmall>
__device__ __forceinline__ double combine(const float (&lv)[kLevels], int ea, int eb) {
    int v[kLevels];
#pragma unroll
    for (int L = 0; L < kLevels; ++L)
        v[L] = kSmall ? __float_as_int(__fadd_rn(lv[L], 12582912.0f)) - 0x4B400000 : __float2int_rn(lv[L]);
    long long hi = v[0];
#pragma unroll
    for (int L = 1; L < 5; ++L) hi = hi * 128 + v[L];
    long long lo = v[5];
#pragma unroll
    for (int L = 6; L < kLevels; ++L) lo = lo * 128 + v[L];
    // |hi| < 2^48, |lo| < 2^45: exact through the 1.5 * 2^52 offset
    const double H = __longlong_as_double(0x4338000000000000ll + hi);
    const double Lo = __longlong_as_double(0x4338000000000000ll + lo);
    const double hm = __dsub_rn(H, 0x1.8p52 + 0x1.8p24);            // hi - 1.5 * 2^24, exact
    const double r = __fma_rn(Lo, 0x1p-28, hm);                      // hi + lo 2^-28, one rounding
    // scale by 2^s on the exponent field when r and the result are normal
    const int s = ea + eb - 40;
    const long long rb = __double_as_longlong(r);
    const int ef = (int)((rb >> 52) & 0x7ff);
    if (ef != 0 && ef + s >= 1 && ef + s <= 2046) return __longlong_as_double(rb + ((long long)s << 52));
    if ((rb << 1) == 0) return r;
    return scale_slow(r, s);
}

}  // namespace split
}  // namespace jsvd
