// The 8-bit digit form of the FP64-accurate block update on tcgen05
// (Eq. (2.9): [A_P A_Q] := [A_P A_Q] V').
//
// Same fixed point as the 7-bit form (split_mma.cuh): every row of the left
// operand and every column of the right one gets a power-of-two scale 2^E
// with |x| < 2^E and becomes Y = trunc(x 2^(62-E)), |Y| < 2^62.  Y is written
// in balanced base 256 with 8 digits d_0..d_7 in [-128, 127]:
// Z = Y + 0x8080808080808080 (all bytes biased by 128), d_i = byte(7-i) - 128,
// Y = sum_i d_i 256^(7-i); every digit is an exact bf16.  A product sum
//   sum_j Y_A Y_B = 2^56 T,  T = sum_{L<=7} lev_L 256^(7-L),
//   lev_L = sum_{i+l=L} sum_j a_i(j) b_l(j),
// keeps the 36 digit products with i + l <= 7 (the dropped ones are below
// 2^-59 of the scale product).  For a contraction of length K <= 64 every
// level sum is an integer of magnitude <= 8 * 64 * 128^2 = 2^23, so FP32
// accumulation in the tensor cores is exact; the 8 level accumulators of 64
// output columns fill the 512 TMEM columns exactly (9 levels of the 7-bit
// form would not fit).  T is recombined in integers and rounded once to FP64;
// the result is T 2^(E_A + E_B - 68).
//
// Right-factor image (written by the per-pair Jacobi kernel, copied whole
// into shared memory by the update kernel): for output-column half h (of NH,
// NC = BB / NH columns each) and K-step ks (16 inputs) a block of 8 * NC
// rows -- slice l's rows l*NC .. l*NC + NC - 1 hold output columns
// h*NC .. h*NC + NC - 1 -- of 16 bf16 each, in the no-swizzle K-major
// core-matrix layout of tc_umma.cuh; blocks ordered (ks, h).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "split_mma.cuh"
#include "tc_umma.cuh"

namespace jsvd {
namespace split8 {

constexpr int kSlices = 8;
constexpr unsigned long long kBias = 0x8080808080808080ull;

template <int BB> struct TcCfg {
    static constexpr int kKS = BB / 16;                 // K-steps of 16
    static constexpr int kNH = BB == 64 ? 2 : 1;        // output-column halves
    static constexpr int kNC = BB / kNH;                // columns per half: 32, 32, 16
    static constexpr int kDW = kSlices * kNC;           // TMEM columns of one accumulator set
    static constexpr int kTmemCols = 2 * kDW;           // two sets: 512, 512, 256
    static constexpr int kBBlock = kSlices * kNC * 32;  // bytes of one (ks, h) block
    static constexpr int kBBytes = kKS * kNH * kBBlock; // 16 BB^2
};

// bf16 elements of one version of a pair's right-factor image.
template <int BB>
constexpr int image_elems() { return TcCfg<BB>::kBBytes / 2; }

// Z = kBias + trunc(x 2^(off + 62 - E)), given |x 2^off| < 2^E.
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

// Digit I (0 = most significant) of z as an FP32 value: the byte is placed
// under the exponent of 2^23 (0x4B0000uu = 2^23 + u) and 2^23 + 128 is
// subtracted, both exact.
template <int I>
__device__ __forceinline__ float digit_f32(unsigned long long z) {
    constexpr int byte = 7 - I;
    const uint32_t w = byte >= 4 ? (uint32_t)(z >> 32) : (uint32_t)z;
    const uint32_t f = __byte_perm(w, 0x4B000000u, 0x7540u | (uint32_t)(byte & 3));
    return __fsub_rn(__uint_as_float(f), 8388736.0f);
}

// Digits I of z0 (low half) and z1 (high half) as one bf16x2 word (exact).
template <int I>
__device__ __forceinline__ uint32_t digit_pair(unsigned long long z0, unsigned long long z1) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(digit_f32<I>(z1)), "f"(digit_f32<I>(z0)));
    return d;
}

// The 8 slices of 8 consecutive K entries z[0..7] (one 16-byte row chunk of a
// core matrix per slice): dst points at slice 0's chunk, slices slice_stride
// bytes apart.
__device__ __forceinline__ void store_digits8(unsigned char *dst, int slice_stride, const unsigned long long (&z)[8]) {
#define JSVD_S8(I)                                                                                          \
    *reinterpret_cast<uint4 *>(dst + (I) * slice_stride) =                                                  \
        make_uint4(digit_pair<I>(z[0], z[1]), digit_pair<I>(z[2], z[3]), digit_pair<I>(z[4], z[5]),      \
                   digit_pair<I>(z[6], z[7]));
    JSVD_S8(0) JSVD_S8(1) JSVD_S8(2) JSVD_S8(3) JSVD_S8(4) JSVD_S8(5) JSVD_S8(6) JSVD_S8(7)
#undef JSVD_S8
}

// Level L of a length-64 contraction as an int.  The top digits d_0 lie in
// [-64, 64] (|Y| < 2^62) and the others in [-128, 127], so |lev_L| <= 2^22 for
// L <= 4 (for L = 4: 64 (2 * 64 * 128 + 3 * 128^2) = 2^22) and one FP32 add of
// 1.5 * 2^23 puts the integer into the low significand bits; levels 5..7 can
// reach 64 (2 * 64 * 128 + (L - 1) * 128^2) <= 1.75 * 2^22, beyond that
// trick's range, and take the exact conversion instruction.
__device__ __forceinline__ int level_int(float v, int L) {
    return L <= 4 ? __float_as_int(__fadd_rn(v, 12582912.0f)) - 0x4B400000 : __float2int_rn(v);
}

// The FP64 value 2^(e - 68) * T, T = sum_L lev[L] 256^(7-L), rounded once to
// nearest (ties to even).  Level values are ints, |lev| < 2^30 (a length-64
// contraction's FP32 levels through combine32, or the Gram's sums over
// several chunks), so hi = sum_{L<4} lev[L] 256^(3-L) and lo = sum_{L>=4}
// lev[L] 256^(7-L) are below 2^55 and T = H 2^32 + R0 with H = hi + floor(lo
// / 2^32), 0 <= R0 < 2^32.  |T| = M 2^32 + R (M < 2^56) is shifted right by
// k in {0, 8, 16, 24} bits, the least multiple of 8 that brings it below
// 2^64: X = floor(|T| / 2^k) then has at least 57 significant bits when
// k > 0, and the discarded bits are ORed into its last bit (rounding to
// odd), so the correctly rounded conversion of X to FP64 (nearest, ties to
// even) is |T| 2^-k rounded once to 53 bits -- at least 2 bits beyond the
// 53 kept and a sticky last bit decide the rounding as the exact value
// would.  The power of two 2^(k + e - 68) is added to the exponent field.
__device__ __forceinline__ double combine_levels(const int (&l)[kSlices], int e) {
    const long long hi = (long long)l[0] * 16777216ll + (long long)l[1] * 65536ll + (long long)l[2] * 256ll + l[3];
    const long long lo = (long long)l[4] * 16777216ll + (long long)l[5] * 65536ll + (long long)l[6] * 256ll + l[7];
    const long long H = hi + (lo >> 32);               // arithmetic: floor division by 2^32
    const uint32_t R0 = (uint32_t)(unsigned long long)lo;
    const bool neg = H < 0;
    // |T| = M 2^32 + R: for T < 0, -T = (-H - 1) 2^32 + (2^32 - R0), or (-H) 2^32 if R0 = 0
    const unsigned long long M =
        neg ? (R0 != 0u ? (unsigned long long)(~H) : (unsigned long long)(-H)) : (unsigned long long)H;
    const uint32_t R = neg ? 0u - R0 : R0;
    const uint32_t Mh = (uint32_t)(M >> 32);           // < 2^24
    const int k = (32 - __clz((int)Mh) + 7) & ~7;      // 0 if Mh = 0, else 8 ceil(bits(Mh) / 8)
    unsigned long long X = (M << (32 - k)) | (unsigned long long)(R >> k);
    X |= (R & ((1u << k) - 1u)) != 0u ? 1ull : 0ull;
    const double d = __ull2double_rn(X);                // the one rounding
    if (X == 0ull) return 0.0;
    const int s = k + e - 68;
    const int dh = __double2hiint(d);                   // d > 0: sign bit clear
    const int be = (dh >> 20) + s;
    const int sign = neg ? (int)0x80000000u : 0;
    if (be >= 1 && be <= 2046) return __hiloint2double(sign | (dh + s * 1048576), __double2loint(d));
    return split::scale_slow(neg ? -d : d, s);          // rare: outside the normal range
}

__device__ __forceinline__ double combine32(const float (&lv)[kSlices], int e) {
    int l[kSlices];
#pragma unroll
    for (int L = 0; L < kSlices; ++L) l[L] = level_int(lv[L], L);
    return combine_levels(l, e);
}

// Right-factor images of one pivot pair (see above): version 0 = D V' for
// [G_P G_Q] (D = diag(2^dx[j])), version 1 = V' for [V_P V_Q].  W is V' in
// shared memory (column-major, ld ldw); bexp[ver * BB + k] receives column
// k's exponent bound F_k.  Executed by NT threads.
template <int BB, int NT>
__device__ __forceinline__ void right_factor_image(const double *W, int ldw, const int *dx,
                                                   uint16_t *__restrict__ img, int *__restrict__ bexp) {
    using C = TcCfg<BB>;
    for (int t = threadIdx.x; t < 2 * BB; t += NT) {
        const int ver = t / BB, k = t % BB;
        const double *w = W + k * ldw;
        int F = split::kNoExp;
        for (int j = 0; j < BB; ++j) F = max(F, split::exp_bound(w[j], ver ? 0 : dx[j]));
        if (F == split::kNoExp) F = 0;
        bexp[ver * BB + k] = F;
        const int h = k / C::kNC, n = k % C::kNC;
        unsigned char *base = reinterpret_cast<unsigned char *>(img + (size_t)ver * image_elems<BB>());
        for (int j = 0; j < BB; j += 8) {
            unsigned long long z[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) z[u] = fixed_biased(w[j + u], ver ? 0 : dx[j + u], F);
            const int ks = j / 16, kk = j % 16;
            unsigned char *dst = base + (ks * C::kNH + h) * C::kBBlock + tc::op_offset(n, kk);
            store_digits8(dst, C::kNC * 32, z);
        }
    }
}

}  // namespace split8
}  // namespace jsvd
