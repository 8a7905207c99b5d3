// Jacobi rotation arithmetic on the device (Sec. 4.3 and 4.3.1 of the paper).
//
// Every floating-point operation below is a single correctly rounded IEEE
// operation written with an explicit intrinsic, so the compiler cannot
// contract or reorder it: given the same (hpp, hqq, hpq) the parameters are
// bit-identical to any other correctly rounded evaluation of the same
// formulas.  Comparisons of values that are known to be non-negative (absolute
// values, sums of squares) are done on their bit patterns, which order
// non-negative doubles exactly like the numbers: same results, and the FP64
// pipe (the scarce unit on this GPU) is left to the arithmetic.
#pragma once
#include <cuda_runtime.h>

namespace jsvd {

constexpr double kEps = 0x1p-53;                   // eps = 2^-53 (App. A)
constexpr double kSqrtEps = 0x1.6a09e667f3bcdp-27; // sqrt(2^-53), correctly rounded
constexpr double kSqrt2OverEps = 0x1p27;           // sqrt(2/eps) = 2^27 exactly

struct Rot {
    double cs;   // cos (trig) or cosh (hyperbolic)
    double tn;   // tan or tanh
};

// a < b for a, b >= +0 (no NaN)
__device__ __forceinline__ bool nonneg_lt(double a, double b) {
    return __double_as_longlong(a) < __double_as_longlong(b);
}

// Eqs. (4.3)-(4.6) with the cs_2 form of (4.6).  hyperbolic selects t = -1
// (Eq. (4.2)), else t = +1 (Eq. (4.1)).  For the hyperbolic case a
// |coth 2phi| <= 1 (which can only arise from rounding) is replaced by 5/4 with
// its sign kept; sgn(x) is copysign(1, x).
__device__ __forceinline__ Rot rot_params(double hpp, double hqq, double hpq, bool hyperbolic) {
    const double t = hyperbolic ? -1.0 : 1.0;
    const double h = hyperbolic ? __dadd_rn(hqq, hpp) : __dsub_rn(hqq, hpp);   // hqq - t*hpp
    double ct2 = __ddiv_rn(h, __dmul_rn(2.0, hpq));
    if (hyperbolic) ct2 = -ct2;                                              // t * (h / (2 hpq))
    const double act2 = fabs(ct2);
    if (hyperbolic && !nonneg_lt(1.0, act2)) ct2 = copysign(1.25, ct2);     // |ct2| <= 1
    const double a2 = fabs(ct2);
    double act;
    if (!nonneg_lt(a2, kSqrt2OverEps))                                      // |ct2| >= 2^27
        act = __dmul_rn(2.0, a2);
    else if (!hyperbolic && nonneg_lt(a2, kSqrtEps))
        act = __dadd_rn(a2, 1.0);
    else
        act = __dadd_rn(a2, __dsqrt_rn(__fma_rn(ct2, ct2, t)));
    Rot r;
    r.tn = copysign(__drcp_rn(act), ct2);
    r.cs = !nonneg_lt(act, kSqrt2OverEps) ? 1.0 : __ddiv_rn(act, __dsqrt_rn(__fma_rn(act, act, t)));
    return r;
}

// Relative orthogonality test of Sec. 4.3 (subphase 2): no rotation when
// h_pq = 0 or |h_pq| < c(eps) * (sqrt(h_pp) * sqrt(h_qq)), c(eps) = eps*sqrt(nhat),
// every operation correctly rounded.
__device__ __forceinline__ bool needs_rotation_exact(double hpp, double hqq, double hpq, double c_eps) {
    const double a = fabs(hpq);
    if (__double_as_longlong(a) == 0) return false;
    return !nonneg_lt(a, __dmul_rn(c_eps, __dmul_rn(__dsqrt_rn(hpp), __dsqrt_rn(hqq))));
}

// The same decision, mostly without the two square roots (each about eight
// FP64-pipe instructions, the scarce unit): with T the correctly rounded
// threshold above, T = c sqrt(h_pp h_qq) (1 + t), |t| <= 4u (u = 2^-53), and
// the squares compared in FP64, RN(a^2) = a^2 (1 + d1), RN(c^2 RN(h_pp h_qq))
// = c^2 h_pp h_qq (1 + d2), |d1| <= u, |d2| <= 3u (c^2 given correctly
// rounded), so a squared ratio outside [1 - m, 1 + m], m = 2^-48, decides
// a >= T or a < T for certain (m / 2 - 3u > 4u).  Inside that band, or when
// an exponent lies outside [-400, 400] (products could leave the normal
// range), the exact evaluation decides.  Bit-identical decisions.
__device__ __forceinline__ bool needs_rotation(double hpp, double hqq, double hpq, double c_eps, double c_eps2) {
    const double a = fabs(hpq);
    if (__double_as_longlong(a) == 0) return false;
    const int ea = (int)((__double_as_longlong(a) >> 52) & 0x7ff) - 1023;
    const int ep = (int)((__double_as_longlong(hpp) >> 52) & 0x7ff) - 1023;
    const int eq = (int)((__double_as_longlong(hqq) >> 52) & 0x7ff) - 1023;
    if (hpp > 0.0 && hqq > 0.0 && ea >= -400 && ea <= 400 && ep >= -400 && ep <= 400 && eq >= -400 &&
        eq <= 400) {
        const double lhs = __dmul_rn(a, a);
        const double rhs = __dmul_rn(c_eps2, __dmul_rn(hpp, hqq));
        if (lhs > __dmul_rn(rhs, 1.0 + 0x1p-48)) return true;
        if (lhs < __dmul_rn(rhs, 1.0 - 0x1p-48)) return false;
    }
    return needs_rotation_exact(hpp, hqq, hpq, c_eps);
}

// cs != 1 (cs > 0)
__device__ __forceinline__ bool is_proper(const Rot &r) {
    return __double_as_longlong(r.cs) != __double_as_longlong(1.0);
}

// Eq. (4.1) (trigonometric) or Eq. (4.2) (hyperbolic) on one row of a column
// pair: an FMA, then a multiply by cs unless cs == 1.
__device__ __forceinline__ void rot_apply(double &x, double &y, bool hyperbolic, const Rot &r) {
    const double xn = __fma_rn(hyperbolic ? r.tn : -r.tn, y, x);
    const double yn = __fma_rn(r.tn, x, y);
    if (is_proper(r)) {
        x = __dmul_rn(r.cs, xn);
        y = __dmul_rn(r.cs, yn);
    } else {
        x = xn;
        y = yn;
    }
}

// ---------------------------------------------------------------------------
// The same rotation in FP32 (the first stage of the mixed FP32 -> FP64 solver,
// whose sweeps only precondition the FP64 ones): Eqs. (4.3)-(4.6) with
// eps = 2^-24, so sqrt(eps) = 2^-12 and sqrt(2 / eps) = 2^12.5 (rounded to
// FP32), every operation a correctly rounded FP32 intrinsic.
constexpr float kSqrtEps32 = 0x1p-12f;
constexpr float kSqrt2OverEps32 = 5792.6187f;

struct RotF {
    float cs;
    float tn;
};

__device__ __forceinline__ RotF rot_params_f(float hpp, float hqq, float hpq, bool hyperbolic) {
    const float t = hyperbolic ? -1.0f : 1.0f;
    const float h = hyperbolic ? __fadd_rn(hqq, hpp) : __fsub_rn(hqq, hpp);
    float ct2 = __fdiv_rn(h, __fmul_rn(2.0f, hpq));
    if (hyperbolic) ct2 = -ct2;
    if (hyperbolic && !(fabsf(ct2) > 1.0f)) ct2 = copysignf(1.25f, ct2);
    const float a2 = fabsf(ct2);
    float act;
    if (a2 >= kSqrt2OverEps32)
        act = __fmul_rn(2.0f, a2);
    else if (!hyperbolic && a2 < kSqrtEps32)
        act = __fadd_rn(a2, 1.0f);
    else
        act = __fadd_rn(a2, __fsqrt_rn(__fmaf_rn(ct2, ct2, t)));
    RotF r;
    r.tn = copysignf(__frcp_rn(act), ct2);
    r.cs = act >= kSqrt2OverEps32 ? 1.0f : __fdiv_rn(act, __fsqrt_rn(__fmaf_rn(act, act, t)));
    return r;
}

__device__ __forceinline__ bool needs_rotation_f(float hpp, float hqq, float hpq, float c_eps) {
    const float a = fabsf(hpq);
    if (a == 0.0f) return false;
    return !(a < __fmul_rn(c_eps, __fmul_rn(__fsqrt_rn(hpp), __fsqrt_rn(hqq))));
}

}  // namespace jsvd
