// Jacobi rotation arithmetic on the device (Sec. 4.3 and 4.3.1 of the paper).
//
// Every operation below is a single correctly rounded IEEE operation written
// with an explicit intrinsic, so the compiler cannot contract or reorder it:
// given the same (hpp, hqq, hpq) the parameters are bit-identical to any
// other correctly rounded evaluation of the same formulas.
#pragma once
#include <cuda_runtime.h>

namespace jsvd {

constexpr double kEps = 0x1p-53;            // eps = 2^-53 (App. A)
constexpr double kSqrt2OverEps = 0x1p27;    // sqrt(2/eps) = 2^27 exactly

struct Rot {
    double cs;   // cos (trig) or cosh (hyperbolic)
    double tn;   // tan or tanh
};

// Eqs. (4.3)-(4.6) with the cs_2 form of (4.6).  t = +1 (trigonometric) or
// t = -1 (hyperbolic).  For the hyperbolic case a |coth 2phi| <= 1 (which can
// only arise from rounding) is replaced by 5/4 with its sign kept; sgn(x) is
// copysign(1, x).
__device__ __forceinline__ Rot rot_params(double hpp, double hqq, double hpq, double t) {
    const double h = __dsub_rn(hqq, __dmul_rn(t, hpp));
    double ct2 = __dmul_rn(t, __ddiv_rn(h, __dmul_rn(2.0, hpq)));
    if (t < 0.0 && fabs(ct2) <= 1.0) ct2 = copysign(1.25, ct2);
    const double act2 = fabs(ct2);
    double act;
    if (act2 >= kSqrt2OverEps)
        act = __dmul_rn(2.0, act2);
    else if (t > 0.0 && act2 < __dsqrt_rn(kEps))
        act = __dadd_rn(act2, 1.0);
    else
        act = __dadd_rn(act2, __dsqrt_rn(__fma_rn(ct2, ct2, t)));
    Rot r;
    r.tn = copysign(__drcp_rn(act), ct2);
    r.cs = (act >= kSqrt2OverEps) ? 1.0 : __ddiv_rn(act, __dsqrt_rn(__fma_rn(act, act, t)));
    return r;
}

// Relative orthogonality test of Sec. 4.3 (subphase 2): no rotation when
// h_pq = 0 or |h_pq| < c(eps) * (sqrt(h_pp) * sqrt(h_qq)), c(eps) = eps*sqrt(nhat).
__device__ __forceinline__ bool needs_rotation(double hpp, double hqq, double hpq, double c_eps) {
    if (hpq == 0.0) return false;
    return !(fabs(hpq) < __dmul_rn(c_eps, __dmul_rn(__dsqrt_rn(hpp), __dsqrt_rn(hqq))));
}

// Eq. (4.1) (t = +1) or Eq. (4.2) (t = -1) on one row of a column pair:
// an FMA, then a multiply by cs unless cs == 1.
__device__ __forceinline__ void rot_apply(double &x, double &y, double t, const Rot &r) {
    const double xn = __fma_rn(t > 0.0 ? -r.tn : r.tn, y, x);
    const double yn = __fma_rn(r.tn, x, y);
    if (r.cs != 1.0) {
        x = __dmul_rn(r.cs, xn);
        y = __dmul_rn(r.cs, yn);
    } else {
        x = xn;
        y = yn;
    }
}

}  // namespace jsvd
