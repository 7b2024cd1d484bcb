// FP64 per-point arithmetic of the formal solutions without Lambda*,
// shared by the Cartesian kernel (fs.cu) and the spherical one (sph.cu). The
// FP64 pipe is the bound, so everything that can leave it does: branch tests
// on the high word of non-negative doubles (integer compares), reciprocals
// seeded in FP32, widening by integer moves. The interval functions follow
// the construction documented at the top of fs.cu (Olson & Kunasz 1987
// weights; the update in difference form).
#pragma once
#include "fs_step.cuh"

namespace rt3d {

// Whether x < b for a double x >= 0 and a bound b > 0 whose low word is
// zero, given the high word of b: an unsigned compare of the high words, so
// a NaN of either sign (0 * Inf where a zero-opacity interval meets a zero
// one) counts as not below.
__device__ __forceinline__ bool hi_below(double x, int b_hi) {
    return (unsigned)__double2hiint(x) < (unsigned)b_hi;
}

// 1/x for x > 0. Seed: x truncated to FP32 by integer moves (for x and 1/x
// inside the FP32 normal range: exponent field 897..1148), its FP32
// reciprocal, widened back; then one third-order Newton-Raphson step
// r = r0 + r0 (e + e^2), e = 1 - x r0, which takes the seed's relative error
// (< 2^-21) to below 2^-63, so the result is within an ulp or so of 1/x.
// Outside that range (and for 0, Inf, NaN): IEEE division.
__device__ __forceinline__ double recip64(double x) {
    const unsigned hi = (unsigned)__double2hiint(x);
    if (((hi >> 20) & 0x7ffu) - 897u > 251u || (hi >> 31)) return 1.0 / x;
    const unsigned lo = (unsigned)__double2loint(x);
    const float xf = __uint_as_float(((hi - 0x38000000u) << 3) | (lo >> 29));
    const double r0 = widen_f32(__frcp_rn(xf));
    const double e = fma(-x, r0, 1.0);
    return fma(r0, fma(e, e, e), r0);
}

// Interval functions in FP64 (as interval(double)); for u < 1/2 p(u) =
// e2/u^3 is a degree-9 polynomial fitted to the exact function (least squares
// in relative error at 300 Chebyshev nodes of [0, 1/2]; FP64 Horner error
// 1.6e-16 relative, the rounding of its leading coefficient 1/3). ru = 1/u
// for u >= 1/2 (carried from the previous step, or computed here if CARRY is
// false). Returns e0, a, d for the update in difference form.
struct IntervalDE {
    double e0, a, d;
};
template <bool CARRY>
__device__ __forceinline__ IntervalDE interval64(double u, double ru) {
    IntervalDE r;
    if (hi_below(u, 0x3FE00000)) {
        double p = -3.4475018036590732e-09;
        p = fma(p, u, 4.9354831016668725e-08);
        p = fma(p, u, -5.507115670485655e-07);
        p = fma(p, u, 5.511310234105578e-06);
        p = fma(p, u, -4.9603140878306714e-05);
        p = fma(p, u, 3.9682539230545495e-04);
        p = fma(p, u, -2.777777777429071e-03);
        p = fma(p, u, 1.6666666666652976e-02);
        p = fma(p, u, -8.333333333333312e-02);
        p = fma(p, u, 3.333333333333333e-01);
        const double b = u * p;
        const double hu = 0.5 * u;
        const double a = fma(-hu, b, hu);
        r.e0 = fma(-u, a, u);
        r.a = a;
        r.d = a - b;
    } else {
        if (!CARRY) ru = recip64(u);
        const double e0 = 1.0 - exp(-u);
        const double a = fma(-e0, ru, 1.0);
        r.e0 = e0;
        r.a = a;
        r.d = fma(2.0, a, -e0) * ru;
    }
    return r;
}

}  // namespace rt3d
