// Float-float ("double-float") arithmetic on the FP32 pipe: a value is the
// unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, about
// 48 significant bits. The error-free transformations are Knuth's two-sum,
// Dekker's fast two-sum (|a| >= |b|) and the FMA-based exact product; the
// compound operations follow the "sloppy" double-double algorithms of Hida,
// Li and Bailey (2001): relative error a few units of 2^-48 except under
// cancellation, where the error stays a few units of 2^-48 of the operands.
// Every product that must stay unfused is written with fmaf explicitly.
#pragma once

namespace rt3d {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_of(float x) { return ff{x, 0.0f}; }

// nearest float-float of a double (the two FP32 conversions run on the FP64
// pipe: for per-voxel or per-step preprocessing, not per-segment work)
__device__ __forceinline__ ff ff_split(double x) {
    const float h = __double2float_rn(x);
    return ff{h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = a + b;
    const float v = s - a;
    return ff{s, (a - (s - v)) + (b - v)};
}

__device__ __forceinline__ ff quick_two_sum(float a, float b) {
    const float s = a + b;
    return ff{s, b - (s - a)};
}

__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = a * b;
    return ff{p, fmaf(a, b, -p)};
}

__device__ __forceinline__ ff ff_neg(ff x) { return ff{-x.hi, -x.lo}; }

__device__ __forceinline__ ff ff_add(ff x, ff y) {
    const ff s = two_sum(x.hi, y.hi);
    return quick_two_sum(s.hi, s.lo + (x.lo + y.lo));
}

__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

__device__ __forceinline__ ff ff_add_f(ff x, float y) {
    const ff s = two_sum(x.hi, y);
    return quick_two_sum(s.hi, s.lo + x.lo);
}

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    const ff p = two_prod(x.hi, y.hi);
    return quick_two_sum(p.hi, fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo)));
}

__device__ __forceinline__ ff ff_mul_f(ff x, float y) {
    const ff p = two_prod(x.hi, y);
    return quick_two_sum(p.hi, fmaf(x.lo, y, p.lo));
}

// x * y + z
__device__ __forceinline__ ff ff_fma(ff x, ff y, ff z) {
    const ff p = two_prod(x.hi, y.hi);
    const float e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo));
    const ff s = two_sum(p.hi, z.hi);
    return quick_two_sum(s.hi, s.lo + (e + z.lo));
}

// exact scaling by a power of two (no overflow or underflow in range)
__device__ __forceinline__ ff ff_scale(ff x, float p2) { return ff{x.hi * p2, x.lo * p2}; }

// 1/x for x > 0: FP32 reciprocal r, then one Newton-Raphson step
// r + r (1 - x r) with the residual 1 - x r formed exactly enough in
// float-float (it is ~2^-23, so its FP32 product with r adds < 2^-46).
__device__ __forceinline__ ff ff_recip(ff x) {
    const float r = __frcp_rn(x.hi);
    const ff xr = ff_mul_f(x, r);
    const ff e = ff_sub(ff_of(1.0f), xr);
    return quick_two_sum(r, r * e.hi);
}

// FP64 value of a float-float (the widening of each part is exact; the sum
// rounds once, on the FP64 pipe)
__device__ __forceinline__ double ff_to_double(ff x) { return (double)x.hi + (double)x.lo; }

}  // namespace rt3d
