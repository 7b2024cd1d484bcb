// Per-point arithmetic of the FP32 formal solution without Lambda*, shared
// by the single-problem kernel (fs.cu) and the batched-wavelength kernel
// (batch.cu). The interval functions and the update follow the construction
// documented at the top of fs.cu (Olson & Kunasz 1987 weights with the
// limited parabola; the update in difference form).
#pragma once
#include "rt3d_internal.cuh"

namespace rt3d {

// FP32 interval functions for the formal solution without Lambda*: e0, a
// and d of the interval of optical depth u (the update in difference form
// needs neither E nor a0). For u < 1, p(u) = e2/u^3 is a degree-5 polynomial
// fitted to the exact function (least squares in relative error at 200
// Chebyshev nodes of [0, 1]; FP32 Horner error 1.2e-7 relative, as for the
// 9-term Taylor series). For u >= 1 the caller passes ru = 1/u.
struct IntervalE {
    float e0, a, d;
};
__device__ __forceinline__ IntervalE interval_fast(float u, float ru) {
    IntervalE r;
    if (u < 1.0f) {
        float p = -3.569704858819023e-05f;
        p = fmaf(p, u, 3.819821577053517e-04f);
        p = fmaf(p, u, -2.770215505734086e-03f);
        p = fmaf(p, u, 1.6664894297719002e-02f);
        p = fmaf(p, u, -8.333317935466766e-02f);
        p = fmaf(p, u, 3.333333432674408e-01f);
        const float b = u * p;
        const float hu = 0.5f * u;
        const float a = fmaf(-hu, b, hu);
        r.e0 = fmaf(-u, a, u);
        r.a = a;
        r.d = a - b;
    } else {
        const float e0 = 1.0f - __expf(-u);
        const float a = fmaf(-e0, ru, 1.0f);
        r.e0 = e0;
        r.a = a;
        r.d = fmaf(2.0f, a, -e0) * ru;
    }
    return r;
}

// x as an FP64 value, by moving the fields of its IEEE binary32 encoding
// into binary64 with the exponent rebiased by 1023 - 127: exact for every
// normal x; a zero or subnormal x becomes +-2^-127 (1 + m 2^-23), below
// 1.2e-38 in magnitude. Infinities and NaNs are not preserved: the kernel
// below checks the intensity at the end of each characteristic instead
// (a non-finite value persists along the recurrence). Integer instructions
// only, where the conversion instruction would load the FP64 pipe.
__device__ __forceinline__ double widen_f32(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned lo = b << 29;
    const unsigned hi = (((b >> 3) & 0x0fffffffu) + 0x38000000u) | (b & 0x80000000u);
    return __hiloint2double((int)hi, (int)lo);
}

template <bool WIDEN> __device__ __forceinline__ double to_f64(float x) {
    if (WIDEN) return widen_f32(x);
    return (double)x;
}

// State of one characteristic: intensity, optical depth u of the interval
// ending at the current point (and 1/u), half optical depth of the current
// point's chord, S at the previous and current points and their difference,
// replicated offsets of the face cell and of the current point.
struct RayF {
    float I, u, ru, hc, Sp, Sc, dS;
    int base, vc;
    bool live;
};

// One point of the FP32 formal solution: gather the next point's (chi, S)
// (record rn: offset, l/2), update I at the current point with the
// difference form of the file header, add cwc I to J at the current point,
// advance. BRANCHLESS evaluates the parabolic correction also where its
// blend weight is 0 (no divergent branch).
template <bool PARAB, bool WIDEN, bool BRANCHLESS>
__device__ __forceinline__ void fast_step(RayF &s, const float2 *__restrict__ chiS,
                                          double *__restrict__ Jd, const float4 &rn, float cwc) {
    const int vn = s.base + __float_as_int(rn.x);
    const float2 cn = chiS[vn];
    const float hn = cn.x * rn.y;
    const float dSn = cn.y - s.Sc;
    const float w = s.hc + hn;
    // 1/w with w floored at 1e-30: a zero-opacity pair (w = 0) gives q = 0 or
    // a large finite q (blend weight 0) instead of Inf or NaN
    const float rw = __fdividef(1.0f, fmaxf(w, 1e-30f));
    const float u = s.u;
    const IntervalE f = interval_fast(u, PARAB ? s.ru : __fdividef(1.0f, u));
    float In = fmaf(f.e0, s.Sp - s.I, s.I);
    In = fmaf(f.a, s.dS, In);
    if (PARAB) {
        const float q = u * rw;
        const float fw = __saturatef(fmaf(-2.0f, u, 2.0f)) * __saturatef(fmaf(-0.5f, q, 2.0f));
        if (BRANCHLESS || fw > 0.0f) {
            const float sd = fw * __fdividef(u, u + fmaxf(w, 1e-30f)) * f.d;
            In = fmaf(sd, fmaf(-q, dSn, s.dS), In);
        }
    }
    s.I = In;
    if (s.live) atomicAdd(Jd + s.vc, to_f64<WIDEN>(cwc * In));
    s.u = w;
    s.ru = rw;
    s.hc = hn;
    s.Sp = s.Sc;
    s.Sc = cn.y;
    s.dS = dSn;
    s.vc = vn;
}

}  // namespace rt3d
