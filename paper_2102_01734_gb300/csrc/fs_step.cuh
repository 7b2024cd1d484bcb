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
// (record rn: offset, J weight, l/2, l/2), update I at the current point with the
// difference form of the file header, add cwc I to J at the current point,
// advance. BRANCHLESS evaluates the parabolic correction also where its
// blend weight is 0 (no divergent branch).
// The same given the next point's replicated offset vn and its gathered
// (chi, S) cn (loaded ahead by the caller).
template <bool PARAB, bool WIDEN, bool BRANCHLESS>
__device__ __forceinline__ void fast_step_c(RayF &s, double *__restrict__ Jd, const float4 &rn,
                                            float cwc, int vn, const float2 cn) {
    const float hn = cn.x * rn.z;
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

template <bool PARAB, bool WIDEN, bool BRANCHLESS>
__device__ __forceinline__ void fast_step(RayF &s, const float2 *__restrict__ chiS,
                                          double *__restrict__ Jd, const float4 &rn, float cwc) {
    const int vn = s.base + __float_as_int(rn.x);
    fast_step_c<PARAB, WIDEN, BRANCHLESS>(s, Jd, rn, cwc, vn, chiS[vn]);
}


// ---- Two characteristics per thread in packed FP32x2 arithmetic ----
// The sm_100 family executes add, sub, mul and fma on a pair of FP32 values
// in one instruction (each component rounded as its scalar operation). The
// pair kernel gives a thread the characteristics of face cells (x0, y) and
// (x0, y + 1): component .x and .y of every float2 below.

__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 pk1(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ unsigned long long f2_bits(float2 a) {
    return ((unsigned long long)__float_as_uint(a.y) << 32) | __float_as_uint(a.x);
}
__device__ __forceinline__ float2 f2_from_bits(unsigned long long r) {
    return make_float2(__uint_as_float((unsigned)r), __uint_as_float((unsigned)(r >> 32)));
}
// a - b per component
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from_bits(r);
}
// MUFU approximations (PTX rcp.approx / ex2.approx, subnormals flushed)
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct IntervalE2 {
    float2 e0, a, d;
};
// interval_fast's polynomial branch (u < 1) on both components
__device__ __forceinline__ IntervalE2 interval_poly2(float2 u) {
    float2 p = fma2(pk1(-3.569704858819023e-05f), u, pk1(3.819821577053517e-04f));
    p = fma2(p, u, pk1(-2.770215505734086e-03f));
    p = fma2(p, u, pk1(1.6664894297719002e-02f));
    p = fma2(p, u, pk1(-8.333317935466766e-02f));
    p = fma2(p, u, pk1(3.333333432674408e-01f));
    const float2 b = mul2(u, p);
    const float2 hu = mul2(u, pk1(0.5f));
    IntervalE2 r;
    r.a = mul2(hu, sub2(pk1(1.0f), b));       // u (1 - b) / 2
    r.e0 = mul2(u, sub2(pk1(1.0f), r.a));     // u (1 - a)
    r.d = sub2(r.a, b);
    return r;
}
// interval_fast's exponential branch (u >= 1) on both components, given
// nru = -1/u
__device__ __forceinline__ IntervalE2 interval_exp2(float2 u, float2 nru) {
    const float2 t = mul2(u, pk1(-1.4426950408889634f));  // -u log2(e)
    IntervalE2 r;
    r.e0 = sub2(pk1(1.0f), pk(ex2_approx(t.x), ex2_approx(t.y)));
    r.a = fma2(r.e0, nru, pk1(1.0f));                    // 1 - e0/u
    r.d = mul2(fma2(r.a, pk1(-2.0f), r.e0), nru);         // (2a - e0)/u
    return r;
}
// Per component the branch of interval_fast; a thread whose two intervals
// fall on different sides of u = 1 evaluates both and selects (a NaN u takes
// the exponential branch, as in the scalar form).
__device__ __forceinline__ IntervalE2 interval2(float2 u, float2 nru) {
    const bool sx = u.x < 1.0f, sy = u.y < 1.0f;
    if (sx && sy) return interval_poly2(u);
    if (!sx && !sy) return interval_exp2(u, nru);
    const IntervalE2 p = interval_poly2(u), e = interval_exp2(u, nru);
    IntervalE2 r;
    r.e0 = pk(sx ? p.e0.x : e.e0.x, sy ? p.e0.y : e.e0.y);
    r.a = pk(sx ? p.a.x : e.a.x, sy ? p.a.y : e.a.y);
    r.d = pk(sx ? p.d.x : e.d.x, sy ? p.d.y : e.d.y);
    return r;
}

// State of a pair of characteristics: as RayF, with -1/u in place of 1/u
// (the form the exponential branch and q use).
struct RayP {
    float2 I, u, nru, hc, Sp, Sc, dS;
};

// One point of a pair of characteristics, given c, the pair-packed (chi, S)
// of the next point, and hl, the pair (l/2, l/2) of its chord: the update of
// fast_step on both characteristics (the parabolic correction always
// evaluated, its blend weight 0 where the linear form applies), and the
// advance to the next point. Returns the intensities at the current point.
// The two reciprocals of the scalar step come from one: with
// X = wf (u + wf), 1/wf = (u + wf)/X and u/(u + wf) = u wf/X, where wf is
// the next interval floored at 1e-15 (so X >= 1e-30 stays a normal FP32
// number; a zero-opacity interval gets q = 0 or blend weight 0).
template <bool PARAB>
__device__ __forceinline__ float2 pair_advance_c(RayP &s, const float4 &c, float2 hl) {
    const float2 hn = mul2(pk(c.x, c.y), hl);
    const float2 Sn = pk(c.z, c.w);
    const float2 dSn = sub2(Sn, s.Sc);
    const float2 w = add2(s.hc, hn);
    const IntervalE2 f = interval2(s.u, s.nru);
    float2 In = fma2(f.e0, sub2(s.Sp, s.I), s.I);
    In = fma2(f.a, s.dS, In);
    const float2 nwf = pk(fminf(-w.x, -1e-15f), fminf(-w.y, -1e-15f));  // -wf
    float2 nrw;
    if (PARAB) {
        const float2 nuw = sub2(nwf, s.u);                 // -(u + wf)
        const float2 X = mul2(nwf, nuw);                   // wf (u + wf)
        const float2 R = pk(rcp_approx(X.x), rcp_approx(X.y));
        nrw = mul2(nuw, R);                                // -1/wf
        const float2 nq = mul2(s.u, nrw);                  // -q
        const float2 fw = mul2(pk(__saturatef(fmaf(-2.0f, s.u.x, 2.0f)),
                                  __saturatef(fmaf(-2.0f, s.u.y, 2.0f))),
                               pk(__saturatef(fmaf(0.5f, nq.x, 2.0f)),
                                  __saturatef(fmaf(0.5f, nq.y, 2.0f))));
        const float2 ns = mul2(mul2(s.u, nwf), R);         // -u/(u + wf)
        const float2 cd = fma2(nq, dSn, s.dS);             // dS - q dSn
        const float2 g = mul2(mul2(fw, f.d), ns);          // -f s d
        In = sub2(In, mul2(g, cd));
    } else {
        nrw = pk(rcp_approx(nwf.x), rcp_approx(nwf.y));
    }
    s.I = In;
    s.u = w;
    s.nru = nrw;
    s.hc = hn;
    s.Sp = s.Sc;
    s.Sc = Sn;
    s.dS = dSn;
    return In;
}

// The last point of a pair (linear form): its intensities.
__device__ __forceinline__ float2 pair_last(const RayP &s) {
    const IntervalE2 f = interval2(s.u, s.nru);
    return fma2(f.a, s.dS, fma2(f.e0, sub2(s.Sp, s.I), s.I));
}

// A pair at its first point: the entry interval has chi_{-1} l_{-1} = 0 and
// S_{-1} = S_0; c = pair-packed (chi, S) of the first point, hl = l/2 of its
// chord, (Ia, Ib) the boundary intensities.
__device__ __forceinline__ void pair_init(RayP &s, const float4 &c, float2 hl, float Ia, float Ib) {
    s.I = pk(Ia, Ib);
    s.hc = mul2(pk(c.x, c.y), hl);
    s.u = s.hc;
    s.Sc = pk(c.z, c.w);
    s.Sp = s.Sc;
    s.dS = pk1(0.0f);
    s.nru = pk(rcp_approx(fminf(-s.hc.x, -1e-15f)), rcp_approx(fminf(-s.hc.y, -1e-15f)));
}

// FP32 contribution to FP64 for a reduction: CONV 1 integer moves, else the
// conversion instruction.
template <int CONV> __device__ __forceinline__ double pair_widen(float x) {
    return CONV == 1 ? widen_f32(x) : (double)x;
}

}  // namespace rt3d
