// Formal solution J = Lambda S (Eq. frmsol) by long characteristics on the
// periodic Cartesian box, with the optional non-local Lambda* band (Sec. 4:
// "computing the Lambda* operator (only in the first iteration)"), following
// the per-slot steps of the paper's Listing 1: gather the previous and next S
// and chi, compute dtau, compute alpha/beta/gamma, fix up at the boundary,
// store Lambda* data, compute Delta I and exp(-dtau).
//
// Mapping: one thread integrates one characteristic (all nx*ny
// characteristics of a solid angle are translates of the cached one, so the
// threads of a warp walk neighbouring voxels of the same layer in lock step:
// the (chi, S) gathers of a warp hit one or two 128-byte lines). Blocks are
// (ray bundle, solid angle) with angles ordered longest first. Contributions
// are accumulated in FP64 (red.global.add.f64), also in the FP32 mode.
//
// Interval functions. For the interval of optical depth u between points
// k-1 and k, with e0 = 1 - e^-u, e1 = u - e0, e2 = u^2 - 2 e1 (Olson &
// Kunasz 1987), the kernel works with
//   a = e1/u, b = e2/u^2, a0 = e0 - a, d = a - b,
// which stay O(1) or O(u) at both ends of the range. Small u: e2 = u^3 p(u)
// with p(u) = 2 sum_m (-1)^m u^m / (m+3)!, from the Taylor series of exp,
// then a = u (1 - b)/2, e0 = u (1 - a), E = 1 - e0. Large u: E = exp(-u),
// a = 1 - e0/u, a0 = (1 - (1+u) E)/u, d = (2a - e0)/u.
// Coefficients (s = u/(u+w), q = u/w, w the next interval):
//   linear:    alpha = a0, beta = a, gamma = 0
//   parabolic: beta + gamma = a + f s d, gamma = -f q s d, alpha = a0 - f s d,
// where f = clamp(2 - 2u, 0, 1) clamp(2 - q/2, 0, 1) blends the Olson-Kunasz
// parabola (f = 1: u <= 1/2 and q <= 2) continuously into the linear form
// (f = 0: u >= 1 or q >= 4), which keeps every weight of an optically thick
// interval non-negative (the OS matrix stays diagonally dominant),
// and I_k = E I_{k-1} + alpha S_{k-1} + (beta+gamma) S_k + gamma (S_{k+1} - S_k)
// so that large |gamma| (short next interval) multiplies a difference instead
// of cancelling between two products. The kernels without Lambda* use the
// same update in difference form, I_k = I_{k-1} + e0 (S_{k-1} - I_{k-1}) +
// a (S_k - S_{k-1}) + f s d ((S_k - S_{k-1}) - q (S_{k+1} - S_k)), which
// needs neither E nor a0. The last point of a characteristic is
// linear; the entry point has S_{-1} = S_0 and chi_{-1} l_{-1} = 0.
#include "fs_step.cuh"

namespace rt3d {

namespace {

template <typename R> struct V2;
template <> struct V2<float> { using T = float2; };
template <> struct V2<double> { using T = double2; };

// Taylor coefficients of p(u) = e2/u^3 = 2 sum_m (-1)^m u^m / (m+3)!.
constexpr double fact(int n) { return n <= 1 ? 1.0 : n * fact(n - 1); }
constexpr double pc(int m) { return (m % 2 ? -2.0 : 2.0) / fact(m + 3); }
template <int M> struct PC { static constexpr double v = pc(M); };
template <int M> struct PCf { static constexpr float v = (float)pc(M); };

// Horner evaluation of p(u) from degree M down to 0, unrolled at compile time.
template <int M> struct Horner {
    __device__ __forceinline__ static double eval(double acc, double u) {
        return Horner<M - 1>::eval(fma(acc, u, PC<M - 1>::v), u);
    }
};
template <> struct Horner<0> {
    __device__ __forceinline__ static double eval(double acc, double) { return acc; }
};

struct IntervalF {
    float E, a0, a, d;
};
struct IntervalD {
    double E, a0, a, d;
};

__device__ __forceinline__ IntervalF interval(float u) {
    IntervalF r;
    if (u < 1.0f) {
        // Horner, m = 8 .. 0: truncation < 1.3e-8 relative at u = 1
        float p = PCf<8>::v;
        p = fmaf(p, u, PCf<7>::v);
        p = fmaf(p, u, PCf<6>::v);
        p = fmaf(p, u, PCf<5>::v);
        p = fmaf(p, u, PCf<4>::v);
        p = fmaf(p, u, PCf<3>::v);
        p = fmaf(p, u, PCf<2>::v);
        p = fmaf(p, u, PCf<1>::v);
        p = fmaf(p, u, PCf<0>::v);
        const float b = u * p;
        const float a = 0.5f * u * (1.0f - b);
        const float e0 = u * (1.0f - a);
        r.E = 1.0f - e0;
        r.a = a;
        r.a0 = e0 - a;
        r.d = a - b;
    } else {
        const float E = __expf(-u);
        const float ru = __fdividef(1.0f, u);
        const float e0 = 1.0f - E;
        const float a = fmaf(-e0, ru, 1.0f);
        r.E = E;
        r.a = a;
        r.a0 = fmaf(-(1.0f + u), E, 1.0f) * ru;
        r.d = fmaf(2.0f, a, -e0) * ru;
    }
    return r;
}

__device__ __forceinline__ IntervalD interval(double u) {
    IntervalD r;
    if (u < 0.5) {
        // Horner, m = 17 .. 0: truncation ~1e-23 relative at u = 1/2
        const double p = Horner<17>::eval(PC<17>::v, u);
        const double b = u * p;
        const double a = 0.5 * u * (1.0 - b);
        const double e0 = u * (1.0 - a);
        r.E = 1.0 - e0;
        r.a = a;
        r.a0 = e0 - a;
        r.d = a - b;
    } else {
        const double E = exp(-u);
        const double ru = 1.0 / u;
        const double e0 = 1.0 - E;
        const double a = fma(-e0, ru, 1.0);
        r.E = E;
        r.a = a;
        r.a0 = fma(-(1.0 + u), E, 1.0) * ru;
        r.d = fma(2.0, a, -e0) * ru;
    }
    return r;
}

template <typename R> __device__ __forceinline__ R div_fast(R x, R y);
template <> __device__ __forceinline__ float div_fast<float>(float x, float y) {
    return __fdividef(x, y);
}
template <> __device__ __forceinline__ double div_fast<double>(double x, double y) {
    return x / y;
}

template <typename R> __device__ __forceinline__ R clamp01(R x) {
    return x < R(0) ? R(0) : (x > R(1) ? R(1) : x);
}

__device__ __forceinline__ int voxel_of(uint32_t c, int x0, int y0, int nx, int ny) {
    int x = x0 + (int)(c & 0x7ffu);
    int y = y0 + (int)((c >> 11) & 0x7ffu);
    if (x >= nx) x -= nx;
    if (y >= ny) y -= ny;
    return x + nx * (y + ny * (int)(c >> 22));
}

// index of the same point in the 2 x 2-replicated packed (chi, S) array
__device__ __forceinline__ int rep_of(uint32_t c, int x0, int y0, int nx, int ny) {
    return (int)rep_index(x0 + (int)(c & 0x7ffu), y0 + (int)((c >> 11) & 0x7ffu), (int)(c >> 22),
                          nx, ny);
}

template <typename R, bool PARAB, bool LSTAR>
__global__ void __launch_bounds__(128) fs_kernel(FsParams p) {
    using R2 = typename V2<R>::T;
    const int nray = p.nx * p.ny;
    const int ray = blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= nray) return;
    const int o = p.order[blockIdx.y];
    const int x0 = ray % p.nx, y0 = ray / p.nx;
    const long long t0 = p.toff[o];
    const int K = p.tlen[o];
    const uint32_t *__restrict__ code = p.code + t0;
    const R *__restrict__ len = static_cast<const R *>(p.len) + t0;
    const R *__restrict__ cw = static_cast<const R *>(p.cw) + t0;
    const R2 *__restrict__ chiS = static_cast<const R2 *>(p.chiS);
    const long long N = (long long)nray * p.nz;

    double I0 = 0.0;
    if (!p.homogeneous) {
        if (p.up[o]) I0 = p.bot_face ? p.bot_face[ray] : p.I_bot;
        else I0 = p.top_face ? p.top_face[ray] : p.I_top;
    }
    R I = (R)I0;

    int v = voxel_of(__ldg(code), x0, y0, p.nx, p.ny);
    R2 cs = chiS[rep_of(__ldg(code), x0, y0, p.nx, p.ny)];
    R chil_c = cs.x * __ldg(len);
    R chil_p = R(0);
    R S_c = cs.y, S_p = cs.y;
    R ring[kWin];
#pragma unroll
    for (int i = 0; i < kWin; ++i) ring[i] = R(0);

    for (int k = 0; k < K; ++k) {
        const R u = R(0.5) * (chil_p + chil_c);
        const auto f = interval(u);
        const bool has_next = (k + 1 < K);
        int vn = v;
        R chil_n = R(0), S_n = S_c;
        if (has_next) {
            const uint32_t cn = __ldg(code + k + 1);
            vn = voxel_of(cn, x0, y0, p.nx, p.ny);
            const R2 c2 = chiS[rep_of(cn, x0, y0, p.nx, p.ny)];
            chil_n = c2.x * __ldg(len + k + 1);
            S_n = c2.y;
        }
        R al = f.a0, bg = f.a, ga = R(0);
        if (PARAB && has_next) {
            const R w = R(0.5) * (chil_c + chil_n);
            if (w > R(0)) {
                const R q = div_fast(u, w);
                const R fw = clamp01(R(2) - R(2) * u) * clamp01(R(2) - R(0.5) * q);
                if (fw > R(0)) {
                    const R sd = fw * div_fast(u, u + w) * f.d;
                    bg = f.a + sd;
                    ga = -q * sd;
                    al = f.a0 - sd;
                }
            }
        }
        I = f.E * I + al * S_p + bg * S_c + ga * (S_n - S_c);
        const R c = __ldg(cw + k);
        atomicAdd(p.J + v, (double)(c * I));
        if (LSTAR) {
            // ring[i] = dI_k / dS_{k-7+i}
#pragma unroll
            for (int i = 0; i < kWin - 1; ++i) ring[i] = f.E * ring[i + 1];
            const R be = bg - ga;
            if (k == 0) ring[7] += al;  // S_{-1} = S_0 at the entry point
            else ring[6] += al;
            ring[7] += be;
            ring[8] = ga;
            const uint64_t wc = __ldg(reinterpret_cast<const unsigned long long *>(p.win + t0 + k));
#pragma unroll
            for (int i = 0; i < kWin; ++i) {
                const unsigned dc = (unsigned)(wc >> (5 * i)) & 31u;
                if (dc != kWinNone) atomicAdd(p.lstar + (long long)dc * N + v, (double)(c * ring[i]));
            }
        }
        chil_p = chil_c;
        chil_c = chil_n;
        S_p = S_c;
        S_c = S_n;
        v = vn;
    }
}

// FP32 formal solution without Lambda* (every iteration after the first).
// A thread integrates RPT characteristics of one solid angle (face cells
// ray, ray + blockDim.x, ...), sharing the 16-byte broadcast load of each
// step record (replicated offset, l/2, J weight). Per point and
// characteristic: one integer add for the replicated address, one 8-byte
// (chi, S) gather, the interval arithmetic, and one FP64 reduction
// (red.global.add.f64) into the replicated J, folded afterwards; the FP32
// contribution is widened by integer moves, by the conversion instruction
// (which runs on the FP64 pipe), or alternately by both (the autotuner
// picks, see fast_step and fs_fast_kernel). FP64 accumulation keeps the operator's error at the
// level of its FP32 arithmetic (an FP32 reduction over ~10^3 contributions
// per voxel and angle group was measured to cost the refinement a fourth
// FP64 formal solution and 60 more FP32 ones at 129^3). The reciprocal of
// the next interval is carried into the next step. The last point (linear
// form) is peeled off; the loop takes two points per trip so that the
// carried values rotate through registers without moves.
// CONV: how FP32 contributions become FP64 for the reduction: 0 the
// conversion instruction (FP64 pipe), 1 integer moves, 2 alternating between
// the two from point to point (both pipes half loaded).
template <bool PARAB, int RPT, int CONV, bool BRANCHLESS>
__global__ void __launch_bounds__(256) fs_fast_kernel(FsParams p) {
    const int nray = p.nx * p.ny;
    const int ray0 = blockIdx.x * (blockDim.x * RPT) + threadIdx.x;
    if (ray0 >= nray) return;
    const int o = p.order[blockIdx.y];
    const int K = p.tlen[o];
    const float4 *__restrict__ rec = p.rec32 + p.toff[o];
    const float2 *__restrict__ chiS = static_cast<const float2 *>(p.chiS);
    double *__restrict__ Jd = p.Jrep;
    constexpr bool W0 = CONV == 1, W1 = CONV >= 1;

    RayF ray[RPT];
    const float4 r = __ldg(rec);
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        RayF &s = ray[j];
        const int rj = ray0 + j * blockDim.x;
        s.live = rj < nray;
        const int rr = s.live ? rj : ray0;
        const int x0 = rr % p.nx, y0 = rr / p.nx;
        s.base = x0 + 2 * p.nx * y0;
        double I0 = 0.0;
        if (!p.homogeneous) {
            if (p.up[o]) I0 = p.bot_face ? p.bot_face[rr] : p.I_bot;
            else I0 = p.top_face ? p.top_face[rr] : p.I_top;
        }
        s.I = (float)I0;
        s.vc = s.base + __float_as_int(r.x);
        const float2 cs = chiS[s.vc];
        s.hc = cs.x * r.y;  // half the optical depth of the chord of the point
        s.u = s.hc;         // the entry interval: chi_{-1} l_{-1} = 0
        s.Sc = cs.y;
        s.Sp = cs.y;        // S_{-1} = S_0
        s.dS = 0.0f;
        s.ru = __fdividef(1.0f, s.hc);
    }
    float cwc = r.z;
    int k = 1;
    // two points per trip: the carried values rotate through registers
    for (; k + 1 < K; k += 2) {
        const float4 r1 = __ldg(rec + k), r2 = __ldg(rec + k + 1);
#pragma unroll
        for (int j = 0; j < RPT; ++j) fast_step<PARAB, W0, BRANCHLESS>(ray[j], chiS, Jd, r1, cwc);
#pragma unroll
        for (int j = 0; j < RPT; ++j) fast_step<PARAB, W1, BRANCHLESS>(ray[j], chiS, Jd, r2, r1.z);
        cwc = r2.z;
    }
    if (k < K) {
        const float4 r1 = __ldg(rec + k);
#pragma unroll
        for (int j = 0; j < RPT; ++j) fast_step<PARAB, W0, BRANCHLESS>(ray[j], chiS, Jd, r1, cwc);
        cwc = r1.z;
    }
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        RayF &s = ray[j];
        const IntervalE f = interval_fast(s.u, PARAB ? s.ru : __fdividef(1.0f, s.u));
        s.I = fmaf(f.a, s.dS, fmaf(f.e0, s.Sp - s.I, s.I));
        if (s.live) {
            atomicAdd(Jd + s.vc, to_f64<W1>(cwc * s.I));
            if (!(fabsf(s.I) <= 3.402823466e38f))  // non-finite: make J NaN
                atomicAdd(Jd + s.vc, __longlong_as_double(0x7ff8000000000000LL));
        }
    }
}

// ---- FP64 formal solution without Lambda* (refinement residuals, FP64 mode
// after the first iteration). The FP64 pipe is the bound, so everything that
// can leave it does: branch tests on the high word of non-negative doubles
// (integer compares), reciprocals seeded in FP32, widening by integer moves.

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

// One thread per characteristic; per point: the replicated offset (FP32
// record), the FP64 (l/2, J weight) record, the (chi, S) gather, and one
// red.global.add.f64 into the replicated J (folded afterwards). The
// parabolic blend f = clamp(2 - 2u) clamp(2 - q/2) is taken apart on integer
// tests: f > 0 iff u < 1 and q < 4, each factor is 1 below 1/2 (resp. 2) and
// one FMA between.
template <bool PARAB>
__global__ void __launch_bounds__(128) fs64_fast_kernel(FsParams p) {
    const int nray = p.nx * p.ny;
    const int ray = blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= nray) return;
    const int o = p.order[blockIdx.y];
    const int K = p.tlen[o];
    const long long t0 = p.toff[o];
    const float4 *__restrict__ rec = p.rec32 + t0;
    const double2 *__restrict__ rd = p.rec64 + t0;
    const double2 *__restrict__ chiS = static_cast<const double2 *>(p.chiS);
    double *__restrict__ J = p.Jrep;
    const int x0 = ray % p.nx, y0 = ray / p.nx;
    const int base = x0 + 2 * p.nx * y0;

    double I = 0.0;
    if (!p.homogeneous) {
        if (p.up[o]) I = p.bot_face ? p.bot_face[ray] : p.I_bot;
        else I = p.top_face ? p.top_face[ray] : p.I_top;
    }
    int vc = base + __float_as_int(__ldg(&rec[0].x));
    double2 r = __ldg(rd);
    const double2 cs = chiS[vc];
    double hc = cs.x * r.x;  // half the optical depth of the chord of the point
    double cwc = r.y;
    double u = hc;  // the entry interval: chi_{-1} l_{-1} = 0
    double Sc = cs.y, Sp = cs.y, dS = 0.0;  // S_{-1} = S_0
    double ru = PARAB ? recip64(hc) : 0.0;
    for (int k = 1; k < K; ++k) {
        const int vn = base + __float_as_int(__ldg(&rec[k].x));
        const double2 rn = __ldg(rd + k);
        const double2 cn = chiS[vn];
        const double hn = cn.x * rn.x;
        const double dSn = cn.y - Sc;
        const double w = hc + hn;
        const IntervalDE f = interval64<PARAB>(u, ru);
        // difference form of the update (as in the FP32 kernel)
        double In = fma(f.e0, Sp - I, I);
        In = fma(f.a, dS, In);
        if (PARAB) {
            const double rw = recip64(w);
            const double q = u * rw;
            if (hi_below(u, 0x3FF00000) && hi_below(q, 0x40100000)) {
                double fw = 1.0;
                if (!hi_below(u, 0x3FE00000)) fw = fma(-2.0, u, 2.0);
                if (!hi_below(q, 0x40000000)) fw *= fma(-0.5, q, 2.0);
                const double sd = fw * (u * recip64(u + w)) * f.d;
                In = fma(sd, fma(-q, dSn, dS), In);
            }
            ru = rw;
        }
        I = In;
        atomicAdd(J + vc, cwc * I);
        u = w;
        hc = hn;
        Sp = Sc;
        Sc = cn.y;
        dS = dSn;
        vc = vn;
        cwc = rn.y;
    }
    const IntervalDE f = interval64<PARAB>(u, ru);
    I = fma(f.a, dS, fma(f.e0, Sp - I, I));
    atomicAdd(J + vc, cwc * I);
}

// J[v] = sum of the four replicas of v in Jrep (FP64); Jrep zeroed for the
// next launch.
__global__ void fold_kernel(int nx, int ny, int nz, double *__restrict__ Jrep,
                            double *__restrict__ J) {
    const long long n = (long long)nx * ny * nz;
    const long long dy = 2LL * nx * ny;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long long)nx * ny));
        const long long i0 = rep_index(x, y, z, nx, ny);
        J[v] = (Jrep[i0] + Jrep[i0 + nx]) + (Jrep[i0 + dy] + Jrep[i0 + dy + nx]);
        Jrep[i0] = 0.0;
        Jrep[i0 + nx] = 0.0;
        Jrep[i0 + dy] = 0.0;
        Jrep[i0 + dy + nx] = 0.0;
    }
}

template <typename R, bool PARAB, bool LSTAR>
cudaError_t launch_t(const FsParams &p, cudaStream_t s) {
    const int threads = 128;
    dim3 grid((p.nx * p.ny + threads - 1) / threads, p.nangles);
    fs_kernel<R, PARAB, LSTAR><<<grid, threads, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace

template <bool PARAB, int CONV, bool BL>
void launch_fast_t(const FsParams &p, dim3 grid, int block, int rpt, cudaStream_t s) {
    if (rpt == 2) fs_fast_kernel<PARAB, 2, CONV, BL><<<grid, block, 0, s>>>(p);
    else fs_fast_kernel<PARAB, 1, CONV, BL><<<grid, block, 0, s>>>(p);
}

template <bool PARAB>
void launch_fast_p(const FsParams &p, dim3 grid, const FsShape &sh, cudaStream_t s) {
    const int b = sh.block, r = sh.rays_per_thread;
    if (sh.branchless) {
        if (sh.widen == 0) launch_fast_t<PARAB, 0, true>(p, grid, b, r, s);
        else if (sh.widen == 1) launch_fast_t<PARAB, 1, true>(p, grid, b, r, s);
        else launch_fast_t<PARAB, 2, true>(p, grid, b, r, s);
    } else {
        if (sh.widen == 0) launch_fast_t<PARAB, 0, false>(p, grid, b, r, s);
        else if (sh.widen == 1) launch_fast_t<PARAB, 1, false>(p, grid, b, r, s);
        else launch_fast_t<PARAB, 2, false>(p, grid, b, r, s);
    }
}

bool fs_shape_valid(const FsShape &sh) {
    return (sh.block == 64 || sh.block == 128 || sh.block == 256) &&
           (sh.rays_per_thread == 1 || sh.rays_per_thread == 2) && sh.widen >= 0 && sh.widen <= 2 &&
           (sh.branchless == 0 || sh.branchless == 1);
}

cudaError_t launch_fs_fast(const FsParams &p, bool parabolic, const FsShape &sh, cudaStream_t s) {
    if (!fs_shape_valid(sh)) return cudaErrorInvalidValue;
    const int per = sh.block * sh.rays_per_thread;
    dim3 grid((p.nx * p.ny + per - 1) / per, p.nangles);
    if (parabolic) launch_fast_p<true>(p, grid, sh, s);
    else launch_fast_p<false>(p, grid, sh, s);
    return cudaGetLastError();
}

cudaError_t launch_fs64_fast(const FsParams &p, bool parabolic, cudaStream_t s) {
    const int threads = 128;
    dim3 grid((p.nx * p.ny + threads - 1) / threads, p.nangles);
    if (parabolic) fs64_fast_kernel<true><<<grid, threads, 0, s>>>(p);
    else fs64_fast_kernel<false><<<grid, threads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_fold(int nx, int ny, int nz, double *Jrep, double *J, cudaStream_t s) {
    const long long n = (long long)nx * ny * nz;
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    fold_kernel<<<(int)b, 256, 0, s>>>(nx, ny, nz, Jrep, J);
    return cudaGetLastError();
}

cudaError_t launch_fs(const FsParams &p, bool fp64, bool parabolic, bool lstar, cudaStream_t s) {
    if (fp64) {
        if (parabolic) return lstar ? launch_t<double, true, true>(p, s) : launch_t<double, true, false>(p, s);
        return lstar ? launch_t<double, false, true>(p, s) : launch_t<double, false, false>(p, s);
    }
    if (parabolic) return lstar ? launch_t<float, true, true>(p, s) : launch_t<float, true, false>(p, s);
    return lstar ? launch_t<float, false, true>(p, s) : launch_t<float, false, false>(p, s);
}

}  // namespace rt3d
