// Float-float formal solution without Lambda*: the formal solution of
// fs.cu (Eq. frmsol, long characteristics, parabolic or linear weights of
// Olson & Kunasz with the limited parabola, the update in difference form)
// evaluated in float-float arithmetic (ff.cuh, about 48 significant bits) on
// the FP32 pipe. It serves the refinement residuals of the mixed-precision
// solve, which need FP64-class accuracy (about 1e-13 relative here, against
// 2e-5 for the FP32 formal solution) but not the FP64 pipe, which on this GPU
// runs at about 1/64 of the FP32 rate; the residual that certifies a
// solution is still an FP64 formal solution.
//
// Inputs are split once per formal solution: the packed replicated (chi, S)
// as float4 (chi_hi, chi_lo, S_hi, S_lo), and per step of the geometry
// cache a float4 (l/2 hi, lo, J weight hi, lo). The J contribution cw I is
// reduced in FP64 (the two widened parts added on the FP64 pipe, one
// operation per point).
#include "ff.cuh"
#include "fs_step.cuh"
#include "sph_ff.cuh"

namespace rt3d {

namespace {

// Cody-Waite split of ln2/32: c1 and c2 carry 11 significant bits (so n c1
// and n c2 are exact for |n| < 2^13), (c3, c4) the rest as a float-float.
constexpr float kC1 = 0.02166748f, kC2 = -6.6310167e-06f;
constexpr float kC3 = -5.9520444e-11f, kC4 = -2.744745e-18f;
constexpr float kInvL = 46.16624f;  // 32 / ln2

// e^-u for u >= 1/2 (Tang's table-driven method, in float-float): n =
// nearest integer to u 32/ln2, r = u - n ln2/32 (|r| <= ln2/64 + rounding),
// e^-u = 2^-(n>>5) 2^-((n&31)/32) e^-r with tab[j] = 2^(-j/32) and
// e^-r = 1 - r + r^2/2 (float-float) + (-r^3/6 + r^4/24 - r^5/120) (FP32,
// below 2.2e-7 in magnitude). Returns 0 for u > 87 (below 1.7e-38).
__device__ __forceinline__ ff ff_exp_neg(ff u, const float2 *tab) {
    if (u.hi > 87.0f) return ff_of(0.0f);
    const float nf = rintf(u.hi * kInvL);
    const int n = (int)nf;
    ff r = two_sum(fmaf(-nf, kC1, u.hi), -nf * kC2);
    r = ff_add_f(r, u.lo);
    r = ff_sub(r, ff_mul_f(ff{kC3, kC4}, nf));
    ff e = ff_add(ff_sub(ff_of(1.0f), r), ff_scale(ff_mul(r, r), 0.5f));
    const float x = r.hi;
    e = ff_add_f(e, x * x * x * fmaf(x, fmaf(-x, 1.0f / 120.0f, 1.0f / 24.0f), -1.0f / 6.0f));
    const float2 t = tab[n & 31];
    e = ff_mul(e, ff{t.x, t.y});
    return ff_scale(e, __int_as_float((127 - (n >> 5)) << 23));
}

struct IntervalFF {
    ff e0, a, d;
};

// e0, a, d of the interval of optical depth u (the quantities of
// interval_fast). u < 1/2: p(u) = e2/u^3 as the degree-9 polynomial fitted to
// it on [0, 1/2] (approximation error 1.6e-18 relative with exact
// coefficients), levels 9..6 of its Horner scheme in FP32 (their share of p
// is below 2.6e-7; their coefficients rounded to FP32 make the polynomial's
// error 9.3e-15 relative), 5..0 in float-float; b = u p, a = u/2 (1 - b), e0 = u (1 - a), d = a - b. Otherwise
// E = e^-u, e0 = 1 - E, a = 1 - e0/u, d = (2a - e0)/u with ru = 1/u.
__device__ __forceinline__ IntervalFF interval_ff(ff u, ff ru, const float2 *tab) {
    IntervalFF r;
    if (u.hi < 0.5f) {
        float q = -3.4475018e-09f;
        q = fmaf(q, u.hi, 4.935483e-08f);
        q = fmaf(q, u.hi, -5.5071155e-07f);
        q = fmaf(q, u.hi, 5.51131e-06f);
        ff P = ff_fma(ff_of(q), u, ff{-4.9603143e-05f, 1.6644579e-12f});
        P = ff_fma(P, u, ff{3.968254e-04f, -9.971136e-12f});
        P = ff_fma(P, u, ff{-2.7777778e-03f, 6.7610896e-11f});
        P = ff_fma(P, u, ff{1.6666668e-02f, -8.692481e-10f});
        P = ff_fma(P, u, ff{-8.3333336e-02f, 2.4835272e-09f});
        P = ff_fma(P, u, ff{3.3333334e-01f, -9.934108e-09f});
        const ff b = ff_mul(u, P);
        const ff hu = ff_scale(u, 0.5f);
        r.a = ff_sub(hu, ff_mul(hu, b));
        r.e0 = ff_sub(u, ff_mul(u, r.a));
        r.d = ff_sub(r.a, b);
    } else {
        r.e0 = ff_sub(ff_of(1.0f), ff_exp_neg(u, tab));
        r.a = ff_sub(ff_of(1.0f), ff_mul(r.e0, ru));
        r.d = ff_mul(ff_sub(ff_scale(r.a, 2.0f), r.e0), ru);
    }
    return r;
}

// 1/x with x floored at 1e-30 (a zero-opacity pair gives a blend weight 0)
__device__ __forceinline__ ff ff_recip_floor(ff x) {
    return ff_recip(x.hi > 1e-30f ? x : ff_of(1e-30f));
}

// State of one characteristic: intensity, optical depth u of the interval
// ending at the current point and its reciprocal, half optical depth of the
// current point's chord, S at the previous and current points and their
// difference (the update in difference form).
struct RayFF {
    ff I, u, ru, hc, Sp, Sc, dS;
};

// Starts a characteristic at its first point (half optical depth h0, source S0,
// entry intensity I0): the entry interval has chi_{-1} l_{-1} = 0 and S_{-1} = S_0.
__device__ __forceinline__ void ff_start(RayFF &s, ff h0, ff S0, double I0) {
    s.I = ff_split(I0);
    s.hc = h0;
    s.u = h0;
    s.Sc = S0;
    s.Sp = S0;
    s.dS = ff_of(0.0f);
    s.ru = ff_recip_floor(h0);
}

// Moves to the next point (half optical depth hn, source Sn): s.I becomes the
// intensity at the current point.
template <bool PARAB>
__device__ __forceinline__ void ff_advance(RayFF &s, ff hn, ff Sn, const float2 *tab) {
    const ff dSn = ff_sub(Sn, s.Sc);
    const ff w = ff_add(s.hc, hn);
    const IntervalFF f = interval_ff(s.u, s.ru, tab);
    ff In = ff_fma(f.e0, ff_sub(s.Sp, s.I), s.I);
    In = ff_fma(f.a, s.dS, In);
    const ff rw = ff_recip_floor(w);
    if (PARAB) {
        const ff q = ff_mul(s.u, rw);
        if (s.u.hi < 1.0f && q.hi < 4.0f) {
            ff fw = ff_of(1.0f);
            if (!(s.u.hi < 0.5f)) fw = ff_sub(ff_of(2.0f), ff_scale(s.u, 2.0f));
            if (!(q.hi < 2.0f)) fw = ff_mul(fw, ff_sub(ff_of(2.0f), ff_scale(q, 0.5f)));
            const ff sr = ff_mul(s.u, ff_recip_floor(ff_add(s.u, w)));
            const ff sd = ff_mul(ff_mul(fw, sr), f.d);
            In = ff_fma(sd, ff_fma(ff_neg(q), dSn, s.dS), In);
        }
    }
    s.I = In;
    s.u = w;
    s.ru = rw;
    s.hc = hn;
    s.Sp = s.Sc;
    s.Sc = Sn;
    s.dS = dSn;
}

// The last point of a characteristic (linear form): s.I becomes its intensity.
__device__ __forceinline__ void ff_last(RayFF &s, const float2 *tab) {
    const IntervalFF f = interval_ff(s.u, s.ru, tab);
    s.I = ff_fma(f.a, s.dS, ff_fma(f.e0, ff_sub(s.Sp, s.I), s.I));
}

// The table 2^(-j/32) of ff_exp_neg, built per block in shared memory from the
// FP64 exp2 (every thread of the block must call it).
__device__ __forceinline__ void ff_table(float2 *tab) {
    if (threadIdx.x < 32) {
        const double t = exp2(-(double)threadIdx.x / 32.0);
        const float h = __double2float_rn(t);
        tab[threadIdx.x] = make_float2(h, __double2float_rn(t - (double)h));
    }
    __syncthreads();
}

// One thread per characteristic (blocks: 128 characteristics of one solid
// angle).
template <bool PARAB>
__global__ void __launch_bounds__(128) fsff_kernel(FsParams p, const float4 *__restrict__ recff,
                                                   const float4 *__restrict__ chiS) {
    __shared__ float2 tab[32];
    ff_table(tab);
    const int nray = p.nx * p.ny;
    const int ray = blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= nray) return;
    const int o = p.order[blockIdx.y];
    const int K = p.tlen[o];
    const long long t0 = p.toff[o];
    const float4 *__restrict__ rec = p.rec32 + t0;  // offsets
    const float4 *__restrict__ rf = recff + t0;     // (l/2, J weight) as float-float
    double *__restrict__ J = p.Jrep;
    const int base = ray % p.nx + 2 * p.nx * (ray / p.nx);

    double I0 = 0.0;
    if (!p.homogeneous)
        I0 = entry_intensity(p.up[o], p.mu, o, ray, p.top_face, p.bot_face, p.bot_grad, p.I_top,
                             p.I_bot);
    int vc = base + __float_as_int(__ldg(&rec[0].x));
    float4 r = __ldg(rf);
    float4 cs = chiS[vc];
    RayFF st;
    ff_start(st, ff_mul(ff{cs.x, cs.y}, ff{r.x, r.y}), ff{cs.z, cs.w}, I0);
    ff cw = ff{r.z, r.w};
    for (int k = 1; k < K; ++k) {
        const int vn = base + __float_as_int(__ldg(&rec[k].x));
        const float4 rn = __ldg(rf + k);
        const float4 cn = chiS[vn];
        ff_advance<PARAB>(st, ff_mul(ff{cn.x, cn.y}, ff{rn.x, rn.y}), ff{cn.z, cn.w}, tab);
        const ff c = ff_mul(cw, st.I);
        atomicAdd(J + vc, widen_f32(c.hi) + widen_f32(c.lo));
        vc = vn;
        cw = ff{rn.z, rn.w};
    }
    ff_last(st, tab);
    const ff c = ff_mul(cw, st.I);
    atomicAdd(J + vc, widen_f32(c.hi) + widen_f32(c.lo));
    if (!(fabsf(st.I.hi) <= 3.402823466e38f))  // non-finite: make J NaN
        atomicAdd(J + vc, __longlong_as_double(0x7ff8000000000000LL));
}

// The half chord l/2 as float-float: the record's FP32 l/2 is its nearest
// float, the high part; the low part is l/2 - hi (exact: the two are within
// an ulp), rounded to FP32. Three FP64-pipe operations per point, against
// about 39 for the FP64 formal solution.
__device__ __forceinline__ ff half_chord_ff(float hi, double l) {
    return ff{hi, __double2float_rn(fma(0.5, l, -(double)hi))};
}

// The same on the spherical cache: one thread per characteristic in the
// builder's order; per point the record (replicated index of the cell, the
// J weight as a float-float pair (weight, remainder), the FP32 l/2) and the
// FP64 chord; contributions reduced at the replicated index (folded
// afterwards).
template <bool PARAB>
__global__ void __launch_bounds__(128) sph_fsff_kernel(SphFsParams p, const float4 *__restrict__ chiS,
                                                       double *__restrict__ Jrep) {
    __shared__ float2 tab[32];
    ff_table(tab);
    const long long ray = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (ray >= p.nrays) return;
    const long long s0 = p.ray_off[ray];
    const int K = p.ray_len[ray];
    const int kind = p.ray_kind[ray];
    const float4 *__restrict__ rr = p.rec + s0;
    const double *__restrict__ l64 = p.len64 + s0;
    double I0 = 0.0;
    if (!p.homogeneous) {
        if (kind == 2) I0 = p.core_face ? p.core_face[p.ray_face[ray]] : p.I_core;
        else if (kind == 1) I0 = p.I_irr;
        else I0 = p.I_out;
    }
    float4 r = __ldg(rr);
    int vc = __float_as_int(r.x);
    float4 cs = chiS[vc];
    RayFF st;
    ff_start(st, ff_mul(ff{cs.x, cs.y}, half_chord_ff(r.z, __ldg(l64))), ff{cs.z, cs.w}, I0);
    ff cw = ff{r.y, r.w};
    for (int k = 1; k < K; ++k) {
        r = __ldg(rr + k);
        const int vn = __float_as_int(r.x);
        const float4 cn = chiS[vn];
        ff_advance<PARAB>(st, ff_mul(ff{cn.x, cn.y}, half_chord_ff(r.z, __ldg(l64 + k))),
                          ff{cn.z, cn.w}, tab);
        const ff c = ff_mul(cw, st.I);
        atomicAdd(Jrep + vc, widen_f32(c.hi) + widen_f32(c.lo));
        vc = vn;
        cw = ff{r.y, r.w};
    }
    ff_last(st, tab);
    const ff c = ff_mul(cw, st.I);
    atomicAdd(Jrep + vc, widen_f32(c.hi) + widen_f32(c.lo));
    if (!(fabsf(st.I.hi) <= 3.402823466e38f))  // non-finite: make J NaN
        atomicAdd(Jrep + vc, __longlong_as_double(0x7ff8000000000000LL));
}

// (chi, S) split into float-float, written to the four replicas of every
// voxel; S = src, or (1 - eps) src + eps B when eps is given
__global__ void pack_ff_kernel(int nx, int ny, int nz, const double *chi, const double *src,
                               const double *eps, const double *B, float4 *out) {
    const long long n = (long long)nx * ny * nz;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long long)nx * ny));
        double sv = src[v];
        if (eps) sv = (1.0 - eps[v]) * sv + eps[v] * B[v];
        const ff c = ff_split(chi[v]), s = ff_split(sv);
        const float4 val = make_float4(c.hi, c.lo, s.hi, s.lo);
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) out[rep_index(x + a * nx, y + b * ny, z, nx, ny)] = val;
    }
}

// per step: (l/2, J weight) split into float-float
__global__ void recff_kernel(long long total, const double2 *rec64, float4 *out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const double2 r = rec64[i];
        const ff l = ff_split(r.x), c = ff_split(r.y);
        out[i] = make_float4(l.hi, l.lo, c.hi, c.lo);
    }
}

int blocks_cap(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    const long long cap = 16LL * device_sm_count();
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_fsff(const FsParams &p, const float4 *recff, const float4 *chiS, bool parabolic,
                        cudaStream_t s) {
    const int threads = 128;
    dim3 grid((p.nx * p.ny + threads - 1) / threads, p.nangles);
    if (parabolic) fsff_kernel<true><<<grid, threads, 0, s>>>(p, recff, chiS);
    else fsff_kernel<false><<<grid, threads, 0, s>>>(p, recff, chiS);
    return cudaGetLastError();
}

cudaError_t launch_sph_fsff(const SphFsParams &p, const float4 *chiS, double *Jrep, bool parabolic,
                            cudaStream_t s) {
    const int threads = 128;
    const long long blocks = (p.nrays + threads - 1) / threads;
    if (parabolic) sph_fsff_kernel<true><<<(unsigned)blocks, threads, 0, s>>>(p, chiS, Jrep);
    else sph_fsff_kernel<false><<<(unsigned)blocks, threads, 0, s>>>(p, chiS, Jrep);
    return cudaGetLastError();
}

cudaError_t launch_pack_ff(int nx, int ny, int nz, const double *chi, const double *src,
                           const double *eps, const double *B, float4 *out, cudaStream_t s) {
    const long long n = (long long)nx * ny * nz;
    pack_ff_kernel<<<blocks_cap(n, 256), 256, 0, s>>>(nx, ny, nz, chi, src, eps, B, out);
    return cudaGetLastError();
}

cudaError_t launch_recff(long long total, const double2 *rec64, float4 *out, cudaStream_t s) {
    recff_kernel<<<blocks_cap(total, 256), 256, 0, s>>>(total, rec64, out);
    return cudaGetLastError();
}

}  // namespace rt3d
