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
#include "fs64_step.cuh"

namespace rt3d {

namespace {

template <typename R> struct V2;
template <> struct V2<float> { using T = float2; };
template <> struct V2<double> { using T = double2; };

// A contribution as the FP64 value its reduction adds: FP32 values widened by
// integer moves (widen_f32), keeping the FP64 pipe free.
__device__ __forceinline__ double red_value(float x) { return widen_f32(x); }
__device__ __forceinline__ double red_value(double x) { return x; }

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
    if (!p.homogeneous)
        I0 = entry_intensity(p.up[o], p.mu, o, ray, p.top_face, p.bot_face, p.bot_grad, p.I_top,
                             p.I_bot);
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
        atomicAdd(p.J + v, red_value(c * I));
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
                if (dc != kWinNone) atomicAdd(p.lstar + (long long)dc * N + v, red_value(c * ring[i]));
            }
        }
        chil_p = chil_c;
        chil_c = chil_n;
        S_p = S_c;
        S_c = S_n;
        v = vn;
    }
    // the widening does not carry a non-finite value: a non-finite intensity
    // (it persists along the recurrence) makes J of the last point NaN
    if (!(fabs((double)I) <= 1.79769313486231570e308))
        atomicAdd(p.J + v, __longlong_as_double(0x7ff8000000000000LL));
}

// FP32 formal solution without Lambda* (every iteration after the first),
// one characteristic per thread. Per point: one integer add for the
// replicated address, one 8-byte (chi, S) gather, the interval arithmetic,
// and one FP64 reduction (red.global.add.f64) into the replicated J, folded
// afterwards; the FP32 contribution is widened by integer moves, by the
// conversion instruction (which runs on the FP64 pipe), or alternately by
// both (the autotuner picks, see fast_step). FP64 accumulation keeps the
// operator's error at the level of its FP32 arithmetic (an FP32 reduction
// over ~10^3 contributions per voxel and angle group was measured to cost
// the refinement a fourth FP64 formal solution and 60 more FP32 ones at
// 129^3). The reciprocal of the next interval is carried into the next step.
// The last point (linear form) is peeled off; the loop takes two points per
// trip so that the carried values rotate through registers without moves.
// CONV: how FP32 contributions become FP64 for the reduction: 0 the
// conversion instruction (FP64 pipe), 1 integer moves, 2 alternating between
// the two from point to point (both pipes half loaded).
template <bool PARAB, int CONV, bool BRANCHLESS>
__global__ void __launch_bounds__(256) fs_fast_kernel(FsParams p) {
    const int nray = p.nx * p.ny;
    const int ray = blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= nray) return;
    const int o = p.order[blockIdx.y];
    const int K = p.tlen[o];
    const float4 *__restrict__ rec = p.rec32 + p.toff[o];
    const float2 *__restrict__ chiS = static_cast<const float2 *>(p.chiS);
    double *__restrict__ Jd = p.Jrep;
    constexpr bool W0 = CONV == 1, W1 = CONV >= 1;

    RayF s;
    const float4 r = __ldg(rec);
    s.live = true;
    const int x0 = ray % p.nx, y0 = ray / p.nx;
    s.base = x0 + 2 * p.nx * y0;
    double I0 = 0.0;
    if (!p.homogeneous)
        I0 = entry_intensity(p.up[o], p.mu, o, ray, p.top_face, p.bot_face, p.bot_grad, p.I_top,
                             p.I_bot);
    s.I = (float)I0;
    s.vc = s.base + __float_as_int(r.x);
    const float2 cs = chiS[s.vc];
    s.hc = cs.x * r.z;  // half the optical depth of the chord of the point
    s.u = s.hc;         // the entry interval: chi_{-1} l_{-1} = 0
    s.Sc = cs.y;
    s.Sp = cs.y;        // S_{-1} = S_0
    s.dS = 0.0f;
    s.ru = __fdividef(1.0f, s.hc);
    float cwc = r.y;
    int k = 1;
    // two points per trip: the carried values rotate through registers
    for (; k + 1 < K; k += 2) {
        const float4 r1 = __ldg(rec + k), r2 = __ldg(rec + k + 1);
        fast_step<PARAB, W0, BRANCHLESS>(s, chiS, Jd, r1, cwc);
        fast_step<PARAB, W1, BRANCHLESS>(s, chiS, Jd, r2, r1.y);
        cwc = r2.y;
    }
    if (k < K) {
        const float4 r1 = __ldg(rec + k);
        fast_step<PARAB, W0, BRANCHLESS>(s, chiS, Jd, r1, cwc);
        cwc = r1.y;
    }
    const IntervalE f = interval_fast(s.u, PARAB ? s.ru : __fdividef(1.0f, s.u));
    s.I = fmaf(f.a, s.dS, fmaf(f.e0, s.Sp - s.I, s.I));
    atomicAdd(Jd + s.vc, to_f64<W1>(cwc * s.I));
    if (!(fabsf(s.I) <= 3.402823466e38f))  // non-finite: make J NaN
        atomicAdd(Jd + s.vc, __longlong_as_double(0x7ff8000000000000LL));
}

// FP32 formal solution without Lambda*, two characteristics per thread in
// packed FP32x2 arithmetic (pair_advance_c): face cells (x0, y0) and
// (x0, y0 + 1) with y0 even. Both sit at the same offset of the cached
// characteristic, so one 16-byte load of the pair-packed (chi, S) (p.pairs)
// serves both, and the step record (one 16-byte broadcast load per point) is
// shared. Lanes of a warp take consecutive x0 of one row pair: the gathers of
// a warp cover one contiguous run of 16-byte elements. Per point and
// characteristic one FP64 reduction into the replicated J, as in
// fs_fast_kernel (CONV: 0 both contributions widened by the conversion
// instruction, 1 both by integer moves, 2 the first by conversion and the
// second by integer moves).
// The next point's step record and pair-packed (chi, S) are loaded one point
// ahead, so the gather's L2 latency overlaps the arithmetic of a point.
template <bool PARAB, int CONV>
__global__ void __launch_bounds__(256) fs_pair_kernel(FsParams p) {
    const int nyh = (p.ny + 1) >> 1;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.nx * nyh) return;
    const int o = p.order[blockIdx.y];
    const int K = p.tlen[o];
    const float4 *__restrict__ rec = p.rec32 + p.toff[o];
    const int x0 = t % p.nx, y0 = 2 * (t / p.nx);
    const bool lb = y0 + 1 < p.ny;  // row y0 + 1 exists (ny odd: not in the last pair)
    const int base = x0 + 2 * p.nx * y0;
    const float4 *__restrict__ P = p.pairs + base;
    double *__restrict__ Ja = p.Jrep + base;
    double *__restrict__ Jb = Ja + 2 * p.nx;
    constexpr int CA = CONV == 1 ? 1 : 0, CB = CONV >= 1 ? 1 : 0;

    float Ia = 0.0f, Ib = 0.0f;
    if (!p.homogeneous) {
        const bool up = p.up[o];
        const int fa = y0 * p.nx + x0;
        Ia = (float)entry_intensity(up, p.mu, o, fa, p.top_face, p.bot_face, p.bot_grad, p.I_top,
                                    p.I_bot);
        if (lb)
            Ib = (float)entry_intensity(up, p.mu, o, fa + p.nx, p.top_face, p.bot_face, p.bot_grad,
                                        p.I_top, p.I_bot);
    }
    RayP s;
    const float4 r0 = __ldg(rec);
    int vc = __float_as_int(r0.x);
    pair_init(s, __ldg(P + vc), pk(r0.z, r0.w), Ia, Ib);
    float cwc = r0.y;
    float4 rq = __ldg(rec + (K > 1 ? 1 : 0));
    float4 cq = __ldg(P + __float_as_int(rq.x));
#pragma unroll 2
    for (int k = 1; k < K; ++k) {
        const float4 rn = rq, cn = cq;
        rq = __ldg(rec + (k + 1 < K ? k + 1 : k));
        cq = __ldg(P + __float_as_int(rq.x));
        const float2 cI = mul2(pair_advance_c<PARAB>(s, cn, pk(rn.z, rn.w)), pk1(cwc));
        atomicAdd(Ja + vc, pair_widen<CA>(cI.x));
        if (lb) atomicAdd(Jb + vc, pair_widen<CB>(cI.y));
        vc = __float_as_int(rn.x);
        cwc = rn.y;
    }
    // the last point: linear form
    const float2 In = pair_last(s);
    const float2 cI = mul2(In, pk1(cwc));
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    atomicAdd(Ja + vc, pair_widen<CA>(cI.x));
    if (!(fabsf(In.x) <= 3.402823466e38f)) atomicAdd(Ja + vc, nan);  // non-finite: make J NaN
    if (lb) {
        atomicAdd(Jb + vc, pair_widen<CB>(cI.y));
        if (!(fabsf(In.y) <= 3.402823466e38f)) atomicAdd(Jb + vc, nan);
    }
}

// ---- Four characteristics per thread with the J contributions summed
// across points before the FP64 reduction.
//
// Lane t of the angle's launch integrates face cells (x0, y0 + r), r = 0..3,
// x0 = t mod nx, y0 = 4 (t div nx) (two packed pairs). All characteristics
// of an angle are translates, so at every point the 32 lanes x 4 rays of a
// warp occupy a block of voxels that moves by one voxel in x, in y or in z
// from point to point (the step type is stored with the point's record).
// Each lane keeps four FP32 sums, one per row, for the voxels its rays
// currently occupy, and adds the contribution (J weight x I) of every point.
// When the block moves in x the sums move one lane over with warp shuffles
// (the voxel a lane's rays enter was its neighbour's); in y they move one
// row over inside the lane; a sum whose voxel leaves the block is reduced
// into the replicated FP64 J: after an x-step through a per-warp list in
// shared memory that is drained 32 entries at a time by all lanes, after a
// y-step directly (one row of the block), after a z-step or a diagonal step
// all four. Lanes of one face row (quad of rows) form a segment: the sums
// move only between lanes of the same segment, and only between rows that
// exist (a y-step towards the face's last row reduces the sum of the last
// existing row instead of moving it on). A sum holds the contributions
// of one voxel from successive rays, at most ~(points per layer) of them,
// before its FP64 reduction.
constexpr int kQuadOffBits = 29;
constexpr unsigned kQuadOffMask = (1u << kQuadOffBits) - 1u;
constexpr int kQuadSpill = 64;  // spill list entries per warp

// Reduces a warp's spill list into J (all lanes; entries with index < 0 are
// empty) and empties it. An entry holds the four row sums of a lane, the
// replicated index of its row-0 voxel (low 29 bits) and its last existing
// row (bits 29-30).
template <int CONV>
__device__ __forceinline__ void quad_drain(const float2 *sa, const float2 *sb, int *si,
                                           double *__restrict__ Jrep, int rowp, int lane) {
    __syncwarp();
    for (int e = lane; e < kQuadSpill; e += 32) {
        const int code = si[e];
        if (code >= 0) {
            const float2 va = sa[e], vb = sb[e];
            const int rtop = code >> kQuadOffBits;
            double *j = Jrep + (code & (int)kQuadOffMask);
            atomicAdd(j, pair_widen<CONV>(va.x));
            if (rtop >= 1) atomicAdd(j + rowp, pair_widen<CONV>(va.y));
            if (rtop >= 2) atomicAdd(j + 2 * rowp, pair_widen<CONV>(vb.x));
            if (rtop >= 3) atomicAdd(j + 3 * rowp, pair_widen<CONV>(vb.y));
            si[e] = -1;
        }
    }
    __syncwarp();
}

template <bool PARAB, int CONV>
__global__ void __launch_bounds__(256, 3) fs_quad_kernel(FsParams p) {
    __shared__ float2 sp_a[8][kQuadSpill], sp_b[8][kQuadSpill];
    __shared__ int sp_idx[8][kQuadSpill];
    constexpr unsigned FULL = 0xffffffffu;
    const int nq = (p.ny + 3) >> 2;
    const int nlive = p.nx * nq;
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t - lane >= nlive) return;  // the whole warp is past the face (warp-uniform)
    const bool live = t < nlive;
    const int tt = live ? t : nlive - 1;
    const int o = p.order[blockIdx.y];
    const int K = p.tlen[o];
    const float4 *__restrict__ rec = p.rec4 + p.toff[o];
    const int x0 = tt % p.nx, q = tt / p.nx, y0 = 4 * q;
    const int base = x0 + 2 * p.nx * y0;
    const int rowp = 2 * p.nx;  // one replicated row
    const float4 *__restrict__ PA = p.pairs + base;
    // rows y0 + 2, y0 + 3 (a quad without them reads pair A's data, unused)
    const float4 *__restrict__ PB = (y0 + 2 < p.ny) ? PA + 2 * rowp : PA;
    double *__restrict__ J0 = p.Jrep + base;
    // the quad's last existing row (-1: a lane past the face). Rows past it
    // (the face's last quad when ny is not a multiple of 4) are integrated
    // and summed like the others, but their sums are never reduced and never
    // move into an existing row.
    const int rtop = live ? min(3, p.ny - 1 - y0) : -1;
    // segments: the lanes of one quad of rows (consecutive x0); lane 0 is live
    const int seg = live ? q : -1;
    const int segL = __shfl_up_sync(FULL, seg, 1), segR = __shfl_down_sync(FULL, seg, 1);
    const bool hasL = lane > 0 && live && segL == seg;
    const bool hasR = lane < 31 && live && segR == seg;
    const float2 takeP = pk1(hasR ? 1.0f : 0.0f), takeM = pk1(hasL ? 1.0f : 0.0f);
    const int nsub = 31 / p.nx + 2;           // segments a warp can span
    const int per_drain = kQuadSpill / nsub;  // x-steps between drains of the spill list
    const int slot0 = seg - __shfl_sync(FULL, seg, 0);
    const int spill_tag = (rtop < 0 ? 0 : rtop) << kQuadOffBits;
    float2 *sa = sp_a[wb];
    float2 *sb = sp_b[wb];
    int *si = sp_idx[wb];
    for (int e = lane; e < kQuadSpill; e += 32) si[e] = -1;
    __syncwarp();

    float Iv[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (!p.homogeneous) {
        const bool up = p.up[o];
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (y0 + r < p.ny)
                Iv[r] = (float)entry_intensity(up, p.mu, o, (y0 + r) * p.nx + x0, p.top_face,
                                               p.bot_face, p.bot_grad, p.I_top, p.I_bot);
    }
    RayP a, b;
    const float4 r0 = __ldg(rec);
    int vc = (int)(__float_as_uint(r0.x) & kQuadOffMask);
    pair_init(a, __ldg(PA + vc), pk(r0.z, r0.w), Iv[0], Iv[1]);
    pair_init(b, __ldg(PB + vc), pk(r0.z, r0.w), Iv[2], Iv[3]);
    float2 A01 = pk1(0.0f), A23 = pk1(0.0f);  // sums of rows y0 .. y0 + 3 at the current voxels
    float cwc = r0.y;
    int cnt = 0;
    // the next point's record and data are loaded one point ahead
    float4 rn = __ldg(rec + (K > 1 ? 1 : 0));
    unsigned bits = __float_as_uint(rn.x);
    float4 cA = __ldg(PA + (bits & kQuadOffMask)), cB = __ldg(PB + (bits & kQuadOffMask));
#pragma unroll 2
    for (int k = 1; k < K; ++k) {
        const float4 rq = __ldg(rec + (k + 1 < K ? k + 1 : k));
        const unsigned bq = __float_as_uint(rq.x);
        const float4 qA = __ldg(PA + (bq & kQuadOffMask)), qB = __ldg(PB + (bq & kQuadOffMask));
        const int vn = (int)(bits & kQuadOffMask);
        const float2 hl = pk(rn.z, rn.w);
        const float2 Ia = pair_advance_c<PARAB>(a, cA, hl);
        const float2 Ib = pair_advance_c<PARAB>(b, cB, hl);
        A01 = fma2(Ia, pk1(cwc), A01);
        A23 = fma2(Ib, pk1(cwc), A23);
        // the block moves from the current points (offset vc) to the next
        const unsigned type = bits >> kQuadOffBits;
        if (type <= 1u) {  // x-step: +1 (type 0) or -1 (type 1)
            const bool plus = type == 0u;
            if (live && (plus ? !hasL : !hasR)) {  // no lane takes this voxel over
                const int e = cnt * nsub + slot0;
                sa[e] = A01;
                sb[e] = A23;
                si[e] = (base + vc) | spill_tag;
            }
            float s0, s1, s2, s3;
            if (plus) {
                s0 = __shfl_down_sync(FULL, A01.x, 1);
                s1 = __shfl_down_sync(FULL, A01.y, 1);
                s2 = __shfl_down_sync(FULL, A23.x, 1);
                s3 = __shfl_down_sync(FULL, A23.y, 1);
            } else {
                s0 = __shfl_up_sync(FULL, A01.x, 1);
                s1 = __shfl_up_sync(FULL, A01.y, 1);
                s2 = __shfl_up_sync(FULL, A23.x, 1);
                s3 = __shfl_up_sync(FULL, A23.y, 1);
            }
            const float2 take = plus ? takeP : takeM;
            A01 = mul2(pk(s0, s1), take);
            A23 = mul2(pk(s2, s3), take);
            if (++cnt == per_drain) {
                quad_drain<CONV>(sa, sb, si, p.Jrep, rowp, lane);
                cnt = 0;
            }
        } else if (type == 2u) {  // y-step +1: row y0's voxel leaves
            if (rtop >= 0) atomicAdd(J0 + vc, pair_widen<CONV>(A01.x));
            A01 = pk(A01.y, A23.x);
            A23 = pk(A23.y, 0.0f);
            if (rtop < 3) {  // the last existing row enters a voxel no sum of this lane holds
                if (rtop == 2) A23.x = 0.0f;
                else if (rtop == 1) A01.y = 0.0f;
                else A01.x = 0.0f;
            }
        } else if (type == 3u) {  // y-step -1: the voxel of the last existing row leaves
            const float v = rtop == 3 ? A23.y : (rtop == 2 ? A23.x : (rtop == 1 ? A01.y : A01.x));
            if (rtop >= 0) atomicAdd(J0 + rtop * rowp + vc, pair_widen<CONV>(v));
            A23 = pk(A01.y, A23.x);
            A01 = pk(0.0f, A01.x);
        } else {  // z-step or diagonal step: all four leave
            double *j = J0 + vc;
            if (rtop >= 0) atomicAdd(j, pair_widen<CONV>(A01.x));
            if (rtop >= 1) atomicAdd(j + rowp, pair_widen<CONV>(A01.y));
            if (rtop >= 2) atomicAdd(j + 2 * rowp, pair_widen<CONV>(A23.x));
            if (rtop >= 3) atomicAdd(j + 3 * rowp, pair_widen<CONV>(A23.y));
            A01 = pk1(0.0f);
            A23 = pk1(0.0f);
        }
        vc = vn;
        cwc = rn.y;
        rn = rq;
        bits = bq;
        cA = qA;
        cB = qB;
    }
    // the last point: linear form
    const float2 Ia = pair_last(a), Ib = pair_last(b);
    A01 = fma2(Ia, pk1(cwc), A01);
    A23 = fma2(Ib, pk1(cwc), A23);
    double *j = J0 + vc;
    if (rtop >= 0) atomicAdd(j, pair_widen<CONV>(A01.x));
    if (rtop >= 1) atomicAdd(j + rowp, pair_widen<CONV>(A01.y));
    if (rtop >= 2) atomicAdd(j + 2 * rowp, pair_widen<CONV>(A23.x));
    if (rtop >= 3) atomicAdd(j + 3 * rowp, pair_widen<CONV>(A23.y));
    quad_drain<CONV>(sa, sb, si, p.Jrep, rowp, lane);
    // a non-finite intensity persists along the recurrence: make J NaN
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    if (rtop >= 0 && !(fabsf(Ia.x) <= 3.402823466e38f)) atomicAdd(j, nan);
    if (rtop >= 1 && !(fabsf(Ia.y) <= 3.402823466e38f)) atomicAdd(j + rowp, nan);
    if (rtop >= 2 && !(fabsf(Ib.x) <= 3.402823466e38f)) atomicAdd(j + 2 * rowp, nan);
    if (rtop >= 3 && !(fabsf(Ib.y) <= 3.402823466e38f)) atomicAdd(j + 3 * rowp, nan);
}

// Records of the four-characteristic kernel: (offset | step type << 29,
// J weight, l/2, l/2), the step type of the move from the previous point:
// 0 x + 1, 1 x - 1, 2 y + 1, 3 y - 1, 4 anything else (z, diagonal, first).
__global__ void quad_rec_kernel(int nx, int ny, const long long *__restrict__ toff,
                                const int *__restrict__ tlen, const uint32_t *__restrict__ code,
                                const float4 *__restrict__ rec32, float4 *__restrict__ rec4) {
    const int o = blockIdx.x;
    const long long t0 = toff[o];
    const int K = tlen[o];
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        unsigned type = 4u;
        if (k > 0) {
            const uint32_t c1 = code[t0 + k], c0 = code[t0 + k - 1];
            int ddx = (int)(c1 & 0x7ffu) - (int)(c0 & 0x7ffu);
            int ddy = (int)((c1 >> 11) & 0x7ffu) - (int)((c0 >> 11) & 0x7ffu);
            const int ddz = (int)(c1 >> 22) - (int)(c0 >> 22);
            if (ddx == nx - 1) ddx = -1;  // wrapped offsets: a step across the
            if (ddx == 1 - nx) ddx = 1;   // periodic boundary
            if (ddy == ny - 1) ddy = -1;
            if (ddy == 1 - ny) ddy = 1;
            if (ddz == 0 && ddy == 0 && (ddx == 1 || ddx == -1)) type = ddx == 1 ? 0u : 1u;
            if (ddz == 0 && ddx == 0 && (ddy == 1 || ddy == -1)) type = ddy == 1 ? 2u : 3u;
        }
        const float4 r = rec32[t0 + k];
        const unsigned off = __float_as_uint(r.x);
        rec4[t0 + k] = make_float4(__uint_as_float(off | (type << kQuadOffBits)), r.y, r.z, r.w);
    }
}

// p.pairs from the replicated FP32 (chi, S): at every replicated index the
// values of that row and the next one, (chi(y), chi(y+1), S(y), S(y+1)); the
// last replicated row of a layer pairs with the layer's first (never read by
// an existing characteristic: the pair kernel reads rows <= 2 ny - 2).
__global__ void pair_pack_kernel(int nx, int ny, int nz, const float2 *__restrict__ chiS,
                                 float4 *__restrict__ P) {
    const int rows = 2 * ny * nz, w = 2 * nx;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const long long i0 = (long long)row * w;
        const long long next = (row % (2 * ny) + 1 < 2 * ny) ? w : w - 2LL * ny * w;
        for (int x = threadIdx.x; x < w; x += blockDim.x) {
            const float2 a = chiS[i0 + x], b = chiS[i0 + next + x];
            P[i0 + x] = make_float4(a.x, b.x, a.y, b.y);
        }
    }
}

// ---- FP64 formal solution without Lambda* (refinement residuals, FP64 mode
// after the first iteration). The FP64 pipe is the bound, so everything that
// can leave it does: branch tests on the high word of non-negative doubles
// (integer compares), reciprocals seeded in FP32, widening by integer moves.
// The FP64 helpers (hi_below, recip64, interval64) are in fs64_step.cuh.

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
    if (!p.homogeneous)
        I = entry_intensity(p.up[o], p.mu, o, ray, p.top_face, p.bot_face, p.bot_grad, p.I_top,
                            p.I_bot);
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

template <bool PARAB, bool BL>
void launch_fast_w(const FsParams &p, dim3 grid, int block, int widen, cudaStream_t s) {
    if (widen == 0) fs_fast_kernel<PARAB, 0, BL><<<grid, block, 0, s>>>(p);
    else if (widen == 1) fs_fast_kernel<PARAB, 1, BL><<<grid, block, 0, s>>>(p);
    else fs_fast_kernel<PARAB, 2, BL><<<grid, block, 0, s>>>(p);
}

template <bool PARAB>
void launch_quad_w(const FsParams &p, dim3 grid, int block, int widen, cudaStream_t s) {
    if (widen == 1) fs_quad_kernel<PARAB, 1><<<grid, block, 0, s>>>(p);
    else fs_quad_kernel<PARAB, 0><<<grid, block, 0, s>>>(p);
}

template <bool PARAB>
void launch_pair_w(const FsParams &p, dim3 grid, int block, int widen, cudaStream_t s) {
    if (widen == 0) fs_pair_kernel<PARAB, 0><<<grid, block, 0, s>>>(p);
    else if (widen == 1) fs_pair_kernel<PARAB, 1><<<grid, block, 0, s>>>(p);
    else fs_pair_kernel<PARAB, 2><<<grid, block, 0, s>>>(p);
}

bool quad_applicable(const FsParams &p) {
    return p.rec4 != nullptr && 4LL * p.nx * p.ny * p.nz <= (long long)kQuadOffMask;
}

cudaError_t launch_quad_rec(const Template &t, int nx, int ny, float4 *rec4, cudaStream_t s) {
    quad_rec_kernel<<<t.nangles, 256, 0, s>>>(nx, ny, t.toff, t.tlen, t.code, t.rec32, rec4);
    return cudaGetLastError();
}

bool fs_shape_valid(const FsShape &sh) {
    return (sh.block == 64 || sh.block == 128 || sh.block == 256) &&
           (sh.rays_per_thread == 1 || sh.rays_per_thread == 2 || sh.rays_per_thread == 4) &&
           sh.widen >= 0 && sh.widen <= 2 &&
           (sh.branchless == 0 || sh.branchless == 1);
}

cudaError_t launch_fs_fast(const FsParams &p, bool parabolic, const FsShape &sh, cudaStream_t s) {
    if (!fs_shape_valid(sh)) return cudaErrorInvalidValue;
    if (sh.rays_per_thread >= 2) {
        if (!p.pairs) return cudaErrorInvalidValue;
        if (sh.rays_per_thread == 4 && !quad_applicable(p)) return cudaErrorInvalidValue;
        const int rows = 2 * p.ny * p.nz;
        pair_pack_kernel<<<rows < 65536 ? rows : 65536, 256, 0, s>>>(
            p.nx, p.ny, p.nz, static_cast<const float2 *>(p.chiS), p.pairs);
        if (sh.rays_per_thread == 4) {
            const int nlanes = p.nx * ((p.ny + 3) / 4);
            dim3 grid((nlanes + sh.block - 1) / sh.block, p.nangles);
            if (parabolic) launch_quad_w<true>(p, grid, sh.block, sh.widen, s);
            else launch_quad_w<false>(p, grid, sh.block, sh.widen, s);
            return cudaGetLastError();
        }
        const int npair = p.nx * ((p.ny + 1) / 2);
        dim3 grid((npair + sh.block - 1) / sh.block, p.nangles);
        if (parabolic) launch_pair_w<true>(p, grid, sh.block, sh.widen, s);
        else launch_pair_w<false>(p, grid, sh.block, sh.widen, s);
        return cudaGetLastError();
    }
    dim3 grid((p.nx * p.ny + sh.block - 1) / sh.block, p.nangles);
    if (parabolic) {
        if (sh.branchless) launch_fast_w<true, true>(p, grid, sh.block, sh.widen, s);
        else launch_fast_w<true, false>(p, grid, sh.block, sh.widen, s);
    } else {
        if (sh.branchless) launch_fast_w<false, true>(p, grid, sh.block, sh.widen, s);
        else launch_fast_w<false, false>(p, grid, sh.block, sh.widen, s);
    }
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
    const long long cap = 16LL * device_sm_count();
    if (b > cap) b = cap;
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
