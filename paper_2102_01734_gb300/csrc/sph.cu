// Spherical (r, theta, phi) grid of the paper's SP test case (Sec. 3.2):
// geometry cache of long characteristics and the formal solution over it.
//
// Ray set of a solid angle: the voxels are visited in index order and every
// voxel that no ray of this angle has crossed yet launches the full line
// through its centre, traced from its entry (outer sphere, or the core sphere
// r = r_in) to its exit; all cells it crosses are marked. One warp per
// angle builds the set (pass 1 counts rays and segments, pass 2 writes the
// tables). Crossings with the radial spheres, the polar cones (the plane z = 0
// for theta = pi/2) and the azimuthal half-planes are computed with
// round-to-nearest FP64 intrinsics (no contraction), sorted, equal parameters
// merged, and the cell of every interval found at its midpoint by comparisons
// only (r^2, z|z| against cos|cos| r^2, signs of cross products), so the
// cache is reproducible bit for bit. Per segment the cache stores the cell,
// its index in the 2 x 2-replicated packed (chi, S) array, the chord, the J
// weight w l / (chord sum of the cell for this angle) and the Lambda* window
// (neighbourhood in index space, periodic in phi only).
#include "fs_step.cuh"
#include "fs64_step.cuh"

namespace rt3d {

namespace {

__device__ __forceinline__ double dm(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double da(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double ds(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dd(double a, double b) { return __ddiv_rn(a, b); }

__device__ int sph_cell(const SphTables &T, double p0, double p1, double p2) {
    const double r2 = da(da(dm(p0, p0), dm(p1, p1)), dm(p2, p2));
    int ir = 0;
    while (ir + 1 < T.nr && T.re2[ir + 1] <= r2) ++ir;
    const double key = dm(p2, fabs(p2));
    int it = 0;
    while (it + 1 < T.nt && dm(T.ctk[it + 1], r2) >= key) ++it;
    int ip = 0;
    for (int k = 0; k < T.np; ++k) {
        const int k1 = (k + 1) % T.np;
        const double c0 = ds(dm(T.cpe[k], p1), dm(T.spe[k], p0));
        const double c1 = ds(dm(T.cpe[k1], p1), dm(T.spe[k1], p0));
        if (c0 >= 0.0 && c1 < 0.0) {
            ip = k;
            break;
        }
    }
    return ir + T.nr * (it + T.nt * ip);
}

__device__ __forceinline__ int nb_code_sph(int nr, int nt, int np, int a, int b) {
    const int ra = a % nr, ta = (a / nr) % nt, pa = a / (nr * nt);
    const int rb = b % nr, tb = (b / nr) % nt, pb = b / (nr * nt);
    const int dr = ra - rb, dt = ta - tb;
    int dp = pa - pb;
    if (dp < 0) dp += np;
    if (dp == np - 1) dp = -1;
    else if (dp > 1) return -1;
    if (dr < -1 || dr > 1 || dt < -1 || dt > 1) return -1;
    return (dr + 1) + 3 * (dt + 1) + 9 * (dp + 1);
}

// Warp-cooperative construction of one angle's ray set (one warp per angle,
// the same set and the same arithmetic as the sequential definition in the
// file header): the next launch voxel is the first unset bit of the angle's
// hit bitset at or after a cursor, found 1024 voxels at a time with a ballot;
// the crossing candidates of its line are generated lane-strided over the
// spheres, cones and half-planes (each candidate with the same FP64
// operations as a sequential scan), appended through ballots, sorted by a
// bitonic network in shared memory and merged by lane 0; the cells of the
// intervals are found lane-strided. Shared memory per warp: npow doubles
// (sort buffer, npow = power of two >= ncap), ncap doubles (merged
// parameters) and ncap ints (cells).
__global__ void __launch_bounds__(32) sph_build_kernel(SphBuildParams p, int npow) {
    extern __shared__ double smem[];
    double *sb = smem;                                      // [npow]
    double *ts = smem + npow;                               // [ncap]
    int *cells = reinterpret_cast<int *>(ts + p.ncap);      // [ncap]
    const int lane = threadIdx.x;
    const int lo = blockIdx.x;
    const int o = p.o0 + lo;
    if (lo >= p.nchunk || o >= p.nangles) return;
    const SphTables &T = p.T;
    const int N = T.nr * T.nt * T.np;
    const int words = (N + 31) / 32;
    unsigned *hit = p.hit + (long long)lo * words;
    for (int i = lane; i < words; i += 32) hit[i] = 0u;
    __syncwarp();
    const double d[3] = {p.dir[3 * o], p.dir[3 * o + 1], p.dir[3 * o + 2]};
    long long seg = p.pass == 2 ? p.seg_base[o] : 0;
    long long ray = p.pass == 2 ? p.ray_base[o] : 0;
    const long long seg0 = seg;
    int nrays = 0;
    int cursor = 0;
    for (;;) {
        // next voxel no line of this angle has crossed yet
        int v = -1;
        while (cursor < N) {
            const int w0 = cursor >> 5, wi = w0 + lane;
            unsigned fr = 0u;
            if (wi < words) {
                fr = ~__ldcg(hit + wi);
                if (wi == w0) fr &= ~0u << (cursor & 31);
                if (wi == words - 1 && (N & 31)) fr &= (1u << (N & 31)) - 1u;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, fr != 0u);
            if (bal) {
                const int f = __ffs(bal) - 1;
                const unsigned fm = __shfl_sync(0xffffffffu, fr, f);
                v = (w0 + f) * 32 + __ffs(fm) - 1;
                break;
            }
            cursor = (w0 + 32) * 32;
        }
        if (v < 0) break;
        cursor = v + 1;
        const int ir = v % T.nr, it = (v / T.nr) % T.nt, ip = v / (T.nr * T.nt);
        const double P[3] = {dm(dm(T.rc[ir], T.stc[it]), T.cpc[ip]),
                             dm(dm(T.rc[ir], T.stc[it]), T.spc[ip]), dm(T.rc[ir], T.ctc[it])};
        // ends of the line: entry through the outer sphere, or the core sphere
        const double b = da(da(dm(P[0], d[0]), dm(P[1], d[1])), dm(P[2], d[2]));
        const double P2 = da(da(dm(P[0], P[0]), dm(P[1], P[1])), dm(P[2], P[2]));
        const double disc = ds(dm(b, b), ds(P2, T.re2[T.nr]));
        const double sq = __dsqrt_rn(disc);
        double t0 = ds(-b, sq), t1 = da(-b, sq);
        int entry = 0;
        const double dc = ds(dm(b, b), ds(P2, T.re2[0]));
        if (dc > 0.0) {
            const double sc = __dsqrt_rn(dc);
            const double a = ds(-b, sc), c = da(-b, sc);
            if (c <= 0.0 && c > t0) {
                t0 = c;
                entry = 1;
            }
            if (a >= 0.0 && a < t1) t1 = a;
        }
        // crossing candidates strictly inside (t0, t1), appended in any order
        int n = 0;
        auto put = [&](bool ok, double t) {
            const unsigned bl = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const int at = n + __popc(bl & ((1u << lane) - 1u));
                if (at < npow) sb[at] = t;
            }
            n += __popc(bl);
        };
        for (int i0 = 1; i0 < T.nr; i0 += 32) {
            const int i = i0 + lane;
            bool ok1 = false, ok2 = false;
            double r1 = 0.0, r2 = 0.0;
            if (i < T.nr) {
                const double di = ds(dm(b, b), ds(P2, T.re2[i]));
                if (di > 0.0) {
                    const double s_ = __dsqrt_rn(di);
                    r1 = ds(-b, s_);
                    r2 = da(-b, s_);
                    ok1 = r1 > t0 && r1 < t1;
                    ok2 = r2 > t0 && r2 < t1;
                }
            }
            put(ok1, r1);
            put(ok2, r2);
        }
        for (int j0 = 1; j0 < T.nt; j0 += 32) {
            const int j = j0 + lane;
            bool ok1 = false, ok2 = false;
            double q1 = 0.0, q2 = 0.0;
            if (j < T.nt) {
                if (2 * j == T.nt) {
                    if (d[2] != 0.0) {
                        q1 = dd(-P[2], d[2]);
                        ok1 = q1 > t0 && q1 < t1;
                    }
                } else {
                    const double c2 = dm(T.ct[j], T.ct[j]);
                    const double A = ds(dm(d[2], d[2]), c2);
                    const double Bh = ds(dm(P[2], d[2]), dm(c2, b));
                    const double C = ds(dm(P[2], P[2]), dm(c2, P2));
                    int nq = 0;
                    double roots[2] = {0.0, 0.0};
                    if (A == 0.0) {
                        if (Bh != 0.0) roots[nq++] = dd(-C, dm(2.0, Bh));
                    } else {
                        const double dq = ds(dm(Bh, Bh), dm(A, C));
                        if (dq > 0.0) {
                            const double s_ = __dsqrt_rn(dq);
                            roots[nq++] = dd(ds(-Bh, s_), A);
                            roots[nq++] = dd(da(-Bh, s_), A);
                        }
                    }
                    for (int q = 0; q < nq; ++q) {
                        const double t = roots[q];
                        if (!(t > t0 && t < t1)) continue;
                        const double z = da(P[2], dm(t, d[2]));
                        if (dm(z, T.ct[j]) > 0.0) {
                            if (q == 0) {
                                q1 = t;
                                ok1 = true;
                            } else {
                                q2 = t;
                                ok2 = true;
                            }
                        }
                    }
                }
            }
            put(ok1, q1);
            put(ok2, q2);
        }
        for (int k0 = 0; k0 < T.np; k0 += 32) {
            const int k = k0 + lane;
            bool ok = false;
            double t = 0.0;
            if (k < T.np) {
                const double den = ds(dm(T.cpe[k], d[1]), dm(T.spe[k], d[0]));
                if (den != 0.0) {
                    t = dd(ds(dm(T.spe[k], P[0]), dm(T.cpe[k], P[1])), den);
                    if (t > t0 && t < t1) {
                        const double x = da(P[0], dm(t, d[0])), y = da(P[1], dm(t, d[1]));
                        ok = da(dm(T.cpe[k], x), dm(T.spe[k], y)) > 0.0;
                    }
                }
            }
            put(ok, t);
        }
        if (n + 2 > p.ncap || n > npow) {
            if (lane == 0) atomicCAS(p.err, 0, 4);
            return;
        }
        // bitonic sort of sb[0, npw) ascending (padding +Inf), npw = 2^k >= n
        int npw = 1;
        while (npw < n) npw <<= 1;
        for (int i = n + lane; i < npw; i += 32) sb[i] = __longlong_as_double(0x7ff0000000000000LL);
        __syncwarp();
        for (int kk = 2; kk <= npw; kk <<= 1) {
            for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                for (int i = lane; i < npw; i += 32) {
                    const int ix = i ^ jj;
                    if (ix > i) {
                        const double x = sb[i], y = sb[ix];
                        if ((x > y) == ((i & kk) == 0)) {
                            sb[i] = y;
                            sb[ix] = x;
                        }
                    }
                }
                __syncwarp();
            }
        }
        // merge equal parameters, t0 and t1 at the ends
        if (lane == 0) {
            ts[0] = t0;
            int m = 1;
            for (int i = 0; i < n; ++i)
                if (sb[i] != ts[m - 1]) ts[m++] = sb[i];
            if (t1 != ts[m - 1]) ts[m++] = t1;
            cells[0] = m;  // passed to the other lanes below
        }
        __syncwarp();
        const int m = __shfl_sync(0xffffffffu, lane == 0 ? cells[0] : 0, 0);
        __syncwarp();
        const int K = m - 1;
        if (lane == 0) atomicOr(hit + (v >> 5), 1u << (v & 31));
        for (int k = lane; k < K; k += 32) {
            const double mid = dm(0.5, da(ts[k], ts[k + 1]));
            const int c = sph_cell(T, da(P[0], dm(mid, d[0])), da(P[1], dm(mid, d[1])),
                                   da(P[2], dm(mid, d[2])));
            cells[k] = c;
            atomicOr(hit + (c >> 5), 1u << (c & 31));
        }
        __syncwarp();
        if (p.pass == 2) {
            for (int k = lane; k < K; k += 32) {
                const long long sidx = seg + k;
                const int c = cells[k];
                const int cr = c % T.nr, ct = (c / T.nr) % T.nt, cp = c / (T.nr * T.nt);
                const double l = ds(ts[k + 1], ts[k]);
                const float lh = (float)(0.5 * l);
                // the J weight's slot holds the cell until the weights are known
                p.rec[sidx] = make_float4(__int_as_float((int)rep_index(cr, ct, cp, T.nr, T.nt)),
                                          __int_as_float(c), lh, lh);
                p.len64[sidx] = l;
                // the Lambda* window of the segment (the run of points ending at
                // k + 1 in the 3^3 neighbourhood of its cell) must fit the nine
                // slots of the kernels that build Lambda*, which find it again
                // from the cells
                const int jend = (k + 1 < K) ? k + 1 : k;
                for (int j = jend; j >= 0; --j) {
                    if (nb_code_sph(T.nr, T.nt, T.np, cells[j], c) < 0) break;
                    if (j - k + 7 < 0) {
                        atomicCAS(p.err, 0, 3);
                        break;
                    }
                }
            }
            if (lane == 0) {
                p.ray_off[ray] = seg;
                p.ray_len[ray] = K;
                p.ray_angle[ray] = o;
                p.ray_launch[ray] = v;
                int kind = 0, face = 0;
                if (entry) {
                    kind = 2;
                    const int c0 = cells[0];
                    face = (c0 / T.nr) % T.nt + T.nt * (c0 / (T.nr * T.nt));
                } else if (da(P[0], dm(t0, d[0])) > 0.0 && d[0] < 0.0) {
                    kind = 1;
                }
                p.ray_kind[ray] = kind;
                p.ray_face[ray] = face;
            }
            ++ray;
        }
        seg += K;
        ++nrays;
        __syncwarp();
    }
    if (p.pass == 1) {
        if (lane == 0) {
            p.nrays[o] = nrays;
            p.nseg[o] = seg;
        }
        return;
    }
    // chord sum of every cell for this angle, in segment order (each cell's
    // sum accumulated by one lane), then the J weights
    double *den = p.den + (long long)lo * N;
    for (int c = lane; c < N; c += 32) den[c] = 0.0;
    __syncwarp();
    for (long long sg = seg0; sg < seg; ++sg) {
        const int c = __float_as_int(p.rec[sg].y);
        if ((c & 31) == lane) den[c] += p.len64[sg];
    }
    __syncwarp();
    const double w = p.wt[o];
    for (long long sg = seg0 + lane; sg < seg; sg += 32) {
        const double c = w * (p.len64[sg] / den[__float_as_int(p.rec[sg].y)]);
        const float hi = (float)c;
        p.rec[sg].y = hi;                 // the FP32 kernels' weight
        p.rec[sg].w = (float)(c - hi);   // with it, the FP64 weight to ~2^-48
    }
    for (int c = lane; c < N; c += 32)
        if (!(den[c] > 0.0)) atomicCAS(p.err, 0, 5);
}

// Interval functions (as on the Cartesian grid).
__device__ __forceinline__ void ifn(float u, float &E, float &a0, float &a, float &d) {
    if (u < 1.0f) {
        constexpr float c0 = 2.0f / 6.0f, c1 = -2.0f / 24.0f, c2 = 2.0f / 120.0f,
                        c3 = -2.0f / 720.0f, c4 = 2.0f / 5040.0f, c5 = -2.0f / 40320.0f,
                        c6 = 2.0f / 362880.0f, c7 = -2.0f / 3628800.0f, c8 = 2.0f / 39916800.0f;
        float q = fmaf(c8, u, c7);
        q = fmaf(q, u, c6);
        q = fmaf(q, u, c5);
        q = fmaf(q, u, c4);
        q = fmaf(q, u, c3);
        q = fmaf(q, u, c2);
        q = fmaf(q, u, c1);
        q = fmaf(q, u, c0);
        const float b = u * q;
        a = 0.5f * u * (1.0f - b);
        const float e0 = u * (1.0f - a);
        E = 1.0f - e0;
        a0 = e0 - a;
        d = a - b;
    } else {
        E = __expf(-u);
        const float ru = __fdividef(1.0f, u);
        const float e0 = 1.0f - E;
        a = fmaf(-e0, ru, 1.0f);
        a0 = fmaf(-(1.0f + u), E, 1.0f) * ru;
        d = fmaf(2.0f, a, -e0) * ru;
    }
}

constexpr double pcd(int m) {
    double f = 1.0;
    for (int i = 2; i <= m + 3; ++i) f *= i;
    return (m % 2 ? -2.0 : 2.0) / f;
}
// Taylor coefficients of p(u) = e2/u^3 = 2 sum_m (-1)^m u^m / (m+3)!
__constant__ double kPcd[18] = {pcd(0),  pcd(1),  pcd(2),  pcd(3),  pcd(4),  pcd(5),
                                pcd(6),  pcd(7),  pcd(8),  pcd(9),  pcd(10), pcd(11),
                                pcd(12), pcd(13), pcd(14), pcd(15), pcd(16), pcd(17)};

__device__ __forceinline__ void ifn(double u, double &E, double &a0, double &a, double &d) {
    if (u < 0.5) {
        double q = kPcd[17];
#pragma unroll
        for (int m = 16; m >= 0; --m) q = fma(q, u, kPcd[m]);
        const double b = u * q;
        a = 0.5 * u * (1.0 - b);
        const double e0 = u * (1.0 - a);
        E = 1.0 - e0;
        a0 = e0 - a;
        d = a - b;
    } else {
        E = exp(-u);
        const double ru = 1.0 / u;
        const double e0 = 1.0 - E;
        a = fma(-e0, ru, 1.0);
        a0 = fma(-(1.0 + u), E, 1.0) * ru;
        d = fma(2.0, a, -e0) * ru;
    }
}

template <typename R> struct V2s;
template <> struct V2s<float> { using T = float2; };
template <> struct V2s<double> { using T = double2; };

template <typename R> __device__ __forceinline__ R clamp01s(R x) {
    return x < R(0) ? R(0) : (x > R(1) ? R(1) : x);
}
__device__ __forceinline__ float divs(float x, float y) { return __fdividef(x, y); }
__device__ __forceinline__ double divs(double x, double y) { return x / y; }

// Lambda* neighbour code (dr+1) + 3 (dt+1) + 9 (dp+1) of cell a relative to
// cell b from their (r, theta, phi) indices (periodic in phi), -1 outside the
// 3^3 neighbourhood (as nb_code_sph).
__device__ __forceinline__ int nb_code_rtp(int ra, int ta, int pa, int rb, int tb, int pb, int np) {
    const int dr = ra - rb, dt = ta - tb;
    int dp = pa - pb;
    if (dp < 0) dp += np;
    if (dp == np - 1) dp = -1;
    else if (dp > 1) return -1;
    if (dr < -1 || dr > 1 || dt < -1 || dt > 1) return -1;
    return (dr + 1) + 3 * (dt + 1) + 9 * (dp + 1);
}

__device__ __forceinline__ double red_value_s(float x) { return widen_f32(x); }
__device__ __forceinline__ double red_value_s(double x) { return x; }

// One thread per characteristic of the cache (all angles flattened). Per
// segment it reads the record (cell index, FP32 J weight, half chord, and
// the weight's FP32 remainder) and, in FP64, the FP64 chord; the FP64 J
// weight is the record's two-float sum. With Lambda* the cells of the points
// k-7 .. k+1 ride along in registers and the passage window of point k (the
// run of points ending at k+1 inside the 3^3 neighbourhood of its cell, as
// the oracle defines it) is found from them.
template <typename R, bool PARAB, bool LSTAR>
__global__ void __launch_bounds__(128) sph_fs_kernel(SphFsParams p) {
    using R2 = typename V2s<R>::T;
    constexpr bool F64 = sizeof(R) == 8;
    const long long ray = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (ray >= p.nrays) return;
    const long long s0 = p.ray_off[ray];
    const int K = p.ray_len[ray];
    const int kind = p.ray_kind[ray];
    const R2 *__restrict__ chiS = static_cast<const R2 *>(p.chiS);
    const float4 *__restrict__ rec = p.rec + s0;
    const double *__restrict__ l64 = p.len64 + s0;
    // chord of segment k and its J weight in the kernel's precision (2 (l/2)
    // in FP32 is the FP32 chord exactly)
    auto seg_len = [&](int k) -> R {
        if constexpr (F64) return l64[k];
        else return 2.0f * __ldg(&rec[k].z);
    };
    auto seg_cw = [&](int k) -> R {
        if constexpr (F64) {
            const float4 r = __ldg(&rec[k]);
            return (double)r.y + (double)r.w;
        } else {
            return __ldg(&rec[k].y);
        }
    };
    double I0 = 0.0;
    if (!p.homogeneous) {
        if (kind == 2) I0 = p.core_face ? p.core_face[p.ray_face[ray]] : p.I_core;
        else if (kind == 1) I0 = p.I_irr;
        else I0 = p.I_out;
    }
    R I = (R)I0;
    const int nr2 = 2 * p.nr, nt2 = 2 * p.nt;
    int rep = __float_as_int(__ldg(&rec[0].x));
    int v = sph_cell_of_rep(rep, p.nr, p.nt);
    R2 cs = chiS[rep];
    R chil_c = cs.x * seg_len(0), chil_p = R(0);
    R S_c = cs.y, S_p = cs.y;
    R ring[kWin];
    // (r, theta, phi) of points k-8 .. k (slot 8 = the current point) before
    // the shift of step k; -8 marks no point
    int wr[kWin], wt[kWin], wp[kWin];
#pragma unroll
    for (int i = 0; i < kWin; ++i) {
        ring[i] = R(0);
        wr[i] = -8;
        wt[i] = -8;
        wp[i] = -8;
    }
    if (LSTAR) {
        const int q = rep / nr2, pc = q / nt2;
        wr[kWin - 1] = rep - q * nr2;
        wt[kWin - 1] = q - pc * nt2;
        wp[kWin - 1] = pc;
    }
    for (int k = 0; k < K; ++k) {
        const R u = R(0.5) * (chil_p + chil_c);
        R E, a0, a, d;
        ifn(u, E, a0, a, d);
        const bool has_next = k + 1 < K;
        int vn = v, repn = rep;
        R chil_n = R(0), S_n = S_c;
        if (has_next) {
            repn = __float_as_int(__ldg(&rec[k + 1].x));
            vn = sph_cell_of_rep(repn, p.nr, p.nt);
            const R2 c2 = chiS[repn];
            chil_n = c2.x * seg_len(k + 1);
            S_n = c2.y;
        }
        R al = a0, bg = a, ga = R(0);
        if (PARAB && has_next) {
            const R w = R(0.5) * (chil_c + chil_n);
            if (w > R(0)) {
                const R q = divs(u, w);
                const R fw = clamp01s(R(2) - R(2) * u) * clamp01s(R(2) - R(0.5) * q);
                if (fw > R(0)) {
                    const R sd = fw * divs(u, u + w) * d;
                    bg = a + sd;
                    ga = -q * sd;
                    al = a0 - sd;
                }
            }
        }
        I = E * I + al * S_p + bg * S_c + ga * (S_n - S_c);
        const R c = seg_cw(k);
        atomicAdd(p.J + v, red_value_s(c * I));
        if (LSTAR) {
            // cells of points k-7 .. k+1 in slots 0 .. 8
#pragma unroll
            for (int i = 0; i < kWin - 1; ++i) {
                wr[i] = wr[i + 1];
                wt[i] = wt[i + 1];
                wp[i] = wp[i + 1];
            }
            if (has_next) {
                const int q = repn / nr2, pc = q / nt2;
                wr[kWin - 1] = repn - q * nr2;
                wt[kWin - 1] = q - pc * nt2;
                wp[kWin - 1] = pc;
            } else {
                wr[kWin - 1] = -8;
            }
            // ring[i] = dI_k / dS_{k-7+i}
#pragma unroll
            for (int i = 0; i < kWin - 1; ++i) ring[i] = E * ring[i + 1];
            if (k == 0) ring[7] += al;
            else ring[6] += al;
            ring[7] += bg - ga;
            ring[8] = ga;
            // the window: from point k+1 (or k at the last point) backwards
            // while the points stay in the neighbourhood of point k's cell
            bool run = true;
#pragma unroll
            for (int i = kWin - 1; i >= 0; --i) {
                if (i == kWin - 1 && !has_next) continue;  // the last point: the run ends at k
                const int dc = run ? nb_code_rtp(wr[i], wt[i], wp[i], wr[7], wt[7], wp[7], p.np)
                                   : -1;
                run = dc >= 0;
                if (run) atomicAdd(p.lstar + (long long)dc * p.N + v, red_value_s(c * ring[i]));
            }
        }
        chil_p = chil_c;
        chil_c = chil_n;
        S_p = S_c;
        S_c = S_n;
        v = vn;
        rep = repn;
    }
    // the widening does not carry a non-finite value: a non-finite intensity
    // (it persists along the recurrence) makes J of the last point NaN
    if (!F64 && !(fabs((double)I) <= 1.79769313486231570e308))
        atomicAdd(p.J + v, __longlong_as_double(0x7ff8000000000000LL));
}

template <typename R, bool PARAB, bool LSTAR>
cudaError_t launch_sph_t(const SphFsParams &p, cudaStream_t s) {
    const long long blocks = (p.nrays + 127) / 128;
    sph_fs_kernel<R, PARAB, LSTAR><<<(unsigned)blocks, 128, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sph_build(const SphBuildParams &p, cudaStream_t s) {
    int npow = 1;
    while (npow < p.ncap) npow <<= 1;
    const size_t shm = sizeof(double) * (npow + p.ncap) + sizeof(int) * p.ncap;
    if (shm > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(sph_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        if (e != cudaSuccess) return e;
    }
    sph_build_kernel<<<p.nchunk, 32, shm, s>>>(p, npow);
    return cudaGetLastError();
}

namespace {

// FP32 formal solution without Lambda* on the spherical cache: the
// per-point step of the Cartesian kernel (fast_step, difference form) over
// per-segment records (replicated index of the cell as int bits, J weight, l/2,
// weight), one ray per thread in the builder's order (angle by angle, each
// angle's rays in the order their launch cells were found), so that the rays
// of a warp are mostly parallel neighbours whose gathers and reductions fall
// on nearby cells (21 % faster than ordering by ray length, which matches trip
// counts but scatters a warp over the shell); contributions reduced in FP64
// at the replicated index (folded afterwards).
template <bool PARAB>
__global__ void __launch_bounds__(128) sph_fs_fast_kernel(SphFsParams p, double *__restrict__ Jrep) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= p.nrays) return;
    const long long ray = idx;
    const long long s0 = p.ray_off[ray];
    const int K = p.ray_len[ray];
    const int kind = p.ray_kind[ray];
    const float4 *__restrict__ rr = p.rec + s0;
    const float2 *__restrict__ chiS = static_cast<const float2 *>(p.chiS);
    double I0 = 0.0;
    if (!p.homogeneous) {
        if (kind == 2) I0 = p.core_face ? p.core_face[p.ray_face[ray]] : p.I_core;
        else if (kind == 1) I0 = p.I_irr;
        else I0 = p.I_out;
    }
    RayF st;
    st.live = true;
    st.base = 0;
    st.I = (float)I0;
    const float4 r0 = __ldg(rr);
    st.vc = __float_as_int(r0.x);
    const float2 cs = chiS[st.vc];
    st.hc = cs.x * r0.z;
    st.u = st.hc;
    st.Sc = cs.y;
    st.Sp = cs.y;
    st.dS = 0.0f;
    st.ru = __fdividef(1.0f, fmaxf(st.hc, 1e-30f));
    float cwc = r0.y;
    // two points per trip; contributions widened by integer moves (the FP64
    // pipe stays free). Loading a point ahead (as the Cartesian pair kernel
    // does) was 4 % slower here: the lanes of a warp run rays of different
    // lengths, and the extra loads cost more than the latency they hide.
    int k = 1;
    for (; k + 1 < K; k += 2) {
        const float4 r1 = __ldg(rr + k), r2 = __ldg(rr + k + 1);
        fast_step<PARAB, true, false>(st, chiS, Jrep, r1, cwc);
        fast_step<PARAB, true, false>(st, chiS, Jrep, r2, r1.y);
        cwc = r2.y;
    }
    if (k < K) {
        const float4 r1 = __ldg(rr + k);
        fast_step<PARAB, true, false>(st, chiS, Jrep, r1, cwc);
        cwc = r1.y;
    }
    const IntervalE f = interval_fast(st.u, PARAB ? st.ru : __fdividef(1.0f, st.u));
    st.I = fmaf(f.a, st.dS, fmaf(f.e0, st.Sp - st.I, st.I));
    atomicAdd(Jrep + st.vc, widen_f32(cwc * st.I));
    if (!(fabsf(st.I) <= 3.402823466e38f))  // non-finite: make J NaN
        atomicAdd(Jrep + st.vc, __longlong_as_double(0x7ff8000000000000LL));
}

// FP64 formal solution without Lambda* on the spherical cache: the per-point
// step of the Cartesian FP64 kernel (fs64_fast_kernel: the update in
// difference form, FP32-seeded reciprocals, the fitted series for small
// optical depths, branch tests on high words) over the per-segment records,
// one ray per thread in the builder's order. Half chord l/2 from the FP64
// chord (exact), J weight the record's two-float sum; contributions reduced
// at the replicated index (folded afterwards).
template <bool PARAB>
__global__ void __launch_bounds__(128) sph_fs64_fast_kernel(SphFsParams p, double *__restrict__ Jrep) {
    const long long ray = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (ray >= p.nrays) return;
    const long long s0 = p.ray_off[ray];
    const int K = p.ray_len[ray];
    const int kind = p.ray_kind[ray];
    const float4 *__restrict__ rr = p.rec + s0;
    const double *__restrict__ l64 = p.len64 + s0;
    const double2 *__restrict__ chiS = static_cast<const double2 *>(p.chiS);
    double I = 0.0;
    if (!p.homogeneous) {
        if (kind == 2) I = p.core_face ? p.core_face[p.ray_face[ray]] : p.I_core;
        else if (kind == 1) I = p.I_irr;
        else I = p.I_out;
    }
    float4 r = __ldg(rr);
    int vc = __float_as_int(r.x);
    const double2 cs = chiS[vc];
    double hc = cs.x * (0.5 * __ldg(l64));  // half the optical depth of the point's chord
    double cwc = (double)r.y + (double)r.w;
    double u = hc;  // the entry interval: chi_{-1} l_{-1} = 0
    double Sc = cs.y, Sp = cs.y, dS = 0.0;  // S_{-1} = S_0
    double ru = PARAB ? recip64(hc) : 0.0;
    for (int k = 1; k < K; ++k) {
        r = __ldg(rr + k);
        const int vn = __float_as_int(r.x);
        const double2 cn = chiS[vn];
        const double hn = cn.x * (0.5 * __ldg(l64 + k));
        const double dSn = cn.y - Sc;
        const double w = hc + hn;
        const IntervalDE f = interval64<PARAB>(u, ru);
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
        atomicAdd(Jrep + vc, cwc * I);
        u = w;
        hc = hn;
        Sp = Sc;
        Sc = cn.y;
        dS = dSn;
        vc = vn;
        cwc = (double)r.y + (double)r.w;
    }
    const IntervalDE f = interval64<PARAB>(u, ru);
    I = fma(f.a, dS, fma(f.e0, Sp - I, I));
    atomicAdd(Jrep + vc, cwc * I);
}

}  // namespace

cudaError_t launch_sph_fs64_fast(const SphFsParams &p, double *Jrep, bool parabolic,
                                 cudaStream_t s) {
    const int threads = 128;
    const long long blocks = (p.nrays + threads - 1) / threads;
    if (parabolic) sph_fs64_fast_kernel<true><<<(unsigned)blocks, threads, 0, s>>>(p, Jrep);
    else sph_fs64_fast_kernel<false><<<(unsigned)blocks, threads, 0, s>>>(p, Jrep);
    return cudaGetLastError();
}

cudaError_t launch_sph_fs_fast(const SphFsParams &p, double *Jrep, bool parabolic,
                               cudaStream_t s) {
    const int threads = 128;
    const long long blocks = (p.nrays + threads - 1) / threads;
    if (parabolic) sph_fs_fast_kernel<true><<<(unsigned)blocks, threads, 0, s>>>(p, Jrep);
    else sph_fs_fast_kernel<false><<<(unsigned)blocks, threads, 0, s>>>(p, Jrep);
    return cudaGetLastError();
}

cudaError_t launch_sph_fs(const SphFsParams &p, bool fp64, bool parabolic, bool lstar,
                          cudaStream_t s) {
    if (fp64) {
        if (parabolic) return lstar ? launch_sph_t<double, true, true>(p, s) : launch_sph_t<double, true, false>(p, s);
        return lstar ? launch_sph_t<double, false, true>(p, s) : launch_sph_t<double, false, false>(p, s);
    }
    if (parabolic) return lstar ? launch_sph_t<float, true, true>(p, s) : launch_sph_t<float, true, false>(p, s);
    return lstar ? launch_sph_t<float, false, true>(p, s) : launch_sph_t<float, false, false>(p, s);
}

}  // namespace rt3d
