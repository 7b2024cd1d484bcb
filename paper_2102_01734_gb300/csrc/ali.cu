// Operator-splitting step (Sec. 2.2, Eq. alo) and its Jacobi solver (Sec. 4,
// "OS iteration"), with the reductions of the convergence test.
//
// The OS system for the correction dJ = J_new - J_old is
//   [1 - Lambda*(1 - eps)] dJ = r,  r = J_FS - J_old,
// a 27-point stencil periodic in x and y. os_prep folds (1 - eps) of the
// neighbour into the 26 off-diagonal coefficients a_d(v) = Lambda*[d][v] (1 -
// eps_{v+d}) (FP64, or FP32 in the mixed mode; blocks of 32 voxels with
// their 26 planes contiguous, os_coef_index) and stores 1/diag in FP64.
// A sweep reads the coefficients once (the HBM stream that bounds it), the
// neighbours of dJ through L1/L2, and writes dJ^{m+1} with the two maxima
// of the stop test. Sweeps are launched back to back; each reads the
// previous sweep's maxima and returns at once after the stop test is met,
// so a fixed launch sequence serves any sweep count.
#include "rt3d_internal.cuh"

namespace rt3d {

namespace {

__device__ __forceinline__ unsigned long long dbits(double x) {
    return (unsigned long long)__double_as_longlong(x);
}
__device__ __forceinline__ double bitsd(unsigned long long x) {
    return __longlong_as_double((long long)x);
}

// block-wide max of a non-negative double (NaN propagates: its bit pattern
// is above +inf), then one atomicMax per block.
__device__ __forceinline__ void block_max_atomic(double x, unsigned long long *dst) {
    __shared__ unsigned long long sm[32];
    unsigned long long b = dbits(fabs(x));
    if (x != x) b = 0x7ff8000000000000ULL;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        unsigned long long o = __shfl_xor_sync(0xffffffffu, b, off);
        b = o > b ? o : b;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = b;
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        b = lane < nw ? sm[lane] : 0ULL;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            unsigned long long o = __shfl_xor_sync(0xffffffffu, b, off);
            b = o > b ? o : b;
        }
        if (lane == 0 && b) atomicMax(dst, b);
    }
    __syncthreads();  // sm[] is reused by a following call
}

// Packed (chi, S) written to the four replicas of every voxel.
__global__ void pack_kernel(int nx, int ny, int nz, const double *chi, double scale,
                            const double *S, void *out, bool fp64) {
    const long long n = (long long)nx * ny * nz;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long long)nx * ny));
        const double c = chi[v] * scale, sv = S[v];
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                const long long r = rep_index(x + a * nx, y + b * ny, z, nx, ny);
                if (fp64) static_cast<double2 *>(out)[r] = make_double2(c, sv);
                else static_cast<float2 *>(out)[r] = make_float2((float)c, (float)sv);
            }
    }
}

// S = (1 - eps) J + eps B (or (1 - eps) J for the homogeneous problem),
// written into the S half of the four replicas of the packed (chi, S).
__global__ void source_kernel(int nx, int ny, int nz, const double *J, const double *eps,
                              const double *B, void *out, bool fp64, bool homogeneous) {
    const long long n = (long long)nx * ny * nz;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long long)nx * ny));
        const double e = eps[v];
        double sv = (1.0 - e) * J[v];
        if (!homogeneous) sv += e * B[v];
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                const long long r = rep_index(x + a * nx, y + b * ny, z, nx, ny);
                if (fp64) static_cast<double2 *>(out)[r].y = sv;
                else static_cast<float2 *>(out)[r].y = (float)sv;
            }
    }
}

// Bottom-face arrays of the LTE diffusion inner boundary (the test cases of
// Sec. 3.1): per column f and wavelength, dB/dtau = (B(z=0) - B(z=1)) /
// (1/2 (chi(z=0) + chi(z=1))), the one-sided difference over the unit centre
// spacing with the trapezoidal optical depth (tau grows inward), and the face
// intensity B(z=0) + 1/2 chi(z=0) dB/dtau, B carried linearly to the face half
// a voxel below the innermost centre; a single layer has gradient 0 and face
// value B(z=0).
__global__ void diffusion_bc_kernel(long long nf, int nz, int nl, const double *chi,
                                    const double *B, double *I_face, double *grad) {
    const long long n = nf * nl, N = nf * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long l = i / nf, f = i - l * nf;
        const double *c = chi + l * N, *b = B + l * N;
        if (nz < 2) {
            grad[i] = 0.0;
            I_face[i] = b[f];
            continue;
        }
        const double dtau = __dmul_rn(0.5, __dadd_rn(c[f], c[nf + f]));
        const double gr = __ddiv_rn(__dsub_rn(b[f], b[nf + f]), dtau);
        grad[i] = gr;
        I_face[i] = __dadd_rn(b[f], __dmul_rn(__dmul_rn(0.5, c[f]), gr));
    }
}

// neighbour index of (x, y, z) + (dx, dy, dz) with the periodic axes wrapped;
// -1 outside a non-periodic axis
__device__ __forceinline__ long long nb_index(int x, int y, int z, int dx, int dy, int dz, int nx,
                                              int ny, int nz, Periodic per) {
    int xx = x + dx, yy = y + dy, zz = z + dz;
    if (xx < 0 || xx >= nx) {
        if (!per.x) return -1;
        xx += xx < 0 ? nx : -nx;
    }
    if (yy < 0 || yy >= ny) {
        if (!per.y) return -1;
        yy += yy < 0 ? ny : -ny;
    }
    if (zz < 0 || zz >= nz) {
        if (!per.z) return -1;
        zz += zz < 0 ? nz : -nz;
    }
    return xx + (long long)nx * (yy + (long long)ny * zz);
}

template <typename A>
__global__ void os_prep_kernel(int nx, int ny, int nz, const double *L, const double *eps, A *a,
                               double *inv_diag, Periodic per, bool colour, ColourGeo cg,
                               double *diag) {
    const long long N = (long long)nx * ny * nz;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long long)nx * ny));
        const double dg = 1.0 - L[13 * N + v] * (1.0 - eps[v]);
        inv_diag[v] = 1.0 / dg;
        if (diag) diag[v] = dg;
        const int c = (x & 1) + 2 * (y & 1) + 4 * (z & 1);
        const long long k = (x >> 1) + (long long)cg.nxc[c] * ((y >> 1) + (long long)cg.nyc[c] * (z >> 1));
        int plane = 0;
        for (int d = 0; d < 27; ++d) {
            if (d == 13) continue;
            const long long u = nb_index(x, y, z, d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1, nx, ny, nz, per);
            double val = 0.0;
            if (u >= 0) val = L[(long long)d * N + v] * (1.0 - eps[u]);
            a[colour ? os_colour_index(plane, cg.blk[c], k) : os_coef_index(plane, v)] = (A)val;
            ++plane;
        }
    }
}

// Colour c of the eight-colour sweep: every voxel of the colour from its
// neighbours' values of this sweep where their colour comes earlier (in dst,
// already final) and of the last sweep otherwise (in src: later colours, and
// the same colour, which a periodic axis of odd length makes a neighbour
// across the seam); Jacobi inside a colour, as the oracle's sweep defines it.
// In the mixed mode (A = float) the products take the FP32 copies of the
// iterates (src32, dst32; written beside the FP64 values), as the Jacobi
// sweep does, and the stop-test maxima compare FP32 copies.
template <typename A>
__global__ void __launch_bounds__(256) gs_colour_kernel(int nx, int ny, int nz, ColourGeo cg, int c,
                                                        const A *__restrict__ a,
                                                        const double *__restrict__ inv_diag,
                                                        const double *__restrict__ r,
                                                        const double *__restrict__ src,
                                                        double *__restrict__ dst,
                                                        const float *__restrict__ src32,
                                                        float *__restrict__ dst32, int m, double tol,
                                                        OsState *st, Periodic per) {
    constexpr bool f32 = sizeof(A) == 4;
    if (st->done) return;
    if (c == 0 && m >= 2) {
        const double dm = bitsd(st->dmax[m - 1]), jm = bitsd(st->jmax[m - 1]);
        if (dm <= tol * jm) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                st->done = 1;
                st->count = m - 1;
            }
            return;
        }
    }
    const int px = c & 1, py = (c >> 1) & 1, pz = c >> 2;
    const int nxc = cg.nxc[c], nyc = cg.nyc[c];
    const long long cnt = cg.cnt[c], blk0 = cg.blk[c];
    const int nxy = nx * ny;
    A dmax = A(0), jmax = A(0);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < cnt;
         k += (long long)gridDim.x * blockDim.x) {
        const long long kxy = (long long)nxc * nyc;
        const int zi = (int)(k / kxy), rem = (int)(k - zi * kxy), yi = rem / nxc, xi = rem - yi * nxc;
        const int x = 2 * xi + px, y = 2 * yi + py, z = 2 * zi + pz;
        const int v = x + nx * (y + ny * z);
        const int X[3] = {os_nb_lo(x, nx, per.x), x, os_nb_hi(x, nx, per.x)};
        const int Y[3] = {os_nb_lo(y, ny, per.y), y, os_nb_hi(y, ny, per.y)};
        const int Z[3] = {os_nb_lo(z, nz, per.z), z, os_nb_hi(z, nz, per.z)};
        const A *__restrict__ ab = a + os_colour_index(0, blk0, k);
        A acc = A(0);
#pragma unroll
        for (int d = 0, pl = 0; d < 27; ++d) {
            if (d == 13) continue;
            const int xn = X[d % 3], yn = Y[(d / 3) % 3], zn = Z[d / 9];
            const int cn = (xn & 1) + 2 * (yn & 1) + 4 * (zn & 1);
            const int u = xn + nx * yn + nxy * zn;
            A xv;
            if constexpr (f32) xv = cn < c ? dst32[u] : src32[u];
            else xv = cn < c ? dst[u] : src[u];
            acc += ab[pl * 32] * xv;
            ++pl;
        }
        const double nv = (r[v] + (double)acc) * inv_diag[v];
        dst[v] = nv;
        if constexpr (f32) {
            const float nf = (float)nv;
            dst32[v] = nf;
            dmax = fmaxf(dmax, fabsf(nf - src32[v]));
            jmax = fmaxf(jmax, fabsf(nf));
        } else {
            dmax = fmax(dmax, fabs(nv - src[v]));
            jmax = fmax(jmax, fabs(nv));
        }
    }
    block_max_atomic((double)dmax, &st->dmax[m]);
    block_max_atomic((double)jmax, &st->jmax[m]);
}

// ---- BiCGStab (van der Vorst 1992) on A x = r, A = [1 - Lambda*(1 - eps)],
// from x = 0, as the oracle's orc_os_bicgstab: scalars on the device, dot
// products accumulated by the kernels that produce their operands.

// block sum of v (all threads), added to *out by thread 0 of each block
__device__ __forceinline__ void block_sum_atomic(double v, double *out) {
    __shared__ double part[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) part[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? part[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) atomicAdd(out, v);
    }
}

// (A x)_v = diag_v x_v - sum_d a_d(v) x_{v+d}
template <typename A>
__device__ __forceinline__ double os_apply(const A *a, const double *diag, const double *x, int v,
                                           int nx, int ny, int nz, Periodic per) {
    return diag[v] * x[v] - (double)os_stencil(a, x, v, nx, ny, nz, per);
}

__global__ void bicg_init_kernel(int n, const double *r, BicgVecs vv, BicgState *bs) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        bs->rho = bs->alpha = bs->omega = 1.0;
        bs->rhv = bs->tt = bs->ts = bs->rr = 0.0;
    }
    double acc = 0.0;
    for (int i = tid; i < n; i += gridDim.x * blockDim.x) {
        const double ri = r[i];
        vv.x[i] = 0.0;
        vv.res[i] = ri;
        vv.rh[i] = ri;
        vv.p[i] = 0.0;
        vv.vv[i] = 0.0;
        acc += ri * ri;
    }
    block_sum_atomic(acc, &bs->rr0);
}

// rho1 = rh . res
__global__ void bicg_rho_kernel(int n, BicgVecs v, BicgState *bs) {
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        acc += v.rh[i] * v.res[i];
    block_sum_atomic(acc, &bs->rho1);
}

// p = res + beta (p - omega vv), beta = (rho1/rho)(alpha/omega)
__global__ void bicg_p_kernel(int n, BicgVecs v, BicgState *bs) {
    const double beta = (bs->rho1 / bs->rho) * (bs->alpha / bs->omega), om = bs->omega;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        v.p[i] = v.res[i] + beta * (v.p[i] - om * v.vv[i]);
}

// vv = A p; rhv = rh . vv
template <typename A>
__global__ void __launch_bounds__(256) bicg_vv_kernel(int nx, int ny, int nz, const A *__restrict__ a,
                                                      const double *__restrict__ diag, BicgVecs v,
                                                      BicgState *bs, Periodic per) {
    const int n = nx * ny * nz;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double y = os_apply(a, diag, v.p, i, nx, ny, nz, per);
        v.vv[i] = y;
        acc += v.rh[i] * y;
    }
    block_sum_atomic(acc, &bs->rhv);
}

// alpha = rho1 / rhv; sv = res - alpha vv
__global__ void bicg_s_kernel(int n, BicgVecs v, BicgState *bs) {
    const double alpha = bs->rho1 / bs->rhv;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        v.sv[i] = v.res[i] - alpha * v.vv[i];
}

// t = A sv; tt = t . t; ts = t . sv
template <typename A>
__global__ void __launch_bounds__(256) bicg_t_kernel(int nx, int ny, int nz, const A *__restrict__ a,
                                                     const double *__restrict__ diag, BicgVecs v,
                                                     BicgState *bs, Periodic per) {
    const int n = nx * ny * nz;
    double att = 0.0, ats = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double y = os_apply(a, diag, v.sv, i, nx, ny, nz, per);
        v.t[i] = y;
        att += y * y;
        ats += y * v.sv[i];
    }
    block_sum_atomic(att, &bs->tt);
    block_sum_atomic(ats, &bs->ts);
}

// omega = ts / tt (0 if tt = 0); x += alpha p + omega sv; res = sv - omega t;
// rr = res . res
__global__ void bicg_x_kernel(int n, BicgVecs v, BicgState *bs) {
    const double alpha = bs->rho1 / bs->rhv;
    const double om = bs->tt > 0.0 ? bs->ts / bs->tt : 0.0;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        v.x[i] += alpha * v.p[i] + om * v.sv[i];
        const double ri = v.sv[i] - om * v.t[i];
        v.res[i] = ri;
        acc += ri * ri;
    }
    block_sum_atomic(acc, &bs->rr);
}

// end of an iteration: rho = rho1, alpha and omega kept; accumulators of the
// next iteration zeroed (rr stays for the host's stop test)
__global__ void bicg_next_kernel(BicgState *bs) {
    bs->alpha = bs->rho1 / bs->rhv;
    bs->omega = bs->tt > 0.0 ? bs->ts / bs->tt : 0.0;
    bs->rho = bs->rho1;
    bs->rho1 = 0.0;
    bs->rhv = 0.0;
    bs->tt = 0.0;
    bs->ts = 0.0;
}

__global__ void bicg_zero_rr_kernel(BicgState *bs) { bs->rr = 0.0; }

__global__ void os_set_result_kernel(int n, const double *src, double *dst, int k, OsState *st) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        st->done = 1;
        st->count = k;
        st->sweeps_total += (unsigned long long)k;
    }
    if (dst != src)
        for (int i = tid; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i];
}

// r = Jfs - J (+ extra); dJ0 = r / diag; resets the sweep state.
__global__ void os_init_kernel(int n, const double *Jfs, const double *J, const double *extra,
                               const double *inv_diag, double *r, double *dJ0, float *dJ0_32,
                               OsState *st) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        st->done = 0;
        st->count = 0;
    }
    if (tid < 260) {
        st->dmax[tid] = 0ULL;
        st->jmax[tid] = 0ULL;
    }
    for (int v = tid; v < n; v += gridDim.x * blockDim.x) {
        double rv = Jfs ? Jfs[v] : 0.0;
        if (J) rv -= J[v];
        if (extra) rv += extra[v];
        r[v] = rv;
        const double d0 = rv * inv_diag[v];
        dJ0[v] = d0;
        if (dJ0_32) dJ0_32[v] = (float)d0;
    }
}

// One Jacobi sweep dst = (r + sum_d a_d src_{v+d}) / diag over all voxels
// (os_stencil), with the stop test of the previous sweep first. The mixed
// mode (A = float) multiplies by the FP32 copy of the previous sweep and
// keeps the iterate, r and 1/diag in FP64; its stop test compares against
// that copy.
template <typename A>
__global__ void __launch_bounds__(256) os_sweep_kernel(int nx, int ny, int nz, const A *__restrict__ a,
                                                       const double *__restrict__ inv_diag,
                                                       const double *__restrict__ r,
                                                       const double *__restrict__ src,
                                                       double *__restrict__ dst,
                                                       const float *__restrict__ src32,
                                                       float *__restrict__ dst32, int m, double tol,
                                                       OsState *st, Periodic per) {
    if (st->done) return;
    if (m >= 2) {
        const double dm = bitsd(st->dmax[m - 1]), jm = bitsd(st->jmax[m - 1]);
        if (dm <= tol * jm) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                st->done = 1;
                st->count = m - 1;
            }
            return;
        }
    }
    constexpr bool f32 = sizeof(A) == 4;
    const int N = nx * ny * nz;
    // stop-test maxima in A (FP32 in the mixed mode: a 1e-3 relative test)
    A dmax = A(0), jmax = A(0);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
        A acc;
        if constexpr (f32) acc = os_stencil(a, src32, v, nx, ny, nz, per);
        else acc = os_stencil(a, src, v, nx, ny, nz, per);
        const double nv = (r[v] + (double)acc) * inv_diag[v];
        dst[v] = nv;
        if constexpr (f32) {
            const float nf = (float)nv;
            dst32[v] = nf;
            dmax = fmaxf(dmax, fabsf(nf - src32[v]));
            jmax = fmaxf(jmax, fabsf(nf));
        } else {
            dmax = fmax(dmax, fabs(nv - src[v]));
            jmax = fmax(jmax, fabs(nv));
        }
    }
    block_max_atomic((double)dmax, &st->dmax[m]);
    block_max_atomic((double)jmax, &st->jmax[m]);
}

__global__ void os_finish_kernel(int max_sweeps, double tol, OsState *st) {
    if (!st->done) {
        st->done = 1;
        st->count = max_sweeps;
    }
    st->sweeps_total += (unsigned long long)st->count;
}

// J += dJ (dJ = the final sweep buffer); rel = max |dJ| / |J_new|.
__global__ void ali_update_kernel(int n, double *J, double *const *buf, OsState *st,
                                  double *dJ_out) {
    const double *dJ = buf[st->count & 1];
    double rel = 0.0;
    bool bad = false;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const double d = dJ[v];
        const double jn = J[v] + d;
        J[v] = jn;
        if (dJ_out) dJ_out[v] = d;
        if (d != 0.0) rel = fmax(rel, fabs(d) / fabs(jn));
        bad |= !(fabs(jn) <= 1.79e308);
    }
    block_max_atomic(bad ? __longlong_as_double(0x7ff8000000000000LL) : rel, &st->rel);
}

__global__ void copy_buf_kernel(int n, double *const *buf, const OsState *st, double *dst) {
    const double *src = buf[st->count & 1];
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        dst[v] = src[v];
}

// J += d; rel = max |d| / |J_new|; amax = max |d|.
__global__ void axpy_rel_kernel(int n, double *J, const double *d, OsState *st) {
    double rel = 0.0;
    bool bad = false;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const double jn = J[v] + d[v];
        J[v] = jn;
        if (d[v] != 0.0) rel = fmax(rel, fabs(d[v]) / fabs(jn));
        bad |= !(fabs(jn) <= 1.79e308);
    }
    block_max_atomic(bad ? __longlong_as_double(0x7ff8000000000000LL) : rel, &st->rel);
}

// r = Jfs - J; res = max |r| / |J|.
__global__ void residual_kernel(int n, const double *Jfs, const double *J, double *r,
                                OsState *st) {
    double res = 0.0;
    bool bad = false;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const double rv = Jfs[v] - J[v];
        if (r) r[v] = rv;
        if (rv != 0.0) res = fmax(res, fabs(rv) / fabs(J[v]));
        bad |= !(fabs(rv) <= 1.79e308);
    }
    block_max_atomic(bad ? __longlong_as_double(0x7ff8000000000000LL) : res, &st->res);
}

__global__ void compare_kernel(long long n, const double *a, const double *b, OsState *st) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (__double_as_longlong(a[i]) != __double_as_longlong(b[i])) {
            st->changed = 1;
            return;
        }
    }
}

int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    const long long cap = 16LL * device_sm_count();
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

cudaError_t launch_pack(int nx, int ny, int nz, const double *chi, double scale, const double *S,
                        void *chiS, bool fp64, cudaStream_t s) {
    const long long n = (long long)nx * ny * nz;
    pack_kernel<<<grid_for(n, 256), 256, 0, s>>>(nx, ny, nz, chi, scale, S, chiS, fp64);
    return cudaGetLastError();
}

cudaError_t launch_source(int nx, int ny, int nz, const double *J, const double *eps,
                          const double *B, void *chiS, bool fp64, bool homogeneous,
                          cudaStream_t s) {
    const long long n = (long long)nx * ny * nz;
    source_kernel<<<grid_for(n, 256), 256, 0, s>>>(nx, ny, nz, J, eps, B, chiS, fp64, homogeneous);
    return cudaGetLastError();
}

cudaError_t launch_diffusion_bc(int nx, int ny, int nz, int nl, const double *chi,
                                const double *B, double *I_face, double *grad, cudaStream_t s) {
    const long long nf = (long long)nx * ny;
    diffusion_bc_kernel<<<grid_for(nf * nl, 256), 256, 0, s>>>(nf, nz, nl, chi, B, I_face, grad);
    return cudaGetLastError();
}

ColourGeo colour_geo(int nx, int ny, int nz) {
    ColourGeo cg{};
    long long blk = 0;
    for (int c = 0; c < 8; ++c) {
        const int px = c & 1, py = (c >> 1) & 1, pz = c >> 2;
        cg.nxc[c] = (nx - px + 1) / 2;
        cg.nyc[c] = (ny - py + 1) / 2;
        const long long nzc = (nz - pz + 1) / 2;
        cg.cnt[c] = (long long)cg.nxc[c] * cg.nyc[c] * nzc;
        cg.blk[c] = blk;
        blk += (cg.cnt[c] + 31) >> 5;
    }
    return cg;
}

cudaError_t launch_gs_sweep(int nx, int ny, int nz, const ColourGeo &cg, const void *a, bool a64,
                            const double *inv_diag, const double *r, const double *src,
                            double *dst, const float *src32, float *dst32, int m, double tol,
                            OsState *st, cudaStream_t s, Periodic per) {
    for (int c = 0; c < 8; ++c) {
        const int blocks = grid_for(cg.cnt[c] > 0 ? cg.cnt[c] : 1, 256);
        if (a64)
            gs_colour_kernel<double><<<blocks, 256, 0, s>>>(nx, ny, nz, cg, c,
                                                            static_cast<const double *>(a), inv_diag,
                                                            r, src, dst, nullptr, nullptr, m, tol,
                                                            st, per);
        else
            gs_colour_kernel<float><<<blocks, 256, 0, s>>>(nx, ny, nz, cg, c,
                                                           static_cast<const float *>(a), inv_diag, r,
                                                           src, dst, src32, dst32, m, tol, st, per);
    }
    return cudaGetLastError();
}

cudaError_t launch_bicg_init(int n, const double *r, const BicgVecs &v, BicgState *bs,
                             cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(&bs->rr0, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(&bs->rho1, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    bicg_init_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, r, v, bs);
    return cudaGetLastError();
}

cudaError_t launch_bicg_iteration(int nx, int ny, int nz, const void *a, bool a64,
                                  const double *diag, const BicgVecs &v, BicgState *bs,
                                  cudaStream_t s, Periodic per) {
    const int n = nx * ny * nz;
    const int b = grid_for(n, 256);
    bicg_rho_kernel<<<b, 256, 0, s>>>(n, v, bs);
    bicg_p_kernel<<<b, 256, 0, s>>>(n, v, bs);
    if (a64) bicg_vv_kernel<double><<<b, 256, 0, s>>>(nx, ny, nz, static_cast<const double *>(a), diag, v, bs, per);
    else bicg_vv_kernel<float><<<b, 256, 0, s>>>(nx, ny, nz, static_cast<const float *>(a), diag, v, bs, per);
    bicg_s_kernel<<<b, 256, 0, s>>>(n, v, bs);
    if (a64) bicg_t_kernel<double><<<b, 256, 0, s>>>(nx, ny, nz, static_cast<const double *>(a), diag, v, bs, per);
    else bicg_t_kernel<float><<<b, 256, 0, s>>>(nx, ny, nz, static_cast<const float *>(a), diag, v, bs, per);
    bicg_zero_rr_kernel<<<1, 1, 0, s>>>(bs);
    bicg_x_kernel<<<b, 256, 0, s>>>(n, v, bs);
    bicg_next_kernel<<<1, 1, 0, s>>>(bs);
    return cudaGetLastError();
}

cudaError_t launch_os_set_result(int n, const double *src, double *dst, int k, OsState *st,
                                 cudaStream_t s) {
    os_set_result_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, src, dst, k, st);
    return cudaGetLastError();
}

cudaError_t launch_os_prep(int nx, int ny, int nz, const double *lstar, const double *eps,
                           void *a, bool a64, double *inv_diag, cudaStream_t s, Periodic per,
                           bool colour, double *diag) {
    const long long N = (long long)nx * ny * nz;
    const ColourGeo cg = colour_geo(nx, ny, nz);
    if (a64)
        os_prep_kernel<double><<<grid_for(N, 256), 256, 0, s>>>(
            nx, ny, nz, lstar, eps, static_cast<double *>(a), inv_diag, per, colour, cg, diag);
    else
        os_prep_kernel<float><<<grid_for(N, 256), 256, 0, s>>>(
            nx, ny, nz, lstar, eps, static_cast<float *>(a), inv_diag, per, colour, cg, diag);
    return cudaGetLastError();
}

cudaError_t launch_os_init(int n, const double *Jfs, const double *J, const double *extra,
                           const double *inv_diag, double *r, double *dJ0, float *dJ0_32,
                           OsState *st, cudaStream_t s) {
    int g = grid_for(n, 256);
    if (g < 2) g = 2;  // >= 260 threads to reset the sweep maxima
    os_init_kernel<<<g, 256, 0, s>>>(n, Jfs, J, extra, inv_diag, r, dJ0, dJ0_32, st);
    return cudaGetLastError();
}

cudaError_t launch_os_sweep(int nx, int ny, int nz, const void *a, bool a64,
                            const double *inv_diag, const double *r, double *const *buf,
                            float *const *buf32, int m, double tol, OsState *st, cudaStream_t s,
                            Periodic per) {
    // buf, buf32: host arrays of the two device ping-pong buffers (FP64, FP32 copy)
    const long long N = (long long)nx * ny * nz;
    const double *src = buf[(m - 1) & 1];
    double *dst = buf[m & 1];
    const float *src32 = buf32 ? buf32[(m - 1) & 1] : nullptr;
    float *dst32 = buf32 ? buf32[m & 1] : nullptr;
    if (a64)
        os_sweep_kernel<double><<<grid_for(N, 256), 256, 0, s>>>(
            nx, ny, nz, static_cast<const double *>(a), inv_diag, r, src, dst, src32, dst32, m, tol,
            st, per);
    else
        os_sweep_kernel<float><<<grid_for(N, 256), 256, 0, s>>>(
            nx, ny, nz, static_cast<const float *>(a), inv_diag, r, src, dst, src32, dst32, m, tol,
            st, per);
    return cudaGetLastError();
}

cudaError_t launch_os_finish(int max_sweeps, double tol, OsState *st, cudaStream_t s) {
    os_finish_kernel<<<1, 1, 0, s>>>(max_sweeps, tol, st);
    return cudaGetLastError();
}

cudaError_t launch_ali_update(int n, double *J, double *const *buf, OsState *st, double *dJ_out,
                              cudaStream_t s) {
    ali_update_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, J, buf, st, dJ_out);
    return cudaGetLastError();
}

cudaError_t launch_copy_buf(int n, double *const *buf, const OsState *st, double *dst,
                            cudaStream_t s) {
    copy_buf_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, buf, st, dst);
    return cudaGetLastError();
}

cudaError_t launch_axpy_rel(int n, double *J, const double *d, OsState *st, cudaStream_t s) {
    axpy_rel_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, J, d, st);
    return cudaGetLastError();
}

cudaError_t launch_residual(int n, const double *Jfs, const double *J, double *r, OsState *st,
                            cudaStream_t s) {
    residual_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, Jfs, J, r, st);
    return cudaGetLastError();
}

cudaError_t launch_compare(long long n, const double *a, const double *b, OsState *st,
                           cudaStream_t s) {
    compare_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, a, b, st);
    return cudaGetLastError();
}

}  // namespace rt3d
