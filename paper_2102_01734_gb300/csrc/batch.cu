// Batched wavelengths: n_lambda independent ALI solves (Eq. alo) that share
// the geometry cache (Sec. 4.1: the tracks are the same for every wavelength).
// Every kernel takes its wavelength from the compacted list of active ones,
// alist[blockIdx.y] (or .z), and a block past the active count returns at
// once, so one captured sequence of launches (a CUDA graph) serves every
// iteration whatever the number of wavelengths still active; the host
// re-captures it with a smaller wavelength extent as wavelengths retire, so
// retired wavelengths cost no blocks at all. A wavelength
// retires on the device when the estimated error of its J (last change
// times rho/(1-rho), rho from the last kHist changes) is below tol, or when
// its changes stagnate (the FP32 floor), which hands it to the FP64
// refinement.
#include "fs_step.cuh"

namespace rt3d {

namespace {

__device__ __forceinline__ unsigned long long dbits(double x) {
    return (unsigned long long)__double_as_longlong(x);
}
__device__ __forceinline__ double bitsd(unsigned long long x) {
    return __longlong_as_double((long long)x);
}

__device__ __forceinline__ void bmax_atomic(double x, unsigned long long *dst) {
    __shared__ unsigned long long sm[32];
    unsigned long long b = dbits(fabs(x));
    if (x != x) b = 0x7ff8000000000000ULL;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, b, off);
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
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, b, off);
            b = o > b ? o : b;
        }
        if (lane == 0 && b) atomicMax(dst, b);
    }
    __syncthreads();
}

// S = (1 - eps) J + eps B into the four replicas of the packed (chi, S) of
// every active wavelength (blockIdx.y).
__global__ void b_source(int nx, int ny, int nz, const double *J, const double *eps,
                         const double *B, float2 *chiS, const BatchState *bs) {
    if ((int)blockIdx.y >= bs->nactive) return;
    const int l = bs->alist[blockIdx.y];
    const long long n = (long long)nx * ny * nz;
    const double *Jl = J + l * n, *el = eps + l * n, *Bl = B + l * n;
    float2 *cl = chiS + 4 * l * n;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long long)nx * ny));
        const float s = (float)((1.0 - el[v]) * Jl[v] + el[v] * Bl[v]);
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) cl[rep_index(x + a * nx, y + b * ny, z, nx, ny)].y = s;
    }
}

// FP32 formal solution (no Lambda*) of wavelength blockIdx.z into its
// replicated FP64 J: the per-point step of the unbatched kernel (fast_step),
// two points per trip, in the ray-bundle shape the batched autotuner chose
// (threads per block from the launch; CONV as in fs_fast_kernel: 0 the
// conversion instruction, 1 integer moves, 2 alternating; BL: parabolic
// correction without a branch).
template <bool PARAB, int CONV, bool BL>
__global__ void __launch_bounds__(256) b_fs(BatchFsParams p) {
    constexpr bool W0 = CONV == 1, W1 = CONV >= 1;
    if ((int)blockIdx.z >= p.bs->nactive) return;
    const int l = p.bs->alist[blockIdx.z];
    const int nray = p.nx * p.ny;
    const int ray = blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= nray) return;
    const long long n4 = 4LL * nray * p.nz;
    const int o = p.order[blockIdx.y];
    const int K = p.tlen[o];
    const float4 *__restrict__ rec = p.rec32 + p.toff[o];
    const float2 *__restrict__ chiS = p.chiS + l * n4;
    double *__restrict__ J = p.Jrep + l * n4;
    const long long lf = (long long)l * nray;
    const double I0 = entry_intensity(p.up[o], p.mu, o, ray, p.top_face ? p.top_face + lf : nullptr,
                                      p.bot_face ? p.bot_face + lf : nullptr,
                                      p.bot_grad ? p.bot_grad + lf : nullptr, p.I_top, p.I_bot);
    RayF s;
    s.live = true;
    s.base = ray % p.nx + 2 * p.nx * (ray / p.nx);
    s.I = (float)I0;
    const float4 r = __ldg(rec);
    s.vc = s.base + __float_as_int(r.x);
    const float2 cs = chiS[s.vc];
    s.hc = cs.x * r.z;
    s.u = s.hc;
    s.Sc = cs.y;
    s.Sp = cs.y;
    s.dS = 0.0f;
    s.ru = __fdividef(1.0f, s.hc);
    float cwc = r.y;
    int k = 1;
    for (; k + 1 < K; k += 2) {
        const float4 r1 = __ldg(rec + k), r2 = __ldg(rec + k + 1);
        fast_step<PARAB, W0, BL>(s, chiS, J, r1, cwc);
        fast_step<PARAB, W1, BL>(s, chiS, J, r2, r1.y);
        cwc = r2.y;
    }
    if (k < K) {
        const float4 r1 = __ldg(rec + k);
        fast_step<PARAB, W0, BL>(s, chiS, J, r1, cwc);
        cwc = r1.y;
    }
    const IntervalE f = interval_fast(s.u, PARAB ? s.ru : __fdividef(1.0f, s.u));
    s.I = fmaf(f.a, s.dS, fmaf(f.e0, s.Sp - s.I, s.I));
    atomicAdd(J + s.vc, (double)(cwc * s.I));
    if (!(fabsf(s.I) <= 3.402823466e38f))  // non-finite: make J NaN
        atomicAdd(J + s.vc, __longlong_as_double(0x7ff8000000000000LL));
}

// Jfs = fold(Jrep); r = Jfs - J; dJ0 = r / diag; Jrep zeroed for the next
// formal solution; per-wavelength sweep state reset.
__global__ void b_fold_init(int nx, int ny, int nz, double *Jrep, const double *J,
                            const double *inv_diag, double *r, double *dJ0, float *dJ0_32,
                            BatchState *bs) {
    if ((int)blockIdx.y >= bs->nactive) return;
    const int l = bs->alist[blockIdx.y];
    const long long n = (long long)nx * ny * nz;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        bs->done[l] = 0;
        bs->count[l] = 0;
        bs->rel[l] = 0ULL;
    }
    if (tid <= kBatchSweeps) {
        bs->dmax[l * (kBatchSweeps + 1) + tid] = 0ULL;
        bs->jmax[l * (kBatchSweeps + 1) + tid] = 0ULL;
    }
    double *Jr = Jrep + 4 * l * n;
    for (long long v = tid; v < n; v += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long long)nx * ny));
        const long long i0 = rep_index(x, y, z, nx, ny), i1 = rep_index(x + nx, y, z, nx, ny);
        const long long i2 = rep_index(x, y + ny, z, nx, ny), i3 = rep_index(x + nx, y + ny, z, nx, ny);
        const double jfs = (Jr[i0] + Jr[i1]) + (Jr[i2] + Jr[i3]);
        Jr[i0] = 0.0;
        Jr[i1] = 0.0;
        Jr[i2] = 0.0;
        Jr[i3] = 0.0;
        const double rv = jfs - J[l * n + v];
        r[l * n + v] = rv;
        const double d0 = rv * inv_diag[l * n + v];
        dJ0[l * n + v] = d0;
        dJ0_32[l * n + v] = (float)d0;
    }
}

// Jacobi sweep m of every active wavelength (FP32 products of the stored
// FP32 coefficients, FP64 state), with the stop test of the unbatched solve.
__global__ void __launch_bounds__(256) b_sweep(int nx, int ny, int nz, const float *__restrict__ a,
                                               const double *__restrict__ inv_diag,
                                               const double *__restrict__ r, double *buf0,
                                               double *buf1, float *b32_0, float *b32_1, int m,
                                               double tol, BatchState *bs) {
    if ((int)blockIdx.y >= bs->nactive) return;
    const int l = bs->alist[blockIdx.y];
    if (bs->done[l]) return;
    unsigned long long *dmx = bs->dmax + l * (kBatchSweeps + 1);
    unsigned long long *jmx = bs->jmax + l * (kBatchSweeps + 1);
    if (m >= 2) {
        if (bitsd(dmx[m - 1]) <= tol * bitsd(jmx[m - 1])) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                bs->done[l] = 1;
                bs->count[l] = m - 1;
            }
            return;
        }
    }
    const long long n = (long long)nx * ny * nz;
    double *dst = (m & 1 ? buf1 : buf0) + l * n;
    const float *src32 = ((m - 1) & 1 ? b32_1 : b32_0) + l * n;
    float *dst32 = (m & 1 ? b32_1 : b32_0) + l * n;
    const float *al = a + l * os_coef_count(n);
    const double *il = inv_diag + l * n, *rl = r + l * n;
    double dmax = 0.0, jmax = 0.0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < (int)n; v += gridDim.x * blockDim.x) {
        const float acc = os_stencil(al, src32, v, nx, ny, nz, Periodic{true, true, false});
        const double nv = (rl[v] + (double)acc) * il[v];
        dst[v] = nv;
        const float nf = (float)nv;
        dst32[v] = nf;
        dmax = fmax(dmax, (double)fabsf(nf - src32[v]));
        jmax = fmax(jmax, fabs(nv));
    }
    bmax_atomic(dmax, &dmx[m]);
    bmax_atomic(jmax, &jmx[m]);
}

// J += dJ (final sweep buffer); rel = max |dJ| / |J| per wavelength.
__global__ void b_update(int n, double *J, const double *buf0, const double *buf1,
                         int max_sweeps, BatchState *bs) {
    if ((int)blockIdx.y >= bs->nactive) return;
    const int l = bs->alist[blockIdx.y];
    const int cnt = bs->done[l] ? bs->count[l] : max_sweeps;
    const double *dJ = (cnt & 1 ? buf1 : buf0) + (long long)l * n;
    double *Jl = J + (long long)l * n;
    double rel = 0.0;
    bool bad = false;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const double d = dJ[v];
        const double jn = Jl[v] + d;
        Jl[v] = jn;
        if (d != 0.0) rel = fmax(rel, fabs(d) / fabs(jn));
        bad |= !(fabs(jn) <= 1.79e308);
    }
    bmax_atomic(bad ? __longlong_as_double(0x7ff8000000000000LL) : rel, &bs->rel[l]);
}

// Predicted further ALI iterations that retire a wavelength to the Krylov
// refinement (contraction near 1, eps near 0).
constexpr double kSlowIters = 300.0;

// Per wavelength: record the change, estimate the error from the last kHist
// changes, retire when converged (state 1), stagnated at the rounding floor
// of the formal solution or contracting so slowly that more than kSlowIters
// further iterations are predicted (state 2: both go to the Krylov
// refinement), failed (state 3: NaN) or out of iterations (state 4).
__global__ void b_retire(int nl, double tol, int max_iter, BatchState *bs) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nl || !bs->active[l]) return;
    const double rel = bitsd(bs->rel[l]);
    const int it = ++bs->iters[l];
    double *h = bs->hist + l * kHist;
    h[(it - 1) % kHist] = rel;
    if (!(rel == rel)) {
        bs->active[l] = 0;
        bs->state[l] = 3;
        return;
    }
    double rho = 0.9;
    if (it >= 2) {
        const int m = it - 1 < kHist - 1 ? it - 1 : kHist - 1;
        const double a = h[(it - 1 - m) % kHist];
        rho = (a > 0.0 && rel > 0.0) ? pow(rel / a, 1.0 / m) : 0.0;
        rho = rho > 0.999 ? 0.999 : rho;
    }
    const double est = rel * rho / (1.0 - rho);
    bs->est[l] = est;
    if (it >= 2 && est <= tol) {
        bs->active[l] = 0;
        bs->state[l] = 1;
    } else if (it >= kHist && rel > 0.7 * h[it % kHist] && rel < 1e-2) {
        bs->active[l] = 0;  // no decrease over the window: rounding floor
        bs->state[l] = 2;
    } else if (it >= kHist && rho > 0.0 && log(tol / est) / log(rho) > kSlowIters) {
        // slow contraction (eps near 0): more than kSlowIters further ALI
        // iterations predicted; the Krylov refinement takes it from here
        bs->active[l] = 0;
        bs->state[l] = 2;
    } else if (it >= max_iter) {
        bs->active[l] = 0;
        bs->state[l] = 4;
    }
}

// The active count and the compacted list of active wavelengths (one block
// of 1024 threads: an exclusive scan of the active flags per chunk of 1024).
__global__ void __launch_bounds__(1024) b_count_active(int nl, BatchState *bs) {
    __shared__ int wsum[32];
    __shared__ int total;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) total = 0;
    __syncthreads();
    for (int c0 = 0; c0 < nl; c0 += 1024) {
        const int l = c0 + threadIdx.x;
        const int f = l < nl ? bs->active[l] : 0;
        int incl = f;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int w = wsum[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, off);
                if (lane >= off) w += y;
            }
            wsum[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        const int pos = total + (wid ? wsum[wid - 1] : 0) + incl - f;
        if (f) bs->alist[pos] = l;
        __syncthreads();
        if (threadIdx.x == 0) total += wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) bs->nactive = total;
}

int grid_x(long long n, int threads, int cap) {
    long long b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <bool PARAB, bool BL>
void launch_b_fs_t(const BatchFsParams &p, dim3 grid, int block, int conv, cudaStream_t s) {
    if (conv == 0) b_fs<PARAB, 0, BL><<<grid, block, 0, s>>>(p);
    else if (conv == 1) b_fs<PARAB, 1, BL><<<grid, block, 0, s>>>(p);
    else b_fs<PARAB, 2, BL><<<grid, block, 0, s>>>(p);
}

}  // namespace

cudaError_t launch_b_source(const BatchFsParams &p, int nl, const double *J, const double *eps,
                            const double *B, cudaStream_t s) {
    const long long n = (long long)p.nx * p.ny * p.nz;
    b_source<<<dim3(grid_x(n, 256, 2 * device_sm_count()), nl), 256, 0, s>>>(p.nx, p.ny, p.nz, J, eps, B, p.chiS,
                                                              p.bs);
    return cudaGetLastError();
}

cudaError_t launch_b_fs(const BatchFsParams &p, int nl, const FsShape &sh, bool parabolic,
                        cudaStream_t s) {
    if (!fs_shape_valid(sh)) return cudaErrorInvalidValue;
    const int block = sh.block;  // one characteristic per thread
    dim3 grid((p.nx * p.ny + block - 1) / block, p.nangles, nl);
    if (parabolic) {
        if (sh.branchless) launch_b_fs_t<true, true>(p, grid, block, sh.widen, s);
        else launch_b_fs_t<true, false>(p, grid, block, sh.widen, s);
    } else {
        if (sh.branchless) launch_b_fs_t<false, true>(p, grid, block, sh.widen, s);
        else launch_b_fs_t<false, false>(p, grid, block, sh.widen, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_iteration(const BatchFsParams &p, int nl, int nlaunch, double *J,
                                   const double *eps, const double *B, const float *a,
                                   const double *inv_diag,
                                   double *r, double *buf0, double *buf1, float *b32_0,
                                   float *b32_1, int max_sweeps, double sweep_tol, double tol,
                                   int max_iter, bool parabolic, const FsShape &shape,
                                   cudaStream_t s) {
    const long long n = (long long)p.nx * p.ny * p.nz;
    const int gx = grid_x(n, 256, 2 * device_sm_count());
    const int nw = nlaunch;
    b_source<<<dim3(gx, nw), 256, 0, s>>>(p.nx, p.ny, p.nz, J, eps, B, p.chiS, p.bs);
    const cudaError_t fe = launch_b_fs(p, nw, shape, parabolic, s);
    if (fe != cudaSuccess) return fe;
    b_fold_init<<<dim3(gx < 2 ? 2 : gx, nw), 256, 0, s>>>(p.nx, p.ny, p.nz, p.Jrep, J, inv_diag,
                                                          r, buf0, b32_0, p.bs);
    for (int m = 1; m <= max_sweeps; ++m)
        b_sweep<<<dim3(gx, nw), 256, 0, s>>>(p.nx, p.ny, p.nz, a, inv_diag, r, buf0, buf1, b32_0,
                                            b32_1, m, sweep_tol, p.bs);
    b_update<<<dim3(gx, nw), 256, 0, s>>>((int)n, J, buf0, buf1, max_sweeps, p.bs);
    b_retire<<<(nl + 127) / 128, 128, 0, s>>>(nl, tol, max_iter, p.bs);
    b_count_active<<<1, 1024, 0, s>>>(nl, p.bs);
    return cudaGetLastError();
}

}  // namespace rt3d
