// Internal declarations of the CUDA library behind include/rt3d.h.
// Device-side geometry cache, kernel parameter blocks and launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/rt3d.h"

namespace rt3d {

// Longest passage-local Lambda* window (points j <= k+1 of one characteristic
// whose voxels lie in the 3x3x3 neighbourhood of point k), as ring positions
// 0..8 <-> points k-7 .. k+1.
constexpr int kWin = 9;
constexpr unsigned kWinNone = 31u;  // 5-bit code: ring position not in the window

// Packed step code of the reference characteristic (face cell (0,0)):
// wrapped x offset | wrapped y offset << 11 | z << 22.
__host__ __device__ inline uint32_t step_code(int dx, int dy, int z) {
    return (uint32_t)dx | ((uint32_t)dy << 11) | ((uint32_t)z << 22);
}

// Geometry cache on the device (Sec. 4.1: traced once, reused by every
// formal solution). One characteristic per solid angle; all nx*ny
// characteristics of that angle are integer translates of it.
struct Template {
    int nangles = 0;
    int kmax = 0;
    long long total = 0;        // points over all angles
    int *tlen = nullptr;        // [nangles] points of the characteristic
    long long *toff = nullptr;  // [nangles] offset of its first point
    int *order = nullptr;       // [nangles] angles by decreasing length
    signed char *up = nullptr;  // [nangles] 1 if mu > 0 (enters at the bottom)
    double *mu = nullptr;       // [nangles] direction cosine to the z axis
    uint32_t *code = nullptr;   // [total] step codes
    double *len64 = nullptr;    // [total] chords
    float *len32 = nullptr;
    double *cw64 = nullptr;     // [total] w_Omega l_k / (sum of l over the layer)
    float *cw32 = nullptr;
    uint64_t *win = nullptr;    // [total] Lambda* window: 9 x 5-bit neighbour codes
    // [total] FP32 step record for the formal solution without Lambda*:
    // (offset in the 2x2-replicated grid as int bits, J weight, l/2, l/2:
    // the last two form the aligned pair of the packed two-characteristic kernel)
    float4 *rec32 = nullptr;
    // [total] FP64 step record of the same: (l/2, J weight)
    double2 *rec64 = nullptr;
    // [total] FP32 step record of the four-characteristic kernel (FP32
    // grids of at most 2^27 voxels): rec32 with the step type in the top
    // three bits of the offset
    float4 *rec4 = nullptr;
};

// The packed (chi, S) arrays are replicated 2 x 2 in x and y: element
// (x, y, z) of the box sits at x + a nx + 2 nx (y + b ny + 2 ny z) for a, b in
// {0, 1}. A characteristic from face cell (x0, y0) then finds its point at
// replicated offset x0 + 2 nx y0 + o_k with o_k the cached offset of the
// reference characteristic (wrapped offsets are < nx, < ny), without any
// periodic wrap test.
__host__ __device__ inline long long rep_index(int x, int y, int z, int nx, int ny) {
    return (long long)x + 2LL * nx * ((long long)y + 2LL * ny * z);
}

// Intensity entering a characteristic through face cell f (Sec. 3.1): the
// top face's for mu < 0, the bottom face's for mu > 0, a face array
// overriding its scalar. A bottom gradient array gives the inner boundary the
// LTE diffusion form of the paper's test cases, I = I_bot + mu dB/dtau (tau
// the vertical optical depth, increasing inward), rounded as a product and a
// sum.
// mu (the direction cosines by angle) is read only with a gradient array.
__device__ __forceinline__ double entry_intensity(bool up, const double *mu, int o, long long f,
                                                  const double *top_face, const double *bot_face,
                                                  const double *bot_grad, double I_top,
                                                  double I_bot) {
    if (!up) return top_face ? top_face[f] : I_top;
    const double I = bot_face ? bot_face[f] : I_bot;
    return bot_grad ? __dadd_rn(I, __dmul_rn(mu[o], bot_grad[f])) : I;
}

struct FsParams {
    int nx, ny, nz;
    int nangles;
    const int *order;
    const long long *toff;
    const int *tlen;
    const signed char *up;
    const uint32_t *code;
    const void *len;   // float or double [total]
    const void *cw;    // float or double [total]
    const uint64_t *win;
    const void *chiS;  // float2 or double2 [4N]: (chi, S), replicated 2 x 2 in x, y
    double *J;         // [N], accumulated into (zeroed by the caller)
    const float4 *rec32;  // FP32 step records (fast path)
    const double2 *rec64; // FP64 (l/2, J weight) records (FP64 path without Lambda*)
    double *Jrep;      // [4N] replicated accumulation target of the fast path
    // [4N] pair-packed FP32 (chi, S) of the two-characteristic kernel: at the
    // replicated index of (x, y, z) the values of rows y and y + 1,
    // (chi(y), chi(y+1), S(y), S(y+1)); written from chiS by launch_fs_fast
    float4 *pairs;
    const float4 *rec4;  // nullable: step records of the four-characteristic kernel
    double *lstar;     // nullable [27][N], accumulated into
    const double *top_face;  // nullable [ny*nx]
    const double *bot_face;  // nullable [ny*nx]
    // nullable [ny*nx]: dB/dtau of the diffusion inner boundary, the upward
    // entry intensity being I_bot (face) + mu dB/dtau; mu = the template's
    const double *bot_grad;
    const double *mu;  // [nangles] direction cosines (read with bot_grad)
    double I_top, I_bot;
    double I_irr;      // spherical grid: irradiation
    int homogeneous;   // 1: zero boundary intensity, whatever the faces say
};

struct TraceParams {
    int nx, ny, nz, nangles;
    const double *dir;        // [nangles][3]
    const double *wt;         // [nangles]
    const long long *toff;    // [nangles]
    const int *cap;           // [nangles] capacity
    int *tlen;                // [nangles] out
    uint32_t *code;
    double *len64;
    float *len32;
    double *cw64;
    float *cw32;
    uint64_t *win;
    float4 *rec32;
    double2 *rec64;
    double *layer_sum;        // scratch [nangles][nz]
    int *err;                 // out: first error code (0 ok)
};

// Launchers (return the launch status).
cudaError_t launch_trace(const TraceParams &p, cudaStream_t s);
cudaError_t launch_fs(const FsParams &p, bool fp64, bool parabolic, bool lstar, cudaStream_t s);
// Ray-bundle shape of the FP32 formal solution without Lambda* (the same
// fields as the public rt3d_fs_shape).
struct FsShape {
    int block;            // 64, 128 or 256 threads
    int rays_per_thread;  // 1; 2: face rows y and y + 1 in packed FP32x2 arithmetic;
                          // 4: rows y .. y + 3, J summed across points in registers
    int widen;            // FP32 -> FP64: 0 conversion, 1 integer moves, 2 alternating
                          // (two per thread: the second characteristic by integer moves)
    int branchless;       // 1: parabolic correction evaluated without a branch
                          // (two per thread: always without)
};
bool fs_shape_valid(const FsShape &sh);
// whether the four-characteristic kernel can run on these parameters (its
// records exist and the replicated grid's offsets fit in 29 bits)
bool quad_applicable(const FsParams &p);
// the four-characteristic kernel's step records from the template
cudaError_t launch_quad_rec(const Template &t, int nx, int ny, float4 *rec4, cudaStream_t s);
// FP32 formal solution without Lambda* into p.Jrep (zero on entry; the fold
// zeroes it again).
cudaError_t launch_fs_fast(const FsParams &p, bool parabolic, const FsShape &sh, cudaStream_t s);
// Float-float formal solution without Lambda* into p.Jrep (zero on entry):
// recff = per-step (l/2, J weight) split, chiS = replicated split (chi, S)
cudaError_t launch_fsff(const FsParams &p, const float4 *recff, const float4 *chiS, bool parabolic,
                        cudaStream_t s);
// split (chi, S) into the four replicas; S = src, or (1 - eps) src + eps B
cudaError_t launch_pack_ff(int nx, int ny, int nz, const double *chi, const double *src,
                           const double *eps, const double *B, float4 *out, cudaStream_t s);
// split the FP64 step records (l/2, J weight)
cudaError_t launch_recff(long long total, const double2 *rec64, float4 *out, cudaStream_t s);
// FP64 formal solution without Lambda* into p.Jrep (zero on entry)
cudaError_t launch_fs64_fast(const FsParams &p, bool parabolic, cudaStream_t s);
// J[v] = sum of the four replicas of v in Jrep; zeroes Jrep
cudaError_t launch_fold(int nx, int ny, int nz, double *Jrep, double *J, cudaStream_t s);

// ---- ALI / OS kernels (ali.cu) ----
struct OsState {
    // reductions as bit patterns of non-negative doubles (atomicMax on u64)
    unsigned long long dmax[260];  // per sweep: max |dJ^{m+1} - dJ^m|
    unsigned long long jmax[260];  // per sweep: max |dJ^{m+1}|
    int done;
    int count;                     // sweeps done
    unsigned long long rel;        // max |dJ|/|J| of an update
    unsigned long long res;        // max |r|/|J| of a residual
    unsigned long long amax;       // max |x| of a vector
    int changed;                   // content comparison flag
    unsigned long long sweeps_total;  // sweeps of all OS solves since the last reset
};

cudaError_t launch_pack(int nx, int ny, int nz, const double *chi, double chi_scale,
                        const double *S, void *chiS, bool fp64, cudaStream_t s);
cudaError_t launch_source(int nx, int ny, int nz, const double *J, const double *eps,
                          const double *B, void *chiS, bool fp64, bool homogeneous,
                          cudaStream_t s);
// bottom-face (B, dB/dtau) of the diffusion inner boundary for nl stacked
// (chi, B) grids, outputs [nl][ny*nx]
cudaError_t launch_diffusion_bc(int nx, int ny, int nz, int nl, const double *chi,
                                const double *B, double *I_face, double *grad, cudaStream_t s);
// periodic axes of the 27-point OS stencil: Cartesian box x and y, spherical
// grid phi (the third index)
struct Periodic {
    bool x, y, z;
};
// Layout of the 26 folded OS coefficients a[plane][v]: blocks of 32
// consecutive voxels, each holding its 26 planes contiguously, so a warp's
// loads of one plane are one 128-byte (FP32) line at a fixed offset.
__host__ __device__ inline long long os_coef_index(int plane, long long v) {
    return ((v >> 5) * 26 + plane) * 32 + (v & 31);
}
__host__ __device__ inline long long os_coef_count(long long N) { return ((N + 31) >> 5) * 26 * 32; }

// Colour layout of the same coefficients for the eight-colour Gauss-Seidel
// sweep: colour c = (x&1) + 2(y&1) + 4(z&1); the voxels of a colour form a
// half-resolution sub-grid (x-major, index k); each colour holds blocks of 32
// consecutive k with their 26 planes contiguous, so the launch of one colour
// reads its coefficients as the Jacobi sweep reads its own.
struct ColourGeo {
    int nxc[8], nyc[8];
    long long cnt[8];  // voxels of colour c
    long long blk[8];  // first 32-voxel block of colour c
};
__host__ __device__ inline long long os_colour_index(int plane, long long blk0, long long k) {
    return ((blk0 + (k >> 5)) * 26 + plane) * 32 + (k & 31);
}
ColourGeo colour_geo(int nx, int ny, int nz);
// coefficients to allocate for either layout
__host__ __device__ inline long long os_coef_alloc(long long N) { return os_coef_count(N) + 8 * 26 * 32; }

// OS solver of a grid (rt3d_grid_set_os_solver)
enum OsKind { kOsJacobi = 0, kOsGaussSeidel = 1, kOsBicgstab = 2 };

#ifdef __CUDACC__
// Coordinate of the neighbour at offset -1 / +1 along an axis of n cells:
// wrapped on a periodic axis, else clamped to the cell itself (its
// coefficient is zero: os_prep stores 0 for a neighbour outside the grid).
__device__ __forceinline__ int os_nb_lo(int c, int n, bool periodic) {
    return c > 0 ? c - 1 : (periodic ? n - 1 : c);
}
__device__ __forceinline__ int os_nb_hi(int c, int n, bool periodic) {
    return c < n - 1 ? c + 1 : (periodic ? 0 : c);
}

// sum_d a_d(v) x_{v+d} over the 26 off-diagonal neighbours of voxel v:
// 26 coefficient loads from the voxel's warp-contiguous block (immediate
// offsets), 26 loads of x at indices built from 9 wrapped or clamped
// coordinates (no branch, all loads independent), then the products in A.
template <typename A, typename T>
__device__ __forceinline__ A os_stencil(const A *__restrict__ a, const T *__restrict__ x, int v,
                                        int nx, int ny, int nz, Periodic per) {
    const int nxy = nx * ny;
    const int z = v / nxy, rem = v - z * nxy, y = rem / nx, xx = rem - y * nx;
    const int X[3] = {os_nb_lo(xx, nx, per.x), xx, os_nb_hi(xx, nx, per.x)};
    const int Y[3] = {os_nb_lo(y, ny, per.y) * nx, y * nx, os_nb_hi(y, ny, per.y) * nx};
    const int Z[3] = {os_nb_lo(z, nz, per.z) * nxy, z * nxy, os_nb_hi(z, nz, per.z) * nxy};
    const A *__restrict__ ab = a + os_coef_index(0, v);
    A c[26], xv[26];
#pragma unroll
    for (int p = 0; p < 26; ++p) c[p] = ab[p * 32];
#pragma unroll
    for (int d = 0, p = 0; d < 27; ++d) {
        if (d == 13) continue;
        xv[p] = (A)x[X[d % 3] + Y[(d / 3) % 3] + Z[d / 9]];
        ++p;
    }
    A acc = A(0);
#pragma unroll
    for (int p = 0; p < 26; ++p) acc += c[p] * xv[p];
    return acc;
}
#endif
// folded coefficients a (os_coef_index layout, or the colour layout when
// colour is set), 1/diag and, when diag is given, diag itself
cudaError_t launch_os_prep(int nx, int ny, int nz, const double *lstar, const double *eps,
                           void *a, bool a64, double *inv_diag, cudaStream_t s,
                           Periodic per = {true, true, false}, bool colour = false,
                           double *diag = nullptr);
// One sweep of the eight-colour Gauss-Seidel iteration (colour layout of a):
// for colour 0 .. 7, every voxel of the colour from the neighbours' values
// of this sweep (earlier colours, in dst) or of the last (src); the stop test
// of sweep m - 1 first (as launch_os_sweep).
// src32/dst32: FP32 copies of src/dst (mixed mode; unused with a64)
cudaError_t launch_gs_sweep(int nx, int ny, int nz, const ColourGeo &cg, const void *a, bool a64,
                            const double *inv_diag, const double *r, const double *src,
                            double *dst, const float *src32, float *dst32, int m, double tol,
                            OsState *st, cudaStream_t s, Periodic per);
// BiCGStab on [1 - Lambda*(1 - eps)] x = r from x = 0 (van der Vorst):
// device scalars and the kernels of one iteration.
struct BicgState {
    double rho, alpha, omega;  // of the last iteration
    double rho1, rhv, tt, ts, rr;  // dot products (accumulated by the kernels)
    double rr0;
};
struct BicgVecs {
    double *x, *res, *rh, *p, *vv, *sv, *t;
};
cudaError_t launch_bicg_init(int n, const double *r, const BicgVecs &v, BicgState *bs,
                             cudaStream_t s);
cudaError_t launch_bicg_iteration(int nx, int ny, int nz, const void *a, bool a64,
                                  const double *diag, const BicgVecs &v, BicgState *bs,
                                  cudaStream_t s, Periodic per);
// dst = src; st: count = k, done, sweeps_total += k
cudaError_t launch_os_set_result(int n, const double *src, double *dst, int k, OsState *st,
                                 cudaStream_t s);
cudaError_t launch_os_init(int n, const double *Jfs, const double *J, const double *rhs_extra,
                           const double *inv_diag, double *r, double *dJ0, float *dJ0_32,
                           OsState *st, cudaStream_t s);
// buf32: FP32 copies of the ping-pong buffers (required when !a64)
cudaError_t launch_os_sweep(int nx, int ny, int nz, const void *a, bool a64,
                            const double *inv_diag, const double *r, double *const *buf,
                            float *const *buf32, int m, double tol, OsState *st, cudaStream_t s,
                            Periodic per = {true, true, false});
cudaError_t launch_os_finish(int max_sweeps, double tol, OsState *st, cudaStream_t s);
cudaError_t launch_ali_update(int n, double *J, double *const *buf, OsState *st,
                              double *dJ_out, cudaStream_t s);
cudaError_t launch_axpy_rel(int n, double *J, const double *d, OsState *st, cudaStream_t s);
cudaError_t launch_residual(int n, const double *Jfs, const double *J, double *r, OsState *st,
                            cudaStream_t s);
cudaError_t launch_compare(long long n, const double *a, const double *b, OsState *st,
                           cudaStream_t s);
cudaError_t launch_copy_buf(int n, double *const *buf, const OsState *st, double *dst,
                            cudaStream_t s);

// ---- batched wavelengths (batch.cu) ----
constexpr int kBatchSweeps = 50;  // Jacobi sweeps per OS solve (stop test 1e-3)
constexpr int kHist = 11;         // changes kept per wavelength for the error estimate

// Per-wavelength state in device memory (arrays of n_lambda, sweep maxima of
// n_lambda x (kBatchSweeps + 1), change history of n_lambda x kHist).
struct BatchState {
    int *active;   // 1 while iterating
    int *alist;    // [nactive] the active wavelengths in increasing order: the
                   // batched kernels take wavelength alist[blockIdx.y] (.z)
    int *state;    // 0 running, 1 converged, 2 stagnated, 3 NaN, 4 iteration cap
    int *done;     // Jacobi stop test met
    int *count;    // Jacobi sweeps done
    int *iters;    // ALI iterations done
    unsigned long long *dmax, *jmax, *rel;
    double *hist, *est;
    int nactive;   // wavelengths still active (written on the device)
};

struct BatchFsParams {
    int nx, ny, nz, nangles;
    const int *order;
    const long long *toff;
    const int *tlen;
    const signed char *up;
    const float4 *rec32;
    float2 *chiS;          // [n_lambda][4N]
    double *Jrep;          // [n_lambda][4N]
    const double *top_face, *bot_face;  // nullable [n_lambda][ny*nx]
    const double *bot_grad;             // nullable [n_lambda][ny*nx]: diffusion dB/dtau
    const double *mu;                   // [nangles] direction cosines
    double I_top, I_bot;
    BatchState *bs;        // device copy
};

// One batched ALI iteration (source, formal solution, fold and OS right-hand
// side, Jacobi sweeps, update, retirement, active count): a fixed launch
// sequence, captured once into a CUDA graph.
// S of every active wavelength into its packed (chi, S)
cudaError_t launch_b_source(const BatchFsParams &p, int nl, const double *J, const double *eps,
                            const double *B, cudaStream_t s);
// batched FP32 formal solution into p.Jrep in the given shape (one
// characteristic per thread; rays_per_thread is not used)
cudaError_t launch_b_fs(const BatchFsParams &p, int nl, const FsShape &sh, bool parabolic,
                        cudaStream_t s);
// nl: all wavelengths (retirement, compaction); nlaunch >= the active count:
// the wavelength extent of the other launches (blocks past the active count
// return at once)
cudaError_t launch_batch_iteration(const BatchFsParams &p, int nl, int nlaunch, double *J,
                                   const double *eps,
                                   const double *B, const float *a, const double *inv_diag,
                                   double *r, double *buf0, double *buf1, float *b32_0,
                                   float *b32_1, int max_sweeps, double sweep_tol, double tol,
                                   int max_iter, bool parabolic, const FsShape &shape,
                                   cudaStream_t s);

// ---- spherical grid (sph.cu) ----
struct SphTables {
    int nr, nt, np;
    const double *re2;              // [nr+1] squared radial edges
    const double *ct, *ctk;         // [nt+1] cos(theta_e), cos|cos|
    const double *cpe, *spe;        // [np] cos/sin of the azimuth edges
    const double *rc, *stc, *ctc, *cpc, *spc;  // cell centres
};

struct SphBuildParams {
    SphTables T;
    int nangles, o0, nchunk, pass, ncap;
    const double *dir, *wt;
    unsigned *hit;      // [nchunk][(N+31)/32]
    double *tbuf;       // [nchunk][ncap]
    double *den;        // [nchunk][N]
    int *nrays;         // [nangles] (pass 1)
    long long *nseg;    // [nangles] (pass 1)
    const long long *ray_base, *seg_base;  // [nangles] (pass 2)
    long long *ray_off;
    int *ray_len, *ray_angle, *ray_launch, *ray_kind, *ray_face;
    // per segment: record (replicated index of the cell as int bits, FP32 J
    // weight, l/2, the FP32 remainder of the FP64 J weight) and the FP64
    // chord (24 bytes in all)
    float4 *rec;
    double *len64;
    int *err;
};

struct SphFsParams {
    long long nrays;
    int N;
    int nr, nt, np;                // grid (cells decoded from the records' indices)
    const long long *ray_off;
    const int *ray_len, *ray_kind, *ray_face;
    const float4 *rec;             // per segment (replicated index bits, J weight, l/2,
                                   // remainder of the FP64 J weight)
    const double *len64;           // per segment FP64 chord
    const void *chiS;              // replicated packed (chi, S)
    double *J, *lstar;
    const double *core_face;       // nullable [np][nt]
    double I_core, I_out, I_irr;
    int homogeneous;
};

cudaError_t launch_sph_build(const SphBuildParams &p, cudaStream_t s);
cudaError_t launch_sph_fs(const SphFsParams &p, bool fp64, bool parabolic, bool lstar,
                          cudaStream_t s);
// FP32 formal solution without Lambda* over the per-segment records, one ray
// per thread in the builder's order, into the replicated FP64 Jrep (zero on
// entry; fold afterwards)
cudaError_t launch_sph_fs_fast(const SphFsParams &p, double *Jrep, bool parabolic,
                               cudaStream_t s);
// the same in FP64 (the Cartesian FP64 kernel's per-point step)
cudaError_t launch_sph_fs64_fast(const SphFsParams &p, double *Jrep, bool parabolic,
                                 cudaStream_t s);
// the cell (r + nr (t + nt p)) of a replicated index r + 2 nr (t + 2 nt p)
__host__ __device__ inline int sph_cell_of_rep(int rep, int nr, int nt) {
    const int q = rep / (2 * nr), p = q / (2 * nt);
    return (rep - q * 2 * nr) + nr * ((q - p * 2 * nt) + nt * p);
}

// Streaming multiprocessors of the current device (queried once per device
// with cudaDeviceGetAttribute), for launches capped at a multiple of them.
int device_sm_count();

// Sets the message returned by rt3d_last_error() on this thread.
void set_last_error(const char *msg);

// ---- Krylov vector kernels (krylov.cu) ----
cudaError_t launch_multi_dot(int n, const double *const *V, int k, const double *w, double *out,
                             cudaStream_t s);
cudaError_t launch_multi_axpy(int n, double *w, const double *const *V, const double *coef, int k,
                              cudaStream_t s);
cudaError_t launch_scale_copy(int n, const double *src, double alpha, double *dst, cudaStream_t s);
cudaError_t launch_sub(int n, const double *a, const double *b, double *out, cudaStream_t s);

}  // namespace rt3d
