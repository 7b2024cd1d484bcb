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
    uint32_t *code = nullptr;   // [total] step codes
    double *len64 = nullptr;    // [total] chords
    float *len32 = nullptr;
    double *cw64 = nullptr;     // [total] w_Omega l_k / (sum of l over the layer)
    float *cw32 = nullptr;
    uint64_t *win = nullptr;    // [total] Lambda* window: 9 x 5-bit neighbour codes
};

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
    const void *chiS;  // float2 or double2 [N]: (chi, S)
    double *J;         // [N], accumulated into (zeroed by the caller)
    double *lstar;     // nullable [27][N], accumulated into
    const double *top_face;  // nullable [ny*nx]
    const double *bot_face;  // nullable [ny*nx]
    double I_top, I_bot;
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
    double *layer_sum;        // scratch [nangles][nz]
    int *err;                 // out: first error code (0 ok)
};

// Launchers (return the launch status).
cudaError_t launch_trace(const TraceParams &p, cudaStream_t s);
cudaError_t launch_fs(const FsParams &p, bool fp64, bool parabolic, bool lstar, cudaStream_t s);

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
};

cudaError_t launch_pack(int n, const double *chi, double chi_scale, const double *S,
                        void *chiS, bool fp64, cudaStream_t s);
cudaError_t launch_source(int n, const double *J, const double *eps, const double *B,
                          void *chiS, bool fp64, bool homogeneous, cudaStream_t s);
cudaError_t launch_os_prep(int nx, int ny, int nz, const double *lstar, const double *eps,
                           void *a, bool a64, double *inv_diag, cudaStream_t s);
cudaError_t launch_os_init(int n, const double *Jfs, const double *J, const double *rhs_extra,
                           const double *inv_diag, double *r, double *dJ0, OsState *st,
                           cudaStream_t s);
cudaError_t launch_os_sweep(int nx, int ny, int nz, const void *a, bool a64,
                            const double *inv_diag, const double *r, double *const *buf,
                            int m, double tol, OsState *st, cudaStream_t s);
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
