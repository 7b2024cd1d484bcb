// rt3d_os_solve_noalloc: the Jacobi OS solve of rt3d_os_solve (FP64) for
// callers that cannot allocate device memory -- for example a host
// application whose device memory is entirely pre-reserved by its own pool
// allocator, or a code path that must not call cudaMalloc/cudaFree (they
// synchronise the device) in the middle of a time-critical loop. The caller
// passes inputs and outputs; the only scratch (the two sweep buffers and the
// reduction state) lives in file-scope __device__ arrays of a fixed maximum
// size, so this entry point never calls cudaMalloc, cudaFree or any
// allocating library routine, and it needs no rt3d_grid (creating one
// allocates).
//
// Set-up: the first call on a device looks up the device addresses of the
// arrays with cudaGetSymbolAddress (host code cannot use the array names as
// device pointers). Make that first call before any stream capture.
//
// Sharing: every call on a device uses the same arrays, which keep the last
// call's contents; the kernels reset what must start at zero. Calls whose
// work overlaps on the GPU (other streams, other host threads) race on the
// arrays: serialise them.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "rt3d_internal.cuh"

namespace {

constexpr int kMaxDevices = 64;
constexpr int kMaxSweeps = 256;

struct NoallocState {
    unsigned long long dmax[kMaxSweeps + 1];
    unsigned long long jmax[kMaxSweeps + 1];
    int done;
    int count;
};

// 2 x RT3D_NOALLOC_MAX_VOXELS doubles = 1 MiB, held by every GPU that loads
// the library until the process exits.
static __device__ __align__(256) double g_noalloc_buf[2 * RT3D_NOALLOC_MAX_VOXELS];
static __device__ __align__(256) NoallocState g_noalloc_state;

std::mutex g_setup_mutex;
double *g_buf_addr[kMaxDevices] = {};
NoallocState *g_state_addr[kMaxDevices] = {};

__device__ __forceinline__ void na_block_max(double x, unsigned long long *dst) {
    __shared__ unsigned long long sm[32];
    unsigned long long b = (unsigned long long)__double_as_longlong(fabs(x));
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

__device__ __forceinline__ double na_inv_diag(const double *L, const double *eps, long long N,
                                              long long v) {
    return 1.0 / (1.0 - L[13 * N + v] * (1.0 - eps[v]));
}

// dJ^0 = r / diag into buf[0..N); resets the reduction state.
__global__ void na_init(int N, const double *L, const double *eps, const double *r, double *buf,
                        NoallocState *st) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        st->done = 0;
        st->count = 0;
    }
    if (tid <= kMaxSweeps) {
        st->dmax[tid] = 0ULL;
        st->jmax[tid] = 0ULL;
    }
    for (int v = tid; v < N; v += gridDim.x * blockDim.x) buf[v] = r[v] * na_inv_diag(L, eps, N, v);
}

// Sweep m: buf[(m&1) N ..] from buf[((m-1)&1) N ..], with the stop test of
// rt3d_os_solve on the previous sweep's maxima.
__global__ void __launch_bounds__(256) na_sweep(int nx, int ny, int nz, const double *__restrict__ L,
                                                const double *__restrict__ eps,
                                                const double *__restrict__ r, double *buf, int m,
                                                double tol, NoallocState *st) {
    if (st->done) return;
    if (m >= 2) {
        const double dm = __longlong_as_double((long long)st->dmax[m - 1]);
        const double jm = __longlong_as_double((long long)st->jmax[m - 1]);
        if (dm <= tol * jm) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                st->done = 1;
                st->count = m - 1;
            }
            return;
        }
    }
    const int N = nx * ny * nz;
    const double *src = buf + (long long)((m - 1) & 1) * N;
    double *dst = buf + (long long)(m & 1) * N;
    double dmax = 0.0, jmax = 0.0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
        const int x = v % nx, y = (v / nx) % ny, z = v / (nx * ny);
        const int xs[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};
        const int ys[3] = {y == 0 ? ny - 1 : y - 1, y, y == ny - 1 ? 0 : y + 1};
        double acc = 0.0;
#pragma unroll
        for (int d = 0; d < 27; ++d) {
            if (d == 13) continue;
            const int zz = z + d / 9 - 1;
            if (zz < 0 || zz >= nz) continue;
            const int u = xs[d % 3] + nx * (ys[(d / 3) % 3] + ny * zz);
            const double coef = L[(long long)d * N + v] * (1.0 - eps[u]);
            acc = fma(coef, src[u], acc);
        }
        const double nv = (r[v] + acc) * na_inv_diag(L, eps, N, v);
        dst[v] = nv;
        dmax = fmax(dmax, fabs(nv - src[v]));
        jmax = fmax(jmax, fabs(nv));
    }
    na_block_max(dmax, &st->dmax[m]);
    na_block_max(jmax, &st->jmax[m]);
}

// The cap was reached if the stop test never fired.
__global__ void na_mark(int max_sweeps, NoallocState *st) {
    if (!st->done) {
        st->done = 1;
        st->count = max_sweeps;
    }
}

// Copies the final sweep buffer (count fixed by na_mark, earlier in stream
// order) to the caller's output.
__global__ void na_finish(int N, const double *buf, double *out, const NoallocState *st) {
    const double *src = buf + (long long)(st->count & 1) * N;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x)
        out[v] = src[v];
}

rt3d_status na_fail(rt3d_status s, const char *fmt, ...) {
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    rt3d::set_last_error(msg);  // reported by rt3d_last_error()
    return s;
}

// Whether p is memory the kernels can use on device dev: device memory of
// dev itself, or managed memory. Device memory of another device is
// rejected (without peer access a kernel on dev cannot read it).
bool na_is_device(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == dev);
}

}  // namespace

extern "C" rt3d_status rt3d_os_solve_noalloc(int nx, int ny, int nz, const double *lstar,
                                             const double *eps, const double *r, double *dJ_out,
                                             int max_sweeps, double tol, int *sweeps_out,
                                             void *cuda_stream) {
    if (!lstar || !eps || !r || !dJ_out) return na_fail(RT3D_EINVAL, "NULL argument");
    if (nx < 4 || ny < 4 || nz < 1)
        return na_fail(RT3D_EINVAL, "grid %d x %d x %d: need nx, ny >= 4, nz >= 1", nx, ny, nz);
    const long long N = (long long)nx * ny * nz;
    if (N > RT3D_NOALLOC_MAX_VOXELS)
        return na_fail(RT3D_EINVAL, "%lld voxels exceed the allocation-free limit of %d", N,
                       (int)RT3D_NOALLOC_MAX_VOXELS);
    if (max_sweeps < 1 || max_sweeps > kMaxSweeps)
        return na_fail(RT3D_EINVAL, "max_sweeps %d outside 1..%d", max_sweeps, kMaxSweeps);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(RT3D_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return na_fail(RT3D_EINVAL, "device %d out of range", dev);
    if (!na_is_device(lstar, dev) || !na_is_device(eps, dev) || !na_is_device(r, dev) ||
        !na_is_device(dJ_out, dev))
        return na_fail(RT3D_EINVAL, "all arrays must be device memory of the current device %d",
                       dev);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return na_fail(RT3D_ECUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(e));
    if (cap != cudaStreamCaptureStatusNone)
        return na_fail(RT3D_EINVAL, "the stream is being captured: this call synchronises its "
                                    "stream and cannot be captured");
    double *buf = nullptr;
    NoallocState *st = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_buf_addr[dev]) {
            void *pb = nullptr, *ps = nullptr;
            e = cudaGetSymbolAddress(&pb, g_noalloc_buf);
            if (e != cudaSuccess)
                return na_fail(RT3D_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            e = cudaGetSymbolAddress(&ps, g_noalloc_state);
            if (e != cudaSuccess)
                return na_fail(RT3D_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_buf_addr[dev] = static_cast<double *>(pb);
            g_state_addr[dev] = static_cast<NoallocState *>(ps);
        }
        buf = g_buf_addr[dev];
        st = g_state_addr[dev];
    }
    const int n = (int)N;
    int blocks = (n + 255) / 256;
    if (blocks < 2) blocks = 2;  // >= 257 threads reset the maxima
    na_init<<<blocks, 256, 0, s>>>(n, lstar, eps, r, buf, st);
    const int sb = (n + 255) / 256;
    for (int m = 1; m <= max_sweeps; ++m)
        na_sweep<<<sb, 256, 0, s>>>(nx, ny, nz, lstar, eps, r, buf, m, tol, st);
    na_mark<<<1, 1, 0, s>>>(max_sweeps, st);
    na_finish<<<sb, 256, 0, s>>>(n, buf, dJ_out, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(RT3D_ECUDA, "launch: %s", cudaGetErrorString(e));
    int cnt = 0;
    e = cudaMemcpyAsync(&cnt, &st->count, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return na_fail(RT3D_ECUDA, "%s", cudaGetErrorString(e));
    if (sweeps_out) *sweeps_out = cnt;
    return RT3D_OK;
}
