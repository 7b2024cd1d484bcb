// C ABI of include/rt3d.h: grid lifetime, the geometry cache, argument
// staging, and the host side of the formal solution, OS solve, ALI step and
// the mixed-precision solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "rt3d_internal.cuh"

using namespace rt3d;

namespace {

thread_local std::string g_err;

rt3d_status fail(rt3d_status st, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
rt3d_status fail(rt3d_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(e_ == cudaErrorMemoryAllocation ? RT3D_ENOMEM : RT3D_ECUDA,     \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                      \
    } while (0)

#define CKL(call)  \
    do {            \
        CK(call);   \
        ++g->launches; \
    } while (0)

#define TRY(expr)                              \
    do {                                       \
        rt3d_status s_ = (expr);               \
        if (s_ != RT3D_OK) return s_;          \
    } while (0)

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

struct rt3d_grid {
    rt3d_grid_desc desc{};
    int nx = 0, ny = 0, nz = 0, nO = 0;
    long long N = 0;
    cudaStream_t stream = nullptr;
    bool fs64 = true;     // formal solution precision
    bool parab = false;
    long long segments = 0;
    long long dev_bytes = 0;
    std::vector<double> mu, wt, dir;
    std::vector<int> K;
    std::vector<void *> allocs;
    Template tpl;

    // work buffers
    double *chi = nullptr, *eps = nullptr, *B = nullptr, *S = nullptr, *J = nullptr;
    double *Jfs = nullptr, *r = nullptr, *dJ[2] = {nullptr, nullptr}, *inv_diag = nullptr;
    double *lstar = nullptr;  // [27][N] FP64 accumulation
    double *top = nullptr, *bot = nullptr, *tmp = nullptr, *delta = nullptr, *r64 = nullptr;
    double *chi_ref = nullptr, *eps_ref = nullptr;
    double **dJ_dev = nullptr;  // device copy of {dJ[0], dJ[1]}
    void *chiS32 = nullptr, *chiS64 = nullptr;
    void *a = nullptr;  // [26][N] OS off-diagonals (f64 in FP64 mode, f32 otherwise)
    bool a64 = true;
    OsState *st = nullptr;
    bool lstar_valid = false;

    // Krylov workspace (allocated on first use): basis V[0..m], preconditioned
    // directions Z[0..m-1], their device pointer arrays, small scalars
    static constexpr int kKrylov = 100;
    bool krylov_ready = false;
    double *V[kKrylov + 1] = {}, *Z[kKrylov] = {};
    double **dV = nullptr, **dZ = nullptr, **dOne = nullptr;
    double *dots = nullptr, *coef = nullptr;

    // instrumentation: formal-solution kernel time (CUDA events on the
    // grid's stream) and kernels launched
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int ev_pending = -1;  // -1 none, 0 FP32, 1 FP64
    double fs_ms[2] = {0.0, 0.0};
    long long launches = 0;

    template <typename T>
    rt3d_status alloc(T **p, size_t count) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(RT3D_ENOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                        cudaGetErrorString(e));
        }
        allocs.push_back(q);
        dev_bytes += (long long)(count * sizeof(T));
        *p = static_cast<T *>(q);
        return RT3D_OK;
    }
    ~rt3d_grid() {
        for (void *p : allocs) cudaFree(p);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
    }
};

namespace {

// Input: a device pointer as is, or a host array copied into `stage`.
rt3d_status stage_in(rt3d_grid *g, const double *p, size_t n, double *stage, const double **out) {
    if (!p) {
        *out = nullptr;
        return RT3D_OK;
    }
    if (is_device_ptr(p)) {
        *out = p;
        return RT3D_OK;
    }
    CK(cudaMemcpyAsync(stage, p, n * sizeof(double), cudaMemcpyHostToDevice, g->stream));
    *out = stage;
    return RT3D_OK;
}

rt3d_status fs_params(rt3d_grid *g, const rt3d_bc *bc, bool fp64, bool homogeneous,
                      FsParams *p) {
    FsParams q{};
    q.nx = g->nx;
    q.ny = g->ny;
    q.nz = g->nz;
    q.nangles = g->nO;
    q.order = g->tpl.order;
    q.toff = g->tpl.toff;
    q.tlen = g->tpl.tlen;
    q.up = g->tpl.up;
    q.code = g->tpl.code;
    q.len = fp64 ? (const void *)g->tpl.len64 : (const void *)g->tpl.len32;
    q.cw = fp64 ? (const void *)g->tpl.cw64 : (const void *)g->tpl.cw32;
    q.win = g->tpl.win;
    q.chiS = fp64 ? g->chiS64 : g->chiS32;
    q.homogeneous = homogeneous ? 1 : 0;
    if (bc && !homogeneous) {
        q.I_top = bc->I_top;
        q.I_bot = bc->I_bottom;
        const double *tf = nullptr, *bf = nullptr;
        const size_t nf = (size_t)g->nx * g->ny;
        TRY(stage_in(g, bc->I_top_face, nf, g->top, &tf));
        TRY(stage_in(g, bc->I_bottom_face, nf, g->bot, &bf));
        q.top_face = tf;
        q.bot_face = bf;
    }
    *p = q;
    return RT3D_OK;
}

// Adds the time of the last timed formal solution (waits for it).
rt3d_status collect_events(rt3d_grid *g) {
    if (g->ev_pending < 0) return RT3D_OK;
    CK(cudaEventSynchronize(g->ev1));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    g->fs_ms[g->ev_pending] += ms;
    g->ev_pending = -1;
    return RT3D_OK;
}

// One formal solution of the packed (chi, S) of the given precision into
// g->Jfs (zeroed here); Lambda* into g->lstar when requested.
rt3d_status run_fs(rt3d_grid *g, const FsParams &base, bool fp64, bool with_lstar) {
    FsParams p = base;
    p.chiS = fp64 ? g->chiS64 : g->chiS32;
    p.len = fp64 ? (const void *)g->tpl.len64 : (const void *)g->tpl.len32;
    p.cw = fp64 ? (const void *)g->tpl.cw64 : (const void *)g->tpl.cw32;
    p.J = g->Jfs;
    p.lstar = with_lstar ? g->lstar : nullptr;
    CK(cudaMemsetAsync(g->Jfs, 0, sizeof(double) * g->N, g->stream));
    if (with_lstar) CK(cudaMemsetAsync(g->lstar, 0, sizeof(double) * 27 * g->N, g->stream));
    TRY(collect_events(g));
    CK(cudaEventRecord(g->ev0, g->stream));
    CK(launch_fs(p, fp64, g->parab, with_lstar, g->stream));
    CK(cudaEventRecord(g->ev1, g->stream));
    g->ev_pending = fp64 ? 1 : 0;
    ++g->launches;
    return RT3D_OK;
}

rt3d_status reset_scalar(rt3d_grid *g, size_t off, size_t sz) {
    CK(cudaMemsetAsync(reinterpret_cast<char *>(g->st) + off, 0, sz, g->stream));
    return RT3D_OK;
}

rt3d_status read_scalar_d(rt3d_grid *g, size_t off, double *out) {
    unsigned long long b = 0;
    CK(cudaMemcpyAsync(&b, reinterpret_cast<char *>(g->st) + off, sizeof b, cudaMemcpyDeviceToHost,
                       g->stream));
    CK(cudaStreamSynchronize(g->stream));
    TRY(collect_events(g));
    double d;
    std::memcpy(&d, &b, sizeof d);
    *out = d;
    return RT3D_OK;
}

// Jacobi solve of [1 - L*(1-eps)] dJ = r with r = Jfs - J (+extra) (or
// r = extra when Jfs, J are null), folded coefficients already prepared.
// Leaves the result in g->dJ[count & 1]; the count stays on the device.
rt3d_status os_solve_dev(rt3d_grid *g, const double *Jfs, const double *J, const double *extra,
                         int max_sweeps, double tol) {
    CK(launch_os_init((int)g->N, Jfs, J, extra, g->inv_diag, g->r, g->dJ[0], g->st, g->stream));
    for (int m = 1; m <= max_sweeps; ++m)
        CK(launch_os_sweep(g->nx, g->ny, g->nz, g->a, g->a64, g->inv_diag, g->r, g->dJ, m, tol,
                           g->st, g->stream));
    CK(launch_os_finish(max_sweeps, tol, g->st, g->stream));
    g->launches += max_sweeps + 2;
    return RT3D_OK;
}

rt3d_status validate_desc(const rt3d_grid_desc *d) {
    if (!d) return fail(RT3D_EINVAL, "desc is NULL");
    if (d->geometry != RT3D_CARTESIAN_PERIODIC_XY)
        return fail(RT3D_EINVAL, "geometry %d is not supported", d->geometry);
    if (d->n[0] < 4 || d->n[0] > 2047 || d->n[1] < 4 || d->n[1] > 2047 || d->n[2] < 1 ||
        d->n[2] > 1023)
        return fail(RT3D_EINVAL, "grid %d x %d x %d outside 4..2047 x 4..2047 x 1..1023",
                    d->n[0], d->n[1], d->n[2]);
    if (d->ntheta < 1 || d->nphi < 1 || (long long)d->ntheta * d->nphi > 65535)
        return fail(RT3D_EINVAL, "bad angle grid %d x %d", d->ntheta, d->nphi);
    if (d->interp != RT3D_LINEAR && d->interp != RT3D_PARABOLIC)
        return fail(RT3D_EINVAL, "bad interp %d", d->interp);
    if (d->precision != RT3D_FP64 && d->precision != RT3D_FP32_FS_FP64_ALI)
        return fail(RT3D_EINVAL, "bad precision %d", d->precision);
    if (d->nlambda > 1) return fail(RT3D_EINVAL, "nlambda > 1 is not supported by this call");
    if (d->accel != RT3D_ACCEL_NONE && d->accel != RT3D_ACCEL_KRYLOV)
        return fail(RT3D_EINVAL, "bad accel %d", d->accel);
    return RT3D_OK;
}

rt3d_status grid_build(rt3d_grid *g) {
    const rt3d_grid_desc &d = g->desc;
    g->nx = d.n[0];
    g->ny = d.n[1];
    g->nz = d.n[2];
    g->N = (long long)g->nx * g->ny * g->nz;
    g->nO = d.ntheta * d.nphi;
    g->stream = static_cast<cudaStream_t>(d.cuda_stream);
    g->fs64 = d.precision == RT3D_FP64;
    g->parab = d.interp == RT3D_PARABOLIC;
    g->a64 = g->fs64;

    // A1: direction set in FP64 on the host (midpoints in mu and phi).
    const int nO = g->nO;
    g->mu.resize(nO);
    g->wt.resize(nO);
    g->dir.resize(3 * nO);
    for (int i = 0; i < d.ntheta; ++i) {
        for (int j = 0; j < d.nphi; ++j) {
            const int o = i * d.nphi + j;
            const double m = -1.0 + (double)(2 * i + 1) / (double)d.ntheta;
            const double ph = (double)(2 * j + 1) * M_PI / (double)d.nphi;
            const double st = std::sqrt((1.0 - m) * (1.0 + m));
            g->mu[o] = m;
            g->wt[o] = 1.0 / (double)nO;
            g->dir[3 * o + 0] = st * std::cos(ph);
            g->dir[3 * o + 1] = st * std::sin(ph);
            g->dir[3 * o + 2] = m;
            if (!(std::fabs(m) > 0.0)) return fail(RT3D_EINVAL, "direction %d has mu = 0", o);
        }
    }
    // Capacity per angle: nz z-steps plus at most |d_x| nz/|mu| + 1 x-steps and
    // likewise in y.
    std::vector<int> cap(nO);
    std::vector<long long> off(nO);
    long long total = 0;
    for (int o = 0; o < nO; ++o) {
        const double span = (double)g->nz / std::fabs(g->dir[3 * o + 2]);
        const double c = g->nz + std::fabs(g->dir[3 * o]) * span + std::fabs(g->dir[3 * o + 1]) * span + 8;
        if (c > 2.0e9) return fail(RT3D_EINVAL, "characteristic of angle %d too long", o);
        cap[o] = (int)c;
        off[o] = total;
        total += cap[o];
    }
    Template &t = g->tpl;
    t.nangles = nO;
    t.total = total;
    TRY(g->alloc(&t.tlen, nO));
    TRY(g->alloc(&t.toff, nO));
    TRY(g->alloc(&t.order, nO));
    TRY(g->alloc(&t.up, nO));
    TRY(g->alloc(&t.code, total));
    TRY(g->alloc(&t.len64, total));
    TRY(g->alloc(&t.len32, total));
    TRY(g->alloc(&t.cw64, total));
    TRY(g->alloc(&t.cw32, total));
    TRY(g->alloc(&t.win, total));
    double *d_dir = nullptr, *d_wt = nullptr, *d_ls = nullptr;
    int *d_cap = nullptr, *d_err = nullptr;
    TRY(g->alloc(&d_dir, 3 * nO));
    TRY(g->alloc(&d_wt, nO));
    TRY(g->alloc(&d_ls, (size_t)nO * g->nz));
    TRY(g->alloc(&d_cap, nO));
    TRY(g->alloc(&d_err, 1));
    cudaStream_t s = g->stream;
    std::vector<signed char> up(nO);
    for (int o = 0; o < nO; ++o) up[o] = g->mu[o] > 0.0 ? 1 : 0;
    CK(cudaMemcpyAsync(d_dir, g->dir.data(), sizeof(double) * 3 * nO, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_wt, g->wt.data(), sizeof(double) * nO, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_cap, cap.data(), sizeof(int) * nO, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(t.toff, off.data(), sizeof(long long) * nO, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(t.up, up.data(), nO, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(d_err, 0, sizeof(int), s));
    TraceParams tp{};
    tp.nx = g->nx;
    tp.ny = g->ny;
    tp.nz = g->nz;
    tp.nangles = nO;
    tp.dir = d_dir;
    tp.wt = d_wt;
    tp.toff = t.toff;
    tp.cap = d_cap;
    tp.tlen = t.tlen;
    tp.code = t.code;
    tp.len64 = t.len64;
    tp.len32 = t.len32;
    tp.cw64 = t.cw64;
    tp.cw32 = t.cw32;
    tp.win = t.win;
    tp.layer_sum = d_ls;
    tp.err = d_err;
    CK(launch_trace(tp, s));
    int herr = 0;
    g->K.resize(nO);
    CK(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(g->K.data(), t.tlen, sizeof(int) * nO, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (herr == 1) return fail(RT3D_EINVAL, "a direction has no z component");
    if (herr == 2) return fail(RT3D_EINVAL, "a characteristic exceeded its capacity");
    if (herr == 3) return fail(RT3D_EINVAL, "a Lambda* window exceeds 9 points (box too small)");
    if (herr) return fail(RT3D_EINVAL, "tracer error %d", herr);
    std::vector<int> order(nO);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return g->K[a] > g->K[b]; });
    CK(cudaMemcpyAsync(t.order, order.data(), sizeof(int) * nO, cudaMemcpyHostToDevice, s));
    t.kmax = *std::max_element(g->K.begin(), g->K.end());
    g->segments = 0;
    for (int o = 0; o < nO; ++o) g->segments += (long long)g->K[o] * g->nx * g->ny;

    // work buffers
    const size_t N = (size_t)g->N, nf = (size_t)g->nx * g->ny;
    TRY(g->alloc(&g->chi, N));
    TRY(g->alloc(&g->eps, N));
    TRY(g->alloc(&g->B, N));
    TRY(g->alloc(&g->S, N));
    TRY(g->alloc(&g->J, N));
    TRY(g->alloc(&g->Jfs, N));
    TRY(g->alloc(&g->r, N));
    TRY(g->alloc(&g->dJ[0], N));
    TRY(g->alloc(&g->dJ[1], N));
    TRY(g->alloc(&g->inv_diag, N));
    TRY(g->alloc(&g->tmp, N));
    TRY(g->alloc(&g->delta, N));
    TRY(g->alloc(&g->r64, N));
    TRY(g->alloc(&g->chi_ref, N));
    TRY(g->alloc(&g->eps_ref, N));
    TRY(g->alloc(&g->lstar, 27 * N));
    TRY(g->alloc(&g->top, nf));
    TRY(g->alloc(&g->bot, nf));
    TRY(g->alloc(&g->dJ_dev, 2));
    TRY(g->alloc(reinterpret_cast<double2 **>(&g->chiS64), N));
    TRY(g->alloc(reinterpret_cast<float2 **>(&g->chiS32), N));
    if (g->a64) TRY(g->alloc(reinterpret_cast<double **>(&g->a), 26 * N));
    else TRY(g->alloc(reinterpret_cast<float **>(&g->a), 26 * N));
    TRY(g->alloc(&g->st, 1));
    CK(cudaMemcpyAsync(g->dJ_dev, g->dJ, sizeof(double *) * 2, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(g->st, 0, sizeof(OsState), s));
    CK(cudaEventCreate(&g->ev0));
    CK(cudaEventCreate(&g->ev1));
    CK(cudaStreamSynchronize(s));
    return RT3D_OK;
}

// Convergence monitor of an iteration from its max relative changes:
// contraction rho from the last `kWindow` changes, error estimate
// rel * rho / (1 - rho), stagnation when the window shows no decrease.
struct Progress {
    static constexpr int kWindow = 10;
    std::vector<double> h;
    void add(double r) { h.push_back(r); }
    double rho() const {
        const int n = (int)h.size();
        if (n < 2) return 0.9;
        const int m = std::min(n - 1, kWindow);
        const double a = h[n - 1 - m], b = h[n - 1];
        if (!(a > 0.0) || !(b > 0.0)) return 0.0;
        return std::min(std::pow(b / a, 1.0 / m), 0.999);
    }
    double error_estimate() const {
        if (h.empty()) return 1.0;
        const double r = rho();
        return h.back() * r / (1.0 - r);
    }
    // no decrease over two windows: the changes sit at the rounding floor
    bool stagnated() const {
        const int n = (int)h.size();
        if (n < 2 * kWindow + 1) return false;
        return h[n - 1] > 0.7 * h[n - 1 - 2 * kWindow] && h.back() < 1e-2;
    }
};

// Copies a device result to a caller array (device or host).
rt3d_status deliver(rt3d_grid *g, double *dst, const double *src, size_t n) {
    if (!dst || dst == src) return RT3D_OK;
    CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, g->stream));
    return RT3D_OK;
}

// Loads chi, eps, B (device or host) into the grid; rebuilds Lambda* lazily
// when chi or eps differ from the last build.
rt3d_status load_problem(rt3d_grid *g, const double *chi, const double *eps, const double *B) {
    const size_t N = (size_t)g->N;
    CK(cudaMemcpyAsync(g->chi, chi, N * sizeof(double), cudaMemcpyDefault, g->stream));
    CK(cudaMemcpyAsync(g->eps, eps, N * sizeof(double), cudaMemcpyDefault, g->stream));
    if (B) CK(cudaMemcpyAsync(g->B, B, N * sizeof(double), cudaMemcpyDefault, g->stream));
    if (g->lstar_valid) {
        CK(cudaMemsetAsync(&g->st->changed, 0, sizeof(int), g->stream));
        CKL(launch_compare((long long)N, g->chi, g->chi_ref, g->st, g->stream));
        CKL(launch_compare((long long)N, g->eps, g->eps_ref, g->st, g->stream));
        int changed = 0;
        CK(cudaMemcpyAsync(&changed, &g->st->changed, sizeof(int), cudaMemcpyDeviceToHost,
                           g->stream));
        CK(cudaStreamSynchronize(g->stream));
        if (changed) g->lstar_valid = false;
    }
    CKL(launch_pack((int)N, g->chi, 1.0, g->chi /*S placeholder*/, g->chiS32, false, g->stream));
    CKL(launch_pack((int)N, g->chi, 1.0, g->chi, g->chiS64, true, g->stream));
    return RT3D_OK;
}

// One ALI iteration on the grid's state (g->J): S from J, FS of the grid's
// FS precision (fp64 flag), Lambda* if not valid, Jacobi, J += dJ.
rt3d_status ali_iteration(rt3d_grid *g, const FsParams &fp, bool fp64, int max_sweeps,
                          double sweep_tol, double *rel) {
    const int N = (int)g->N;
    CKL(launch_source(N, g->J, g->eps, g->B, fp64 ? g->chiS64 : g->chiS32, fp64, false, g->stream));
    const bool build = !g->lstar_valid;
    TRY(run_fs(g, fp, fp64, build));
    if (build) {
        CKL(launch_os_prep(g->nx, g->ny, g->nz, g->lstar, g->eps, g->a, g->a64, g->inv_diag,
                          g->stream));
        CK(cudaMemcpyAsync(g->chi_ref, g->chi, sizeof(double) * N, cudaMemcpyDeviceToDevice,
                           g->stream));
        CK(cudaMemcpyAsync(g->eps_ref, g->eps, sizeof(double) * N, cudaMemcpyDeviceToDevice,
                           g->stream));
        g->lstar_valid = true;
    }
    TRY(os_solve_dev(g, g->Jfs, g->J, nullptr, max_sweeps, sweep_tol));
    TRY(reset_scalar(g, offsetof(OsState, rel), sizeof(unsigned long long)));
    CKL(launch_ali_update(N, g->J, g->dJ_dev, g->st, nullptr, g->stream));
    TRY(read_scalar_d(g, offsetof(OsState, rel), rel));
    return RT3D_OK;
}

rt3d_status krylov_setup(rt3d_grid *g) {
    if (g->krylov_ready) return RT3D_OK;
    const size_t N = (size_t)g->N;
    const int m = rt3d_grid::kKrylov;
    for (int i = 0; i <= m; ++i) TRY(g->alloc(&g->V[i], N));
    for (int i = 0; i < m; ++i) TRY(g->alloc(&g->Z[i], N));
    TRY(g->alloc(&g->dV, m + 1));
    TRY(g->alloc(&g->dZ, m));
    TRY(g->alloc(&g->dOne, 1));
    TRY(g->alloc(&g->dots, m + 1));
    TRY(g->alloc(&g->coef, m + 1));
    CK(cudaMemcpyAsync(g->dV, g->V, sizeof(double *) * (m + 1), cudaMemcpyHostToDevice, g->stream));
    CK(cudaMemcpyAsync(g->dZ, g->Z, sizeof(double *) * m, cudaMemcpyHostToDevice, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    g->krylov_ready = true;
    return RT3D_OK;
}

// <V[i], w> for i < k (V = g->dV) into host out[k]
rt3d_status kdots(rt3d_grid *g, double *const *Vdev, int k, const double *w, double *out) {
    CK(cudaMemsetAsync(g->dots, 0, sizeof(double) * k, g->stream));
    CKL(launch_multi_dot((int)g->N, Vdev, k, w, g->dots, g->stream));
    CK(cudaMemcpyAsync(out, g->dots, sizeof(double) * k, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return RT3D_OK;
}

rt3d_status knorm(rt3d_grid *g, const double *w, double *out) {
    CK(cudaMemcpyAsync(g->dOne, &w, sizeof(double *), cudaMemcpyHostToDevice, g->stream));
    double d = 0.0;
    TRY(kdots(g, g->dOne, 1, w, &d));
    *out = std::sqrt(std::max(d, 0.0));
    return RT3D_OK;
}

// w -= sum_i c[i] Vdev[i]
rt3d_status kaxpy(rt3d_grid *g, double *w, double *const *Vdev, const double *c, int k) {
    CK(cudaMemcpyAsync(g->coef, c, sizeof(double) * k, cudaMemcpyHostToDevice, g->stream));
    CKL(launch_multi_axpy((int)g->N, w, Vdev, g->coef, k, g->stream));
    CK(cudaStreamSynchronize(g->stream));  // c is host memory owned by the caller
    return RT3D_OK;
}

// out = A v = v - Lambda_hom((1 - eps) v), formal solution in FP32 or FP64
rt3d_status apply_A(rt3d_grid *g, const FsParams &fphom, bool fp64, const double *v, double *out) {
    const int n = (int)g->N;
    CKL(launch_source(n, v, g->eps, nullptr, fp64 ? g->chiS64 : g->chiS32, fp64, true, g->stream));
    TRY(run_fs(g, fphom, fp64, false));
    CKL(launch_sub(n, v, g->Jfs, out, g->stream));
    return RT3D_OK;
}

// z = M^-1 v by Jacobi sweeps (the OS solve of Eq. alo)
rt3d_status precond(rt3d_grid *g, const double *v, double *z) {
    TRY(os_solve_dev(g, nullptr, nullptr, v, 50, 1e-3));
    CKL(launch_copy_buf((int)g->N, g->dJ_dev, g->st, z, g->stream));
    return RT3D_OK;
}

// One FGMRES cycle (right preconditioning, classical Gram-Schmidt applied
// twice) for A x = r from x = 0. Stops when the residual estimate falls to
// eta |r| or after kKrylov steps. Returns the achieved reduction and the
// number of operator applications.
rt3d_status fgmres(rt3d_grid *g, const FsParams &fphom, bool fp64, const double *r, double *x,
                   double eta, int max_steps, double *achieved, int *steps) {
    const int n = (int)g->N;
    const int m = std::min(rt3d_grid::kKrylov, std::max(1, max_steps));
    TRY(krylov_setup(g));
    double beta = 0.0;
    TRY(knorm(g, r, &beta));
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, g->stream));
    *steps = 0;
    *achieved = 0.0;
    if (!(beta > 0.0)) return RT3D_OK;
    if (!std::isfinite(beta)) return fail(RT3D_ENUMERIC, "non-finite residual norm");
    CKL(launch_scale_copy(n, r, 1.0 / beta, g->V[0], g->stream));
    std::vector<double> H((m + 1) * m, 0.0), cs(m, 0.0), sn(m, 0.0), gv(m + 1, 0.0), h(m + 1),
        h2(m + 1);
    gv[0] = beta;
    int k = 0;
    for (int j = 0; j < m; ++j) {
        TRY(precond(g, g->V[j], g->Z[j]));
        TRY(apply_A(g, fphom, fp64, g->Z[j], g->V[j + 1]));
        TRY(kdots(g, g->dV, j + 1, g->V[j + 1], h.data()));
        TRY(kaxpy(g, g->V[j + 1], g->dV, h.data(), j + 1));
        TRY(kdots(g, g->dV, j + 1, g->V[j + 1], h2.data()));
        TRY(kaxpy(g, g->V[j + 1], g->dV, h2.data(), j + 1));
        for (int i = 0; i <= j; ++i) h[i] += h2[i];
        double hn = 0.0;
        TRY(knorm(g, g->V[j + 1], &hn));
        if (!std::isfinite(hn)) return fail(RT3D_ENUMERIC, "non-finite Krylov vector");
        if (hn > 0.0) CKL(launch_scale_copy(n, g->V[j + 1], 1.0 / hn, g->V[j + 1], g->stream));
        // Givens rotations on column j
        for (int i = 0; i < j; ++i) {
            const double a = h[i], b = h[i + 1];
            h[i] = cs[i] * a + sn[i] * b;
            h[i + 1] = -sn[i] * a + cs[i] * b;
        }
        const double a = h[j], b = hn;
        const double den = std::hypot(a, b);
        cs[j] = den > 0.0 ? a / den : 1.0;
        sn[j] = den > 0.0 ? b / den : 0.0;
        h[j] = den;
        gv[j + 1] = -sn[j] * gv[j];
        gv[j] = cs[j] * gv[j];
        for (int i = 0; i <= j; ++i) H[i * m + j] = h[i];
        k = j + 1;
        if (std::fabs(gv[j + 1]) <= eta * beta || !(hn > 0.0)) break;
    }
    // back substitution H y = g, then x = sum y_i Z_i
    std::vector<double> y(k, 0.0);
    for (int i = k - 1; i >= 0; --i) {
        double t = gv[i];
        for (int l = i + 1; l < k; ++l) t -= H[i * m + l] * y[l];
        y[i] = H[i * m + i] != 0.0 ? t / H[i * m + i] : 0.0;
    }
    for (int i = 0; i < k; ++i) y[i] = -y[i];
    TRY(kaxpy(g, x, g->dZ, y.data(), k));
    *achieved = std::fabs(gv[k]) / beta;
    *steps = k;
    return RT3D_OK;
}

// Krylov-accelerated solve with FP64 iterative refinement. Rounds: residual
// r = J_FS(S(J)) - J (FP32 before the first converged cycle in the mixed
// mode, FP64 afterwards), FGMRES cycle on A delta = r (A in the grid's FS
// precision), J += delta. The error after a round is estimated as
// gain * (next FP64 residual), gain = |delta|/|r| of the previous round;
// the FP64 residual that meets tol is the certification.
rt3d_status krylov_solve(rt3d_grid *g, const FsParams &fp, const FsParams &fp64p,
                         const FsParams &fphom, double tol, int max_iter, rt3d_solve_stats &s,
                         bool *conv_out) {
    const int n = (int)g->N;
    const bool mixed = !g->fs64;
    bool res64 = !mixed;
    bool conv = false;
    double gain = -1.0, est = 1.0, res = 0.0;
    int it = 0, rounds32 = 0;
    // Reduction asked of one FGMRES cycle: with an FP32 operator the basis
    // carries rounding noise, so cycles stop at 1e-3 and the FP64 residual
    // of the next round drives the refinement.
    const double eta = mixed ? 1e-3 : 1e-4;
    for (int round = 0; round < 60 && it < max_iter; ++round) {
        // residual of the current J (the first one also builds Lambda*)
        const bool fs64 = res64;
        const bool build = !g->lstar_valid;
        CKL(launch_source(n, g->J, g->eps, g->B, fs64 ? g->chiS64 : g->chiS32, fs64, false,
                          g->stream));
        TRY(run_fs(g, fs64 ? fp64p : fp, fs64, build));
        if (fs64) ++s.fs_fp64;
        else ++s.fs_fp32;
        if (build) {
            CKL(launch_os_prep(g->nx, g->ny, g->nz, g->lstar, g->eps, g->a, g->a64, g->inv_diag,
                               g->stream));
            CK(cudaMemcpyAsync(g->chi_ref, g->chi, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                               g->stream));
            CK(cudaMemcpyAsync(g->eps_ref, g->eps, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                               g->stream));
            g->lstar_valid = true;
        }
        TRY(reset_scalar(g, offsetof(OsState, res), sizeof(unsigned long long)));
        CKL(launch_residual(n, g->Jfs, g->J, g->r64, g->st, g->stream));
        TRY(read_scalar_d(g, offsetof(OsState, res), &res));
        if (!(res == res)) return fail(RT3D_ENUMERIC, "NaN in the residual");
        if (fs64) s.residual64 = res;
        // gain < 0: unknown (first round, or a residual relative to J = 0)
        if (fs64 && gain >= 0.0) {
            est = gain * res;
            if (est <= tol) {
                conv = true;
                break;
            }
        }
        double achieved = 0.0;
        int steps = 0;
        TRY(fgmres(g, fphom, g->fs64, g->r64, g->delta, eta, max_iter - it, &achieved, &steps));
        it += steps;
        if (g->fs64) s.fs_fp64 += steps;
        else s.fs_fp32 += steps;
        TRY(reset_scalar(g, offsetof(OsState, rel), sizeof(unsigned long long)));
        CKL(launch_axpy_rel(n, g->J, g->delta, g->st, g->stream));
        double crel = 0.0;
        TRY(read_scalar_d(g, offsetof(OsState, rel), &crel));
        if (!(crel == crel)) return fail(RT3D_ENUMERIC, "NaN in the Krylov correction");
        s.rel_change = crel;
        gain = (res > 0.0 && std::isfinite(res)) ? crel / res : -1.0;
        if (!res64) {
            ++rounds32;
            if (achieved <= eta || rounds32 >= 3) res64 = true;
        }
    }
    s.iterations = it;
    s.est_error = est;
    *conv_out = conv;
    return RT3D_OK;
}

}  // namespace

void rt3d::set_last_error(const char *msg) { g_err = msg; }

extern "C" {

const char *rt3d_last_error(void) { return g_err.c_str(); }

rt3d_status rt3d_grid_create(const rt3d_grid_desc *desc, rt3d_grid **out) {
    if (!out) return fail(RT3D_EINVAL, "out is NULL");
    *out = nullptr;
    TRY(validate_desc(desc));
    rt3d_grid *g = new (std::nothrow) rt3d_grid();
    if (!g) return fail(RT3D_ENOMEM, "host allocation failed");
    g->desc = *desc;
    rt3d_status st = grid_build(g);
    if (st != RT3D_OK) {
        delete g;
        return st;
    }
    *out = g;
    g_err.clear();
    return RT3D_OK;
}

void rt3d_grid_destroy(rt3d_grid *grid) {
    if (!grid) return;
    if (grid->stream) cudaStreamSynchronize(grid->stream);
    else cudaDeviceSynchronize();
    delete grid;
}

rt3d_status rt3d_grid_get_info(const rt3d_grid *g, rt3d_grid_info *info) {
    if (!g || !info) return fail(RT3D_EINVAL, "NULL argument");
    info->nangles = g->nO;
    info->kmax = g->tpl.kmax;
    info->segments = g->segments;
    info->device_bytes = g->dev_bytes;
    return RT3D_OK;
}

rt3d_status rt3d_grid_template(const rt3d_grid *gc, int angle, int *K, int32_t *vox,
                               double *len) {
    rt3d_grid *g = const_cast<rt3d_grid *>(gc);
    if (!g || !K) return fail(RT3D_EINVAL, "NULL argument");
    if (angle < 0 || angle >= g->nO) return fail(RT3D_EINVAL, "angle %d out of range", angle);
    const int k = g->K[angle];
    if (*K < k) {
        *K = k;
        return fail(RT3D_EINVAL, "capacity %d < %d points", *K, k);
    }
    *K = k;
    std::vector<long long> off(g->nO);
    CK(cudaMemcpyAsync(off.data(), g->tpl.toff, sizeof(long long) * g->nO, cudaMemcpyDeviceToHost,
                       g->stream));
    CK(cudaStreamSynchronize(g->stream));
    std::vector<uint32_t> code(k);
    CK(cudaMemcpyAsync(code.data(), g->tpl.code + off[angle], sizeof(uint32_t) * k,
                       cudaMemcpyDeviceToHost, g->stream));
    if (len)
        CK(cudaMemcpyAsync(len, g->tpl.len64 + off[angle], sizeof(double) * k,
                           cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (vox)
        for (int i = 0; i < k; ++i) {
            const uint32_t c = code[i];
            vox[i] = (int32_t)((c & 0x7ff) + g->nx * (((c >> 11) & 0x7ff) + g->ny * (c >> 22)));
        }
    return RT3D_OK;
}

rt3d_status rt3d_formal_solution(rt3d_grid *g, const double *chi, const double *S,
                                 const rt3d_bc *bc, double *J_out, double *lstar_out) {
    if (!g || !chi || !S || !J_out) return fail(RT3D_EINVAL, "NULL argument");
    const size_t N = (size_t)g->N;
    const double *dchi = nullptr, *dS = nullptr;
    TRY(stage_in(g, chi, N, g->chi, &dchi));
    TRY(stage_in(g, S, N, g->S, &dS));
    CKL(launch_pack((int)N, dchi, 1.0, dS, g->fs64 ? g->chiS64 : g->chiS32, g->fs64, g->stream));
    FsParams fp;
    TRY(fs_params(g, bc, g->fs64, false, &fp));
    TRY(run_fs(g, fp, g->fs64, lstar_out != nullptr));
    TRY(deliver(g, J_out, g->Jfs, N));
    if (lstar_out) TRY(deliver(g, lstar_out, g->lstar, 27 * N));
    CK(cudaStreamSynchronize(g->stream));
    return RT3D_OK;
}

rt3d_status rt3d_os_solve(rt3d_grid *g, const double *lstar, const double *eps, const double *r,
                          double *dJ_out, int max_sweeps, double tol, int *sweeps_out) {
    if (!g || !lstar || !eps || !r || !dJ_out) return fail(RT3D_EINVAL, "NULL argument");
    if (max_sweeps < 1 || max_sweeps > 256) return fail(RT3D_EINVAL, "max_sweeps %d", max_sweeps);
    const size_t N = (size_t)g->N;
    CK(cudaMemcpyAsync(g->lstar, lstar, 27 * N * sizeof(double), cudaMemcpyDefault, g->stream));
    CK(cudaMemcpyAsync(g->eps, eps, N * sizeof(double), cudaMemcpyDefault, g->stream));
    CK(cudaMemcpyAsync(g->tmp, r, N * sizeof(double), cudaMemcpyDefault, g->stream));
    g->lstar_valid = false;  // the grid's Lambda* now holds the caller's band
    CKL(launch_os_prep(g->nx, g->ny, g->nz, g->lstar, g->eps, g->a, g->a64, g->inv_diag, g->stream));
    TRY(os_solve_dev(g, nullptr, nullptr, g->tmp, max_sweeps, tol));
    CKL(launch_copy_buf((int)N, g->dJ_dev, g->st, g->delta, g->stream));
    TRY(deliver(g, dJ_out, g->delta, N));
    int cnt = 0;
    CK(cudaMemcpyAsync(&cnt, &g->st->count, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (sweeps_out) *sweeps_out = cnt;
    return RT3D_OK;
}

rt3d_status rt3d_ali_step(rt3d_grid *g, const double *chi, const double *eps, const double *B,
                          const rt3d_bc *bc, double *J_inout, double *rel_change_out) {
    if (!g || !chi || !eps || !B || !J_inout) return fail(RT3D_EINVAL, "NULL argument");
    const size_t N = (size_t)g->N;
    TRY(load_problem(g, chi, eps, B));
    CK(cudaMemcpyAsync(g->J, J_inout, N * sizeof(double), cudaMemcpyDefault, g->stream));
    FsParams fp;
    TRY(fs_params(g, bc, g->fs64, false, &fp));
    double rel = 0.0;
    TRY(ali_iteration(g, fp, g->fs64, 50, 1e-3, &rel));
    TRY(deliver(g, J_inout, g->J, N));
    CK(cudaStreamSynchronize(g->stream));
    if (rel_change_out) *rel_change_out = rel;
    if (!(rel == rel)) return fail(RT3D_ENUMERIC, "NaN in the ALI change");
    return RT3D_OK;
}

rt3d_status rt3d_solve(rt3d_grid *g, const double *chi, const double *eps, const double *B,
                       const rt3d_bc *bc, double *J_inout, double tol, int max_iter,
                       rt3d_solve_stats *stats) {
    const auto t_start = std::chrono::steady_clock::now();
    if (!g || !chi || !eps || !B || !J_inout) return fail(RT3D_EINVAL, "NULL argument");
    if (!(tol > 0.0) || max_iter < 1) return fail(RT3D_EINVAL, "bad tol or max_iter");
    const size_t N = (size_t)g->N;
    const int n = (int)N;
    rt3d_solve_stats s{};
    g->fs_ms[0] = g->fs_ms[1] = 0.0;
    g->launches = 0;
    TRY(load_problem(g, chi, eps, B));
    CK(cudaMemcpyAsync(g->J, J_inout, N * sizeof(double), cudaMemcpyDefault, g->stream));
    FsParams fp;
    TRY(fs_params(g, bc, g->fs64, false, &fp));
    const int max_sweeps = 50;
    const double sweep_tol = 1e-3;
    if (g->desc.accel == RT3D_ACCEL_KRYLOV) {
        FsParams fp64k, fphomk;
        TRY(fs_params(g, bc, true, false, &fp64k));
        TRY(fs_params(g, nullptr, !g->fs64 ? false : true, true, &fphomk));
        bool kconv = false;
        TRY(krylov_solve(g, fp, fp64k, fphomk, tol, max_iter, s, &kconv));
        TRY(deliver(g, J_inout, g->J, N));
        CK(cudaStreamSynchronize(g->stream));
        TRY(collect_events(g));
        s.fs32_ms = g->fs_ms[0];
        s.fs64_ms = g->fs_ms[1];
        s.launches = g->launches;
        s.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        if (stats) *stats = s;
        if (!kconv)
            return fail(RT3D_ENOTCONVERGED, "not converged after %d iterations (est %.3g)",
                        s.iterations, s.est_error);
        return RT3D_OK;
    }

    // Phase 1: ALI iterations in the grid's FS precision. The FP32 formal
    // solution carries rounding noise that the OS correction amplifies by up
    // to 1/(1 - Lambda*_vv (1-eps)); the changes then stop falling. Phase 1
    // ends when the estimated error is below tol (FP64), below the switch
    // level (FP32), or when the changes stagnate.
    double rel = 1.0, est = 1.0;
    bool conv = false;
    int it = 0;
    Progress prog;
    const double switch_at = g->fs64 ? tol : std::max(tol, 1e-6);
    while (it < max_iter) {
        TRY(ali_iteration(g, fp, g->fs64, max_sweeps, sweep_tol, &rel));
        ++it;
        if (g->fs64) ++s.fs_fp64;
        else ++s.fs_fp32;
        if (!(rel == rel)) return fail(RT3D_ENUMERIC, "NaN in the ALI change at iteration %d", it);
        prog.add(rel);
        est = prog.error_estimate();
        if (est <= switch_at && it >= 2) {
            conv = g->fs64;
            break;
        }
        if (prog.stagnated()) break;
    }
    s.rel_change = rel;

    // Phase 2 (mixed precision): defect correction with FP64 residuals,
    // r64 = J_FS64(S(J)) - J, and corrections delta from the homogeneous
    // problem (1 - Lambda(1-eps)) delta = r64 iterated with the FP32 formal
    // solution. The error after J += delta is about |delta| times the relative
    // accuracy of delta; rounds repeat until that estimate is below tol, and
    // a last FP64 formal solution certifies the returned J.
    FsParams fp64p;
    TRY(fs_params(g, bc, true, false, &fp64p));
    FsParams fphom;
    TRY(fs_params(g, nullptr, false, true, &fphom));
    const bool mixed = !g->fs64;
    if ((mixed || !conv) && it < max_iter) {
        for (int round = 0; round < 8 && it < max_iter; ++round) {
            // r64 = J_FS64(S(J)) - J
            CKL(launch_source(n, g->J, g->eps, g->B, g->chiS64, true, false, g->stream));
            TRY(run_fs(g, fp64p, true, false));
            ++s.fs_fp64;
            TRY(reset_scalar(g, offsetof(OsState, res), sizeof(unsigned long long)));
            CKL(launch_residual(n, g->Jfs, g->J, g->r64, g->st, g->stream));
            double res = 0.0;
            TRY(read_scalar_d(g, offsetof(OsState, res), &res));
            s.residual64 = res;
            if (!(res == res)) return fail(RT3D_ENUMERIC, "NaN in the FP64 residual");
            if (conv) break;  // that was the certification of the corrected J
            // delta_0 = M^-1 r64, then ALI on delta with the homogeneous FS
            TRY(os_solve_dev(g, nullptr, nullptr, g->r64, max_sweeps, sweep_tol));
            CKL(launch_copy_buf(n, g->dJ_dev, g->st, g->delta, g->stream));
            double drel = 1.0, dacc = 1.0;
            Progress dprog;
            const bool fs32 = mixed;
            for (int inner = 0; inner < 1000 && it < max_iter; ++inner) {
                CKL(launch_source(n, g->delta, g->eps, nullptr, fs32 ? g->chiS32 : g->chiS64, !fs32,
                                  true, g->stream));
                TRY(run_fs(g, fphom, !fs32, false));
                if (fs32) ++s.fs_fp32;
                else ++s.fs_fp64;
                ++it;
                // r = Lambda_hom((1-eps) delta) + r64 - delta
                TRY(os_solve_dev(g, g->Jfs, g->delta, g->r64, max_sweeps, sweep_tol));
                TRY(reset_scalar(g, offsetof(OsState, rel), sizeof(unsigned long long)));
                CKL(launch_ali_update(n, g->delta, g->dJ_dev, g->st, nullptr, g->stream));
                TRY(read_scalar_d(g, offsetof(OsState, rel), &drel));
                if (!(drel == drel)) return fail(RT3D_ENUMERIC, "NaN in the defect correction");
                dprog.add(drel);
                dacc = std::max(dprog.error_estimate(), drel);
                if (dacc <= 1e-4) break;
                if (dprog.stagnated()) break;
            }
            // J += delta; size of the correction relative to J
            TRY(reset_scalar(g, offsetof(OsState, rel), sizeof(unsigned long long)));
            CKL(launch_axpy_rel(n, g->J, g->delta, g->st, g->stream));
            double crel = 0.0;
            TRY(read_scalar_d(g, offsetof(OsState, rel), &crel));
            est = crel * dacc;
            s.rel_change = crel;
            if (est <= tol) conv = true;
        }
    } else if (conv) {
        // certification residual of the returned J
        CKL(launch_source(n, g->J, g->eps, g->B, g->chiS64, true, false, g->stream));
        TRY(run_fs(g, fp64p, true, false));
        ++s.fs_fp64;
        TRY(reset_scalar(g, offsetof(OsState, res), sizeof(unsigned long long)));
        CKL(launch_residual(n, g->Jfs, g->J, nullptr, g->st, g->stream));
        TRY(read_scalar_d(g, offsetof(OsState, res), &s.residual64));
    }
    s.iterations = it;
    s.est_error = est;
    TRY(deliver(g, J_inout, g->J, N));
    CK(cudaStreamSynchronize(g->stream));
    TRY(collect_events(g));
    s.fs32_ms = g->fs_ms[0];
    s.fs64_ms = g->fs_ms[1];
    s.launches = g->launches;
    s.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (stats) *stats = s;
    if (!conv) return fail(RT3D_ENOTCONVERGED, "not converged after %d iterations (est %.3g)", it, est);
    return RT3D_OK;
}

}  // extern "C"
