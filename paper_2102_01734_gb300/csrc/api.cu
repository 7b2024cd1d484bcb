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
#include "stream.cuh"
#include "sph_bc.cuh"
#include "sph_ff.cuh"

using namespace rt3d;

int rt3d::device_sm_count() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        cudaGetLastError();
        return 1;
    }
    if (dev < 64 && cached[dev] > 0) return cached[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    if (dev < 64) cached[dev] = n;
    return n;
}

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

// Where p points: 0 host memory (pageable or pinned) or unknown, 1 device
// memory of the current device or managed memory (usable by the library's
// kernels as is), 2 device memory of another device.
int ptr_kind(const void *p) {
    if (!p) return 0;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (at.type == cudaMemoryTypeManaged) return 1;
    if (at.type != cudaMemoryTypeDevice) return 0;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 2;
    }
    return at.device == dev ? 1 : 2;
}

bool is_device_ptr(const void *p) { return ptr_kind(p) == 1; }

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
    double *bgrad_face = nullptr;  // staged diffusion gradient face (Cartesian, [ny*nx])
    double *chi_ref = nullptr, *eps_ref = nullptr;
    double **dJ_dev = nullptr;  // device copy of {dJ[0], dJ[1]}
    float *dJ32[2] = {nullptr, nullptr};  // FP32 copies for the mixed-mode stencil
    void *chiS32 = nullptr, *chiS64 = nullptr;  // [4N] replicated 2 x 2 in x, y
    // float-float formal solution (allocated on first use): split step
    // records and split replicated (chi, S); ff_refine: refinement residuals
    // from it (RT3D_FP32_FS_FF_REFINE)
    float4 *recff = nullptr, *chiSff = nullptr;
    bool ff_refine = false;
    // FP32 formal solution without Lambda*: replicated FP64 accumulation
    // (zero between launches) and the kernel shape chosen by fs_tune
    double *Jrep = nullptr;  // [4N]
    float4 *pairs = nullptr;  // [4N] pair-packed FP32 (chi, S) of the two-characteristic kernel
    FsShape fs_shape{0, 0, 0, 0};  // block 0: not chosen yet
    float fs_tune_ms[RT3D_FS_TUNE_SHAPES] = {};  // last tuning: time of each shape
    void *a = nullptr;  // 26 OS off-diagonal planes, os_coef_index layout (f64 in FP64 mode, f32 otherwise)
    bool a64 = true;
    // OS solver (rt3d_grid_set_os_solver): the coefficients use the colour
    // layout under Gauss-Seidel; diag = 1 - Lambda*_0 (1 - eps) for BiCGStab's
    // products; BiCGStab's vectors and scalars allocated on first use
    int os_kind = kOsJacobi;
    double *diag = nullptr;
    double *bres = nullptr, *brh = nullptr, *bp = nullptr, *bvv = nullptr, *bsv = nullptr,
           *bt = nullptr;
    BicgState *bicg = nullptr;
    OsState *st = nullptr;
    bool lstar_valid = false;

    // Krylov workspace (allocated on first use): basis V[0..m], preconditioned
    // directions Z[0..m-1], their device pointer arrays, small scalars
    static constexpr int kKrylov = 100;
    bool krylov_ready = false;
    double *V[kKrylov + 1] = {}, *Z[kKrylov] = {};
    double **dV = nullptr, **dZ = nullptr, **dOne = nullptr;
    double *dots = nullptr, *coef = nullptr;

    // spherical grid: trig tables and the ray cache
    bool sph = false;
    Periodic per{true, true, false};
    double *s_re2 = nullptr, *s_ct = nullptr, *s_ctk = nullptr, *s_cpe = nullptr, *s_spe = nullptr;
    double *s_rc = nullptr, *s_stc = nullptr, *s_ctc = nullptr, *s_cpc = nullptr, *s_spc = nullptr;
    long long s_nrays = 0, s_nseg = 0;
    std::vector<long long> s_ray_base;
    std::vector<int> s_nrays_angle;
    long long *s_ray_off = nullptr;
    int *s_ray_len = nullptr, *s_ray_angle = nullptr, *s_ray_launch = nullptr;
    int *s_ray_kind = nullptr, *s_ray_face = nullptr;
    // per segment (24 bytes): record (replicated index bits, FP32 J weight,
    // l/2, FP32 remainder of the FP64 J weight) and the FP64 chord
    float4 *s_rec = nullptr;
    double *s_len64 = nullptr;
    // host cache modes (RT3D_CACHE_HOST_*): the records above (only the FP64
    // chords in the chords mode) are the device addresses of pinned, mapped
    // host arrays; chunk c holds the angles [c_angle[c], c_angle[c+1]), their
    // rays from c_ray[c] and segments from c_seg[c] (ray offsets relative to
    // c_seg[c]); the streaming modes copy a chunk into slot c % 2 on cstream
    // (c_free: the slot's last kernel is done; c_copied: the chunk is in the
    // slot; c_fork: the formal solution began); without copies the chunks'
    // kernels alternate between the grid's stream and cstream
    int cache = RT3D_CACHE_DEVICE;
    // diffusion inner boundary: the directions on the device, the radial
    // cell centres on the host, and (allocated on first use) every ray's
    // entry intensity with the identity index the kernels read it through
    double *s_dir = nullptr;
    std::vector<double> s_rc_h;
    double *s_ray_I0 = nullptr;
    int *s_ident = nullptr;
    float4 *h_rec = nullptr;
    double *h_len64 = nullptr;
    std::vector<int> c_angle;
    std::vector<long long> c_ray, c_seg, s_angle_chunk_seg;
    float4 *slot_rec[2] = {nullptr, nullptr};
    double *slot_len64[2] = {nullptr, nullptr};
    cudaStream_t cstream = nullptr;
    cudaEvent_t c_fork = nullptr, c_copied[2] = {nullptr, nullptr}, c_free[2] = {nullptr, nullptr};
    std::vector<void *> host_allocs;
    long long host_bytes = 0;

    // batched-wavelength workspace (allocated for the largest n_lambda seen)
    int bl_cap = 0;
    double *bchi = nullptr, *beps = nullptr, *bB = nullptr, *bJ = nullptr, *br = nullptr;
    double *bbuf0 = nullptr, *bbuf1 = nullptr, *binv = nullptr, *bJrep = nullptr;
    float *bb32_0 = nullptr, *bb32_1 = nullptr;
    double *btop = nullptr, *bbot = nullptr, *bgrad = nullptr;
    float2 *bchiS = nullptr;
    float *ba = nullptr;
    BatchState bsh{};             // host copy of the device pointers
    BatchState *bsd = nullptr;    // device copy
    cudaStream_t bstream = nullptr;
    cudaEvent_t bev0 = nullptr, bev1 = nullptr;
    FsShape bfs_shape{0, 0, 0, 0};  // batched FS shape (block 0: not tuned)
    float bfs_tune_ms[RT3D_FS_TUNE_SHAPES] = {};

    // line-transfer workspace (allocated on first use): the profile-averaged
    // Lambda* band [27][N] and formal solution [N], a device table of the
    // vectors they accumulate ({Jfs, Lambda* plane 0..26}) and the negated
    // profile weights (-wphi[l], for multi_axpy's w -= c V)
    double *lbar = nullptr, *jbar_fs = nullptr;
    double **lptr = nullptr;
    double *lcoef = nullptr;
    int lcoef_cap = 0;

    // instrumentation: formal-solution kernel time (CUDA events on the
    // grid's stream) and kernels launched
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int ev_pending = -1;  // -1 none, 0 FP32, 1 FP64, 2 float-float, 3 FP32 with Lambda*
    double fs_ms[4] = {0.0, 0.0, 0.0, 0.0};
    int fs_lstar32 = 0;   // FP32 formal solutions with Lambda* since the last reset
    long long launches = 0;

    template <typename T>
    rt3d_status alloc(T **p, size_t count) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            size_t fr = 0, tot = 0;
            cudaMemGetInfo(&fr, &tot);
            cudaGetLastError();
            return fail(RT3D_ENOMEM,
                        "cudaMalloc of %zu bytes failed: %s (grid holds %lld bytes; %zu of %zu free)",
                        count * sizeof(T), cudaGetErrorString(e), dev_bytes, fr, tot);
        }
        allocs.push_back(q);
        dev_bytes += (long long)(count * sizeof(T));
        *p = static_cast<T *>(q);
        return RT3D_OK;
    }
    // frees a device allocation of alloc() (count elements of T) before the
    // grid is destroyed; synchronises the device (cudaFree)
    template <typename T>
    void release(T *&p, size_t count) {
        if (!p) return;
        auto it = std::find(allocs.begin(), allocs.end(), static_cast<void *>(p));
        if (it != allocs.end()) {
            allocs.erase(it);
            cudaFree(p);
            dev_bytes -= (long long)(count * sizeof(T));
        }
        p = nullptr;
    }
    // pinned, mapped host memory; *dev receives its device address
    template <typename T>
    rt3d_status alloc_host(T **p, T **dev, size_t count) {
        void *q = nullptr;
        cudaError_t e = cudaHostAlloc(&q, count * sizeof(T) + 16, cudaHostAllocMapped);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(RT3D_ENOMEM, "cudaHostAlloc of %zu bytes failed: %s (grid holds %lld "
                        "host bytes)", count * sizeof(T), cudaGetErrorString(e), host_bytes);
        }
        host_allocs.push_back(q);
        host_bytes += (long long)(count * sizeof(T));
        void *d = nullptr;
        e = cudaHostGetDevicePointer(&d, q, 0);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(RT3D_ECUDA, "cudaHostGetDevicePointer failed: %s", cudaGetErrorString(e));
        }
        *p = static_cast<T *>(q);
        *dev = static_cast<T *>(d);
        return RT3D_OK;
    }
    ~rt3d_grid() {
        if (cstream) cudaStreamDestroy(cstream);
        if (c_fork) cudaEventDestroy(c_fork);
        for (int i = 0; i < 2; ++i) {
            if (c_copied[i]) cudaEventDestroy(c_copied[i]);
            if (c_free[i]) cudaEventDestroy(c_free[i]);
        }
        for (void *p : host_allocs) cudaFreeHost(p);
        if (bstream) cudaStreamDestroy(bstream);
        if (bev0) cudaEventDestroy(bev0);
        if (bev1) cudaEventDestroy(bev1);
        for (void *p : allocs) cudaFree(p);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
    }
};

namespace {

// Input: a pointer to the grid's device memory (or managed memory) as is;
// a host array, or another device's array, copied into `stage`.
rt3d_status stage_in(rt3d_grid *g, const double *p, size_t n, double *stage, const double **out) {
    if (!p) {
        *out = nullptr;
        return RT3D_OK;
    }
    if (is_device_ptr(p)) {
        *out = p;
        return RT3D_OK;
    }
    CK(cudaMemcpyAsync(stage, p, n * sizeof(double), cudaMemcpyDefault, g->stream));
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
    q.mu = g->tpl.mu;
    q.code = g->tpl.code;
    q.len = fp64 ? (const void *)g->tpl.len64 : (const void *)g->tpl.len32;
    q.cw = fp64 ? (const void *)g->tpl.cw64 : (const void *)g->tpl.cw32;
    q.win = g->tpl.win;
    q.rec32 = g->tpl.rec32;
    q.rec64 = g->tpl.rec64;
    q.Jrep = g->Jrep;
    q.pairs = g->pairs;
    q.rec4 = g->tpl.rec4;
    q.chiS = fp64 ? g->chiS64 : g->chiS32;
    q.homogeneous = homogeneous ? 1 : 0;
    if (bc && !homogeneous) {
        q.I_top = bc->I_top;
        q.I_bot = bc->I_bottom;
        q.I_irr = bc->I_irr;
        const double *tf = nullptr, *bf = nullptr;
        const size_t nf = (size_t)g->nx * g->ny;
        const size_t nfb = g->sph ? (size_t)g->ny * g->nz : nf;  // spherical core face
        if (!g->sph) TRY(stage_in(g, bc->I_top_face, nf, g->top, &tf));
        TRY(stage_in(g, bc->I_bottom_face, nfb, g->bot, &bf));
        const double *gf = nullptr;
        TRY(stage_in(g, bc->I_bottom_grad, nfb, g->bgrad_face, &gf));
        q.top_face = tf;
        q.bot_face = bf;
        q.bot_grad = gf;
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

// Candidate shapes of the FP32 formal-solution kernel without Lambda* that
// fs_tune times: (threads per block, characteristics per thread, widening,
// branchless parabolic correction). Two characteristics per thread is the
// packed FP32x2 kernel, four the packed kernel that sums J contributions in
// registers before the FP64 reduction (both always branchless; widening 2 of
// the four-characteristic kernel is the conversion, as 0). A grid where a
// candidate cannot run records 0 for it.
constexpr FsShape kFsShapes[RT3D_FS_TUNE_SHAPES] = {
    {256, 1, 0, 1}, {128, 2, 1, 1}, {256, 2, 2, 1}, {256, 4, 1, 1},
    {128, 4, 1, 1}, {64, 4, 1, 1},  {256, 4, 0, 1}, {128, 4, 0, 1}};

// Autotuner of the FP32 formal solution's ray-bundle shape: times one launch
// of every shape on the grid's current (chi, S) (CUDA events on the grid's
// stream, after one untimed launch) and keeps the fastest. Each launch is
// folded into g->Jfs, which the caller's launch overwrites.
rt3d_status fs_tune(rt3d_grid *g, const FsParams &p) {
    TRY(collect_events(g));
    float best = 0.0f;
    int pick = 0;
    for (int i = -1; i < RT3D_FS_TUNE_SHAPES; ++i) {
        const int c = i < 0 ? 0 : i;
        if (kFsShapes[c].rays_per_thread == 4 && !quad_applicable(p)) {
            g->fs_tune_ms[c] = 0.0f;  // not available on this grid
            continue;
        }
        CK(cudaEventRecord(g->ev0, g->stream));
        CK(launch_fs_fast(p, g->parab, kFsShapes[c], g->stream));
        CK(cudaEventRecord(g->ev1, g->stream));
        CK(launch_fold(g->nx, g->ny, g->nz, g->Jrep, g->Jfs, g->stream));
        g->launches += 2;
        CK(cudaEventSynchronize(g->ev1));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
        if (i >= 0) g->fs_tune_ms[i] = ms;
        if (i >= 0 && (i == 0 || ms < best)) {
            best = ms;
            pick = i;
        }
    }
    g->fs_shape = kFsShapes[pick];
    return RT3D_OK;
}

// One formal solution on the spherical cache into g->Jfs (Lambda* into
// g->lstar when requested): kind 0 FP32, 1 FP64, 2 float-float (without
// Lambda*); chiS the replicated (chi, S) of that kind. The FP64 and
// float-float kernels read the FP64 chords, which the host residencies copy
// or read in place with the records.
rt3d_status run_fs_sph(rt3d_grid *g, const FsParams &base, const void *chiS, int kind,
                       bool with_lstar) {
    const bool fp64 = kind != 0;
    SphFsParams sp{};
    sp.nrays = g->s_nrays;
    sp.N = (int)g->N;
    sp.ray_off = g->s_ray_off;
    sp.ray_len = g->s_ray_len;
    sp.ray_kind = g->s_ray_kind;
    sp.ray_face = g->s_ray_face;
    sp.nr = g->nx;
    sp.nt = g->ny;
    sp.np = g->nz;
    sp.rec = g->s_rec;
    sp.len64 = g->s_len64;
    sp.chiS = chiS;
    sp.J = g->Jfs;
    sp.lstar = with_lstar ? g->lstar : nullptr;
    sp.core_face = base.bot_face;
    sp.I_core = base.I_bot;
    sp.I_out = base.I_top;
    sp.I_irr = base.I_irr;
    sp.homogeneous = base.homogeneous;
    if (base.bot_grad && !base.homogeneous) {
        // diffusion condition on the core: every ray's entry intensity,
        // read by the kernels as a per-ray core face
        if (!g->s_ray_I0) {
            TRY(g->alloc(&g->s_ray_I0, g->s_nrays));
            TRY(g->alloc(&g->s_ident, g->s_nrays));
        }
        SphEntryParams ep{g->s_nrays, g->nx, g->ny, g->desc.r_in, g->s_ray_launch,
                          g->s_ray_angle, g->s_ray_kind, g->s_ray_face, g->s_rc,
                          g->s_stc, g->s_ctc, g->s_cpc, g->s_spc, g->s_dir};
        CKL(launch_sph_entry(ep, base.bot_face, base.I_bot, base.bot_grad, g->s_ray_I0,
                             g->s_ident, g->stream));
        sp.core_face = g->s_ray_I0;
        sp.ray_face = g->s_ident;
    }
    // without Lambda*: the record kernels (FP32, FP64 or float-float) into
    // the replicated Jrep, folded after
    const bool sfast = !with_lstar;
    if (!sfast) CK(cudaMemsetAsync(g->Jfs, 0, sizeof(double) * g->N, g->stream));
    if (with_lstar) CK(cudaMemsetAsync(g->lstar, 0, sizeof(double) * 27 * g->N, g->stream));
    TRY(collect_events(g));
    CK(cudaEventRecord(g->ev0, g->stream));
    auto launch = [&](const SphFsParams &q, cudaStream_t ks) -> cudaError_t {
        if (!sfast) return launch_sph_fs(q, fp64, g->parab, with_lstar, ks);
        if (kind == 2)
            return launch_sph_fsff(q, static_cast<const float4 *>(chiS), g->Jrep, g->parab, ks);
        return fp64 ? launch_sph_fs64_fast(q, g->Jrep, g->parab, ks)
                    : launch_sph_fs_fast(q, g->Jrep, g->parab, ks);
    };
    if (g->cache == RT3D_CACHE_DEVICE) {
        CK(launch(sp, g->stream));
        ++g->launches;
    } else {
        // host records, chunk by chunk of solid angles: the streamed mode
        // copies chunk c into slot c % 2 on the copy stream once the
        // kernel of chunk c - 2 has released the slot, and the kernel of
        // chunk c waits for its copy; the mapped mode reads the chunk in
        // place; the chords mode reads the records on the device and
        // streams the FP64 chords, which only the FP64 and float-float
        // kernels read (fp64 here covers both; the FP32 kernels never read
        // cp.len64).
        const bool chords = g->cache == RT3D_CACHE_HOST_CHORDS;
        const bool copy = g->cache == RT3D_CACHE_HOST_STREAMED || (chords && fp64);
        // without copies the chunks' kernels alternate between the grid's
        // stream and the second stream, so that the tail of one overlaps
        // the next (they only add into J and Lambda*)
        const bool alt = !copy;
        CK(cudaEventRecord(g->c_fork, g->stream));
        CK(cudaStreamWaitEvent(g->cstream, g->c_fork, 0));
        const int nch = (int)g->c_angle.size() - 1;
        for (int c = 0; c < nch; ++c) {
            SphFsParams cp = sp;
            const long long r0 = g->c_ray[c], s0 = g->c_seg[c], ns = g->c_seg[c + 1] - s0;
            cp.nrays = g->c_ray[c + 1] - r0;
            cp.ray_off = sp.ray_off + r0;
            cp.ray_len = sp.ray_len + r0;
            cp.ray_kind = sp.ray_kind + r0;
            cp.ray_face = sp.ray_face + r0;
            const int k = c & 1;
            cp.rec = g->s_rec + s0;
            cp.len64 = g->s_len64 + s0;
            if (copy) {
                CK(cudaStreamWaitEvent(g->cstream, g->c_free[k], 0));
                if (!chords) {
                    CK(cudaMemcpyAsync(g->slot_rec[k], g->h_rec + s0, sizeof(float4) * ns,
                                       cudaMemcpyHostToDevice, g->cstream));
                    cp.rec = g->slot_rec[k];
                }
                if (fp64)
                    CK(cudaMemcpyAsync(g->slot_len64[k], g->h_len64 + s0, sizeof(double) * ns,
                                       cudaMemcpyHostToDevice, g->cstream));
                cp.len64 = g->slot_len64[k];
                CK(cudaEventRecord(g->c_copied[k], g->cstream));
                CK(cudaStreamWaitEvent(g->stream, g->c_copied[k], 0));
            }
            cudaStream_t ks = alt && k ? g->cstream : g->stream;
            CK(launch(cp, ks));
            ++g->launches;
            if (copy) CK(cudaEventRecord(g->c_free[k], g->stream));
        }
        if (alt) {  // join
            CK(cudaEventRecord(g->c_copied[0], g->cstream));
            CK(cudaStreamWaitEvent(g->stream, g->c_copied[0], 0));
        }
    }
    CK(cudaEventRecord(g->ev1, g->stream));
    g->ev_pending = kind == 2 ? 2 : fp64 ? 1 : (with_lstar ? 3 : 0);
    if (!fp64 && with_lstar) ++g->fs_lstar32;
    if (sfast) {
        CK(launch_fold(g->nx, g->ny, g->nz, g->Jrep, g->Jfs, g->stream));
        ++g->launches;
    }
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
    if (g->sph) return run_fs_sph(g, base, p.chiS, fp64 ? 1 : 0, with_lstar);
    // without Lambda*: the replicated-accumulation kernels (J folded after)
    const bool fast = !with_lstar;
    if (fast && !fp64 && g->fs_shape.block == 0) TRY(fs_tune(g, p));
    if (!fast) CK(cudaMemsetAsync(g->Jfs, 0, sizeof(double) * g->N, g->stream));
    if (with_lstar) CK(cudaMemsetAsync(g->lstar, 0, sizeof(double) * 27 * g->N, g->stream));
    TRY(collect_events(g));
    CK(cudaEventRecord(g->ev0, g->stream));
    if (fast && fp64) CK(launch_fs64_fast(p, g->parab, g->stream));
    else if (fast) CK(launch_fs_fast(p, g->parab, g->fs_shape, g->stream));
    else CK(launch_fs(p, fp64, g->parab, with_lstar, g->stream));
    CK(cudaEventRecord(g->ev1, g->stream));
    g->ev_pending = fp64 ? 1 : (with_lstar ? 3 : 0);
    if (!fp64 && with_lstar) ++g->fs_lstar32;
    ++g->launches;
    if (fast) {
        CK(launch_fold(g->nx, g->ny, g->nz, g->Jrep, g->Jfs, g->stream));
        ++g->launches;
    }
    return RT3D_OK;
}

// Float-float formal solution of S = src (or (1 - eps) src + eps B when eps
// is given) into g->Jfs; allocates its split inputs on first use.
rt3d_status run_fs_ff(rt3d_grid *g, const FsParams &base, const double *chi, const double *src,
                      const double *eps, const double *B) {
    if (g->sph) {
        // the records carry the float-float J weight and the FP32 half chord;
        // only the split (chi, S) is needed
        if (!g->chiSff) TRY(g->alloc(&g->chiSff, 4 * (size_t)g->N));
        CKL(launch_pack_ff(g->nx, g->ny, g->nz, chi, src, eps, B, g->chiSff, g->stream));
        return run_fs_sph(g, base, g->chiSff, 2, false);
    }
    if (!g->recff) {
        TRY(g->alloc(&g->recff, (size_t)g->tpl.total));
        TRY(g->alloc(&g->chiSff, 4 * (size_t)g->N));
        CKL(launch_recff(g->tpl.total, g->tpl.rec64, g->recff, g->stream));
    }
    CKL(launch_pack_ff(g->nx, g->ny, g->nz, chi, src, eps, B, g->chiSff, g->stream));
    TRY(collect_events(g));
    CK(cudaEventRecord(g->ev0, g->stream));
    CK(launch_fsff(base, g->recff, g->chiSff, g->parab, g->stream));
    CK(cudaEventRecord(g->ev1, g->stream));
    g->ev_pending = 2;
    CK(launch_fold(g->nx, g->ny, g->nz, g->Jrep, g->Jfs, g->stream));
    g->launches += 3;
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
    CK(launch_os_init((int)g->N, Jfs, J, extra, g->inv_diag, g->r, g->dJ[0],
                      g->a64 ? nullptr : g->dJ32[0], g->st, g->stream));
    ++g->launches;
    if (g->os_kind == kOsJacobi) {
        for (int m = 1; m <= max_sweeps; ++m)
            CK(launch_os_sweep(g->nx, g->ny, g->nz, g->a, g->a64, g->inv_diag, g->r, g->dJ,
                               g->a64 ? nullptr : g->dJ32, m, tol, g->st, g->stream, g->per));
        CK(launch_os_finish(max_sweeps, tol, g->st, g->stream));
        g->launches += max_sweeps + 1;
        return RT3D_OK;
    }
    if (g->os_kind == kOsGaussSeidel) {
        // eight launches per sweep; the stop flag is read every fourth sweep
        const ColourGeo cg = colour_geo(g->nx, g->ny, g->nz);
        for (int m = 1; m <= max_sweeps; ++m) {
            CK(launch_gs_sweep(g->nx, g->ny, g->nz, cg, g->a, g->a64, g->inv_diag, g->r,
                               g->dJ[(m - 1) & 1], g->dJ[m & 1],
                               g->a64 ? nullptr : g->dJ32[(m - 1) & 1],
                               g->a64 ? nullptr : g->dJ32[m & 1], m, tol, g->st, g->stream,
                               g->per));
            g->launches += 8;
            if ((m & 3) == 0 && m < max_sweeps) {
                int done = 0;
                CK(cudaMemcpyAsync(&done, &g->st->done, sizeof done, cudaMemcpyDeviceToHost,
                                   g->stream));
                CK(cudaStreamSynchronize(g->stream));
                if (done) break;
            }
        }
        CK(launch_os_finish(max_sweeps, tol, g->st, g->stream));
        ++g->launches;
        return RT3D_OK;
    }
    // BiCGStab from dJ = 0 (dJ[0] holds the iterate), stop on ||res||_2 <=
    // tol ||r||_2 or after max_sweeps iterations, or at a breakdown (omega = 0)
    const int n = (int)g->N;
    if (!g->bicg) {
        TRY(g->alloc(&g->bres, (size_t)n));
        TRY(g->alloc(&g->brh, (size_t)n));
        TRY(g->alloc(&g->bp, (size_t)n));
        TRY(g->alloc(&g->bvv, (size_t)n));
        TRY(g->alloc(&g->bsv, (size_t)n));
        TRY(g->alloc(&g->bt, (size_t)n));
        TRY(g->alloc(&g->bicg, 1));
    }
    const BicgVecs v{g->dJ[0], g->bres, g->brh, g->bp, g->bvv, g->bsv, g->bt};
    CK(launch_bicg_init(n, g->r, v, g->bicg, g->stream));
    ++g->launches;
    BicgState hs{};
    CK(cudaMemcpyAsync(&hs, g->bicg, sizeof hs, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    const double nr0 = std::sqrt(hs.rr0);
    int k = 0;
    if (nr0 > 0.0) {
        while (k < max_sweeps) {
            CK(launch_bicg_iteration(g->nx, g->ny, g->nz, g->a, g->a64, g->diag, v, g->bicg,
                                     g->stream, g->per));
            g->launches += 9;
            ++k;
            CK(cudaMemcpyAsync(&hs, g->bicg, sizeof hs, cudaMemcpyDeviceToHost, g->stream));
            CK(cudaStreamSynchronize(g->stream));
            if (!(hs.rr == hs.rr)) return fail(RT3D_ENUMERIC, "NaN in the BiCGStab residual");
            if (std::sqrt(hs.rr) <= tol * nr0) break;
            if (hs.omega == 0.0) break;
        }
    }
    CK(launch_os_set_result(n, g->dJ[0], g->dJ[k & 1], k, g->st, g->stream));
    ++g->launches;
    return RT3D_OK;
}

// OS solve caps of the solver's own unit: a BiCGStab iteration applies the
// matrix twice, so it counts as two sweeps of a cap given in sweeps.
int os_cap(const rt3d_grid *g, int sweeps) {
    return g->os_kind == kOsBicgstab ? std::max(1, sweeps / 2) : sweeps;
}

// Work buffers of the formal solution and the solvers.
rt3d_status alloc_work(rt3d_grid *g) {
    cudaStream_t s = g->stream;
    // work buffers
    const size_t N = (size_t)g->N;
    const size_t nf = g->sph ? (size_t)g->ny * g->nz : (size_t)g->nx * g->ny;
    TRY(g->alloc(&g->chi, N));
    TRY(g->alloc(&g->eps, N));
    TRY(g->alloc(&g->B, N));
    TRY(g->alloc(&g->S, N));
    TRY(g->alloc(&g->J, N));
    TRY(g->alloc(&g->Jfs, N));
    TRY(g->alloc(&g->r, N));
    TRY(g->alloc(&g->dJ[0], N));
    TRY(g->alloc(&g->dJ[1], N));
    TRY(g->alloc(&g->dJ32[0], N));
    TRY(g->alloc(&g->dJ32[1], N));
    TRY(g->alloc(&g->inv_diag, N));
    TRY(g->alloc(&g->tmp, N));
    TRY(g->alloc(&g->delta, N));
    TRY(g->alloc(&g->r64, N));
    TRY(g->alloc(&g->chi_ref, N));
    TRY(g->alloc(&g->eps_ref, N));
    TRY(g->alloc(&g->lstar, 27 * N));
    TRY(g->alloc(&g->top, nf));
    TRY(g->alloc(&g->bot, nf));
    TRY(g->alloc(&g->bgrad_face, nf));
    TRY(g->alloc(&g->dJ_dev, 2));
    TRY(g->alloc(reinterpret_cast<double2 **>(&g->chiS64), 4 * N));
    TRY(g->alloc(reinterpret_cast<float2 **>(&g->chiS32), 4 * N));
    TRY(g->alloc(&g->Jrep, 4 * N));
    CK(cudaMemsetAsync(g->Jrep, 0, sizeof(double) * 4 * N, s));
    if (!g->sph && !g->fs64) TRY(g->alloc(&g->pairs, 4 * N));
    if (g->a64) TRY(g->alloc(reinterpret_cast<double **>(&g->a), os_coef_alloc(N)));
    else TRY(g->alloc(reinterpret_cast<float **>(&g->a), os_coef_alloc(N)));
    TRY(g->alloc(&g->diag, N));
    TRY(g->alloc(&g->st, 1));
    CK(cudaMemcpyAsync(g->dJ_dev, g->dJ, sizeof(double *) * 2, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(g->st, 0, sizeof(OsState), s));
    CK(cudaEventCreate(&g->ev0));
    CK(cudaEventCreate(&g->ev1));
    CK(cudaStreamSynchronize(s));
    return RT3D_OK;
}

// Host memory this process may still take, in bytes: MemAvailable, lowered
// to the cgroup's limit less its usage where one is set (v2, else v1); -1
// when none of them can be read.
long long host_memory_available() {
    long long avail = -1;
    if (FILE *f = std::fopen("/proc/meminfo", "r")) {
        char line[256];
        long long kb = 0;
        while (std::fgets(line, sizeof line, f))
            if (std::sscanf(line, "MemAvailable: %lld kB", &kb) == 1) avail = kb * 1024;
        std::fclose(f);
    }
    auto read_ll = [](const char *path, long long *v) -> bool {
        FILE *f = std::fopen(path, "r");
        if (!f) return false;
        const bool ok = std::fscanf(f, "%lld", v) == 1;  // "max" (no limit) reads as no number
        std::fclose(f);
        return ok;
    };
    long long lim = 0, used = 0;
    if ((read_ll("/sys/fs/cgroup/memory.max", &lim) && read_ll("/sys/fs/cgroup/memory.current", &used)) ||
        (read_ll("/sys/fs/cgroup/memory/memory.limit_in_bytes", &lim) &&
         read_ll("/sys/fs/cgroup/memory/memory.usage_in_bytes", &used))) {
        const long long room = std::max(0LL, lim - used);
        if (lim < (1LL << 60)) avail = avail < 0 ? room : std::min(avail, room);
    }
    return avail;
}

// Spherical geometry cache: trig tables on the host (plain IEEE arithmetic
// and libm), the ray set of every solid angle built on the device in angle
// chunks (pass 1 counts rays and segments, pass 2 fills the tables). In the
// host cache modes pass 2 runs chunk of angles by chunk of angles (the
// residency chunks of the formal solution) into a device buffer, with
// segment offsets relative to the chunk, and each chunk is copied to the
// pinned host records.
rt3d_status sph_build(rt3d_grid *g) {
    const rt3d_grid_desc &d = g->desc;
    const int nr = g->nx, nt = g->ny, np = g->nz, nO = g->nO;
    const long long N = g->N;
    std::vector<double> re(nr + 1), re2(nr + 1), ct(nt + 1), ctk(nt + 1), cpe(np), spe(np), rc(nr),
        stc(nt), ctc(nt), cpc(np), spc(np);
    for (int i = 0; i <= nr; ++i) re[i] = d.r_in * std::pow(d.r_out / d.r_in, (double)i / (double)nr);
    re[0] = d.r_in;
    re[nr] = d.r_out;
    for (int i = 0; i <= nr; ++i) re2[i] = re[i] * re[i];
    for (int j = 0; j <= nt; ++j) {
        double c = std::cos((double)j * M_PI / (double)nt);
        if (2 * j == nt) c = 0.0;
        if (j == 0) c = 1.0;
        if (j == nt) c = -1.0;
        ct[j] = c;
        ctk[j] = c * std::fabs(c);
    }
    for (int k = 0; k < np; ++k) {
        const double ph = 2.0 * M_PI * (double)k / (double)np;
        cpe[k] = std::cos(ph);
        spe[k] = std::sin(ph);
        const double pc = 2.0 * M_PI * ((double)k + 0.5) / (double)np;
        cpc[k] = std::cos(pc);
        spc[k] = std::sin(pc);
    }
    for (int i = 0; i < nr; ++i) rc[i] = std::sqrt(re[i] * re[i + 1]);
    for (int j = 0; j < nt; ++j) {
        const double t = ((double)j + 0.5) * M_PI / (double)nt;
        stc[j] = std::sin(t);
        ctc[j] = std::cos(t);
    }
    cudaStream_t s = g->stream;
    auto up = [&](double **dst, const std::vector<double> &v) -> rt3d_status {
        TRY(g->alloc(dst, v.size()));
        CK(cudaMemcpyAsync(*dst, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice, s));
        return RT3D_OK;
    };
    TRY(up(&g->s_re2, re2));
    TRY(up(&g->s_ct, ct));
    TRY(up(&g->s_ctk, ctk));
    TRY(up(&g->s_cpe, cpe));
    TRY(up(&g->s_spe, spe));
    TRY(up(&g->s_rc, rc));
    TRY(up(&g->s_stc, stc));
    TRY(up(&g->s_ctc, ctc));
    TRY(up(&g->s_cpc, cpc));
    TRY(up(&g->s_spc, spc));
    double *d_dir = nullptr, *d_wt = nullptr;
    TRY(up(&d_dir, g->dir));
    TRY(up(&d_wt, g->wt));
    SphBuildParams bp{};
    bp.T = SphTables{nr, nt, np, g->s_re2, g->s_ct, g->s_ctk, g->s_cpe, g->s_spe,
                     g->s_rc, g->s_stc, g->s_ctc, g->s_cpc, g->s_spc};
    bp.nangles = nO;
    bp.ncap = 2 * (nr + 1) + 2 * (nt + 1) + np + 8;
    bp.dir = d_dir;
    bp.wt = d_wt;
    // chunk of angles built at once (one warp each): scratch N/8 + 8 N + 8 ncap
    // bytes per angle, within an eighth of the free device memory (at least
    // 2 GiB, at most 16 GiB), so that large grids still fill the GPU with
    // warps
    const long long per_angle = N / 8 + 8 * N + 8LL * bp.ncap + 64;
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    const long long budget =
        std::min<long long>(16LL << 30, std::max<long long>(2LL << 30, (long long)(free_b / 8)));
    int chunk = (int)std::max(1LL, std::min<long long>(nO, budget / per_angle));
    const int words = (int)((N + 31) / 32);
    unsigned *hit = nullptr;
    double *tbuf = nullptr, *den = nullptr;
    int *d_nrays = nullptr, *d_err = nullptr;
    long long *d_nseg = nullptr;
    TRY(g->alloc(&hit, (size_t)chunk * words));
    TRY(g->alloc(&tbuf, (size_t)chunk * bp.ncap));
    TRY(g->alloc(&den, (size_t)chunk * N));
    TRY(g->alloc(&d_nrays, nO));
    TRY(g->alloc(&d_nseg, nO));
    TRY(g->alloc(&d_err, 1));
    CK(cudaMemsetAsync(d_err, 0, sizeof(int), s));
    bp.hit = hit;
    bp.tbuf = tbuf;
    bp.den = den;
    bp.nrays = d_nrays;
    bp.nseg = d_nseg;
    bp.err = d_err;
    bp.pass = 1;
    for (int o0 = 0; o0 < nO; o0 += chunk) {
        bp.o0 = o0;
        bp.nchunk = std::min(chunk, nO - o0);
        CK(launch_sph_build(bp, s));
    }
    std::vector<int> nrays(nO);
    std::vector<long long> nseg(nO);
    int herr = 0;
    CK(cudaMemcpyAsync(nrays.data(), d_nrays, sizeof(int) * nO, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(nseg.data(), d_nseg, sizeof(long long) * nO, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (herr) return fail(RT3D_EINVAL, "spherical tracer error %d", herr);
    std::vector<long long> rbase(nO), sbase(nO);
    long long tr = 0, tsg = 0;
    for (int o = 0; o < nO; ++o) {
        rbase[o] = tr;
        sbase[o] = tsg;
        tr += nrays[o];
        tsg += nseg[o];
    }
    if (tsg >= (1LL << 40)) return fail(RT3D_EINVAL, "spherical cache too large");
    g->s_nrays = tr;
    g->s_nseg = tsg;
    g->s_ray_base = rbase;
    g->s_nrays_angle = nrays;
    // residency chunks: all angles on the device; in the host modes runs of
    // consecutive angles whose records fit stream_bytes (at least one angle)
    const bool host = g->cache != RT3D_CACHE_DEVICE;
    const bool chords = g->cache == RT3D_CACHE_HOST_CHORDS;  // only the FP64 chords on the host
    std::vector<long long> sloc(nO);  // segment base of each angle handed to pass 2
    g->c_angle.assign(1, 0);
    g->c_ray.assign(1, 0);
    g->c_seg.assign(1, 0);
    g->s_angle_chunk_seg.assign(nO, 0);
    if (host) {
        const long long cap = std::max(
            1LL, (d.stream_bytes > 0 ? d.stream_bytes : (1LL << 30)) / (chords ? 8 : 24));
        for (int o = 0; o < nO; ++o) {
            if (sbase[o] > g->c_seg.back() && sbase[o] + nseg[o] - g->c_seg.back() > cap) {
                g->c_angle.push_back(o);
                g->c_ray.push_back(rbase[o]);
                g->c_seg.push_back(sbase[o]);
            }
            g->s_angle_chunk_seg[o] = g->c_seg.back();
            sloc[o] = sbase[o] - g->c_seg.back();
        }
    } else {
        sloc = sbase;
    }
    g->c_angle.push_back(nO);
    g->c_ray.push_back(tr);
    g->c_seg.push_back(tsg);
    const int nch = (int)g->c_angle.size() - 1;
    long long maxc = 0;
    for (int c = 0; c < nch; ++c) maxc = std::max(maxc, g->c_seg[c + 1] - g->c_seg[c]);
    const int nslots = g->cache == RT3D_CACHE_HOST_STREAMED || chords ? 2 : 0;
    {
        // the cache: 28 bytes per ray on the device; 24 per segment on the
        // device, or in pinned host memory with device buffers of the largest chunk
        size_t fr = 0, tot = 0;
        CK(cudaMemGetInfo(&fr, &tot));
        const long long need = 28LL * tr + (!host  ? 24LL * tsg
                                            : chords ? 16LL * tsg + 8LL * (nslots + 1) * maxc
                                                     : 24LL * (nslots + 1) * maxc);
        if ((unsigned long long)need > fr)
            return fail(RT3D_ENOMEM,
                        "spherical cache of %lld rays and %lld segments needs %lld device bytes, "
                        "%zu free (build scratch %lld bytes for %d angles at a time)",
                        tr, tsg, need, fr, g->dev_bytes, chunk);
        if (host) {
            const long long hneed = (chords ? 8LL : 24LL) * tsg, havail = host_memory_available();
            if (havail >= 0 && hneed > havail / 2)
                return fail(RT3D_ENOMEM,
                            "host records of %lld segments need %lld bytes, more than half of "
                            "the %lld bytes of host memory available",
                            tsg, hneed, havail);
        }
    }
    long long *d_rbase = nullptr, *d_sbase = nullptr;
    TRY(g->alloc(&d_rbase, nO));
    TRY(g->alloc(&d_sbase, nO));
    CK(cudaMemcpyAsync(d_rbase, rbase.data(), sizeof(long long) * nO, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_sbase, sloc.data(), sizeof(long long) * nO, cudaMemcpyHostToDevice, s));
    TRY(g->alloc(&g->s_ray_off, tr));
    TRY(g->alloc(&g->s_ray_len, tr));
    TRY(g->alloc(&g->s_ray_angle, tr));
    TRY(g->alloc(&g->s_ray_launch, tr));
    TRY(g->alloc(&g->s_ray_kind, tr));
    TRY(g->alloc(&g->s_ray_face, tr));
    // host modes: pass 2 writes groups of consecutive residency chunks into a
    // transient staging buffer (at most 16 GiB or a quarter of the free
    // memory, at least the largest chunk), so that its launches keep the
    // device full, with segment offsets relative to the group; each group is
    // copied to the host records and the ray offsets are moved to their
    // chunk's origin at the end
    std::vector<int> grp(1, 0);  // residency chunks [grp[i], grp[i+1]) form group i
    float4 *stage_rec = nullptr;
    double *stage_len64 = nullptr;
    long long stage_seg = 0;
    long long *d_shift = nullptr;
    if (host) {
        if (chords) TRY(g->alloc(&g->s_rec, tsg));
        else TRY(g->alloc_host(&g->h_rec, &g->s_rec, tsg));
        TRY(g->alloc_host(&g->h_len64, &g->s_len64, tsg));
        for (int k = 0; k < nslots; ++k) {
            if (!chords) TRY(g->alloc(&g->slot_rec[k], maxc));
            TRY(g->alloc(&g->slot_len64[k], maxc));
        }
        size_t fr = 0, tot = 0;
        CK(cudaMemGetInfo(&fr, &tot));
        stage_seg = std::max(maxc, std::min(tsg, std::min<long long>(16LL << 30, (long long)(fr / 4)) / 24));
        for (int c = 0; c < nch; ++c)
            if (g->c_seg[c + 1] - g->c_seg[grp.back()] > stage_seg) grp.push_back(c);
        grp.push_back(nch);
        std::vector<long long> shift(nO);
        for (size_t i = 0; i + 1 < grp.size(); ++i)
            for (int c = grp[i]; c < grp[i + 1]; ++c)
                for (int o = g->c_angle[c]; o < g->c_angle[c + 1]; ++o) {
                    sloc[o] = sbase[o] - g->c_seg[grp[i]];
                    shift[o] = g->c_seg[c] - g->c_seg[grp[i]];
                }
        TRY(g->alloc(&stage_rec, stage_seg));
        TRY(g->alloc(&stage_len64, stage_seg));
        TRY(g->alloc(&d_shift, nO));
        CK(cudaMemcpyAsync(d_shift, shift.data(), sizeof(long long) * nO, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_sbase, sloc.data(), sizeof(long long) * nO, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));  // shift and sloc leave scope before the copies run otherwise
    } else {
        TRY(g->alloc(&g->s_rec, tsg));
        TRY(g->alloc(&g->s_len64, tsg));
        grp.push_back(nch);
    }
    bp.pass = 2;
    bp.ray_base = d_rbase;
    bp.seg_base = d_sbase;
    bp.ray_off = g->s_ray_off;
    bp.ray_len = g->s_ray_len;
    bp.ray_angle = g->s_ray_angle;
    bp.ray_launch = g->s_ray_launch;
    bp.ray_kind = g->s_ray_kind;
    bp.ray_face = g->s_ray_face;
    bp.rec = host ? stage_rec : g->s_rec;
    bp.len64 = host ? stage_len64 : g->s_len64;
    for (size_t i = 0; i + 1 < grp.size(); ++i) {
        const int a0 = g->c_angle[grp[i]], a1 = g->c_angle[grp[i + 1]];
        for (int o0 = a0; o0 < a1; o0 += chunk) {
            bp.o0 = o0;
            bp.nchunk = std::min(chunk, a1 - o0);
            CK(launch_sph_build(bp, s));
        }
        if (host) {
            // in stream order: the next group's build waits for this copy
            const long long g0 = g->c_seg[grp[i]], ns = g->c_seg[grp[i + 1]] - g0;
            if (chords)
                CK(cudaMemcpyAsync(g->s_rec + g0, stage_rec, sizeof(float4) * ns,
                                   cudaMemcpyDeviceToDevice, s));
            else
                CK(cudaMemcpyAsync(g->h_rec + g0, stage_rec, sizeof(float4) * ns,
                                   cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(g->h_len64 + g0, stage_len64, sizeof(double) * ns,
                               cudaMemcpyDeviceToHost, s));
        }
    }
    if (host) CKL(launch_rebase_ray_off(g->s_ray_off, g->s_ray_angle, d_shift, tr, s));
    CK(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (herr == 3) return fail(RT3D_EINVAL, "a Lambda* window exceeds 9 points");
    if (herr == 5) return fail(RT3D_EINVAL, "a cell is not crossed by some solid angle");
    if (herr) return fail(RT3D_EINVAL, "spherical tracer error %d", herr);
    g->segments = tsg;
    g->tpl.kmax = bp.ncap;
    if (tr > (long long)INT32_MAX) return fail(RT3D_EINVAL, "too many spherical rays");
    // the build scratch (and the mapped mode's build buffer) is not needed again
    g->release(hit, (size_t)chunk * words);
    g->release(tbuf, (size_t)chunk * bp.ncap);
    g->release(den, (size_t)chunk * N);
    g->release(d_nrays, nO);
    g->release(d_nseg, nO);
    g->release(d_err, 1);
    g->release(d_rbase, nO);
    g->release(d_sbase, nO);
    g->s_dir = d_dir;  // kept for the diffusion boundary's entry cosines
    g->s_rc_h = rc;
    g->release(d_wt, g->wt.size());
    g->release(stage_rec, (size_t)stage_seg);
    g->release(stage_len64, (size_t)stage_seg);
    g->release(d_shift, nO);
    if (host) {
        CK(cudaStreamCreateWithFlags(&g->cstream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&g->c_fork, cudaEventDisableTiming));
        for (int k = 0; k < 2; ++k) {
            CK(cudaEventCreateWithFlags(&g->c_copied[k], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&g->c_free[k], cudaEventDisableTiming));
            CK(cudaEventRecord(g->c_free[k], s));
        }
    }
    return alloc_work(g);
}

rt3d_status validate_desc(const rt3d_grid_desc *d) {
    if (!d) return fail(RT3D_EINVAL, "desc is NULL");
    if (d->geometry != RT3D_CARTESIAN_PERIODIC_XY && d->geometry != RT3D_SPHERICAL)
        return fail(RT3D_EINVAL, "geometry %d is not supported", d->geometry);
    if (d->geometry == RT3D_SPHERICAL) {
        if (d->n[0] < 1 || d->n[1] < 2 || d->n[2] < 4 || d->n[0] > 4096 || d->n[1] > 4096 ||
            d->n[2] > 4096)
            return fail(RT3D_EINVAL, "spherical grid %d x %d x %d: need nr >= 1, ntheta >= 2, "
                                     "nphi >= 4", d->n[0], d->n[1], d->n[2]);
        if (!(d->r_in > 0.0) || !(d->r_out > d->r_in))
            return fail(RT3D_EINVAL, "spherical grid needs 0 < r_in < r_out");
    } else if (d->n[0] < 4 || d->n[0] > 2047 || d->n[1] < 4 || d->n[1] > 2047 || d->n[2] < 1 ||
               d->n[2] > 1023) {
        return fail(RT3D_EINVAL, "grid %d x %d x %d outside 4..2047 x 4..2047 x 1..1023",
                    d->n[0], d->n[1], d->n[2]);
    }
    if (4LL * d->n[0] * d->n[1] * d->n[2] >= (1LL << 31))
        return fail(RT3D_EINVAL, "grid too large: 4 nx ny nz must stay below 2^31");
    if (d->ntheta < 1 || d->nphi < 1 || (long long)d->ntheta * d->nphi > 65535)
        return fail(RT3D_EINVAL, "bad angle grid %d x %d", d->ntheta, d->nphi);
    if (d->interp != RT3D_LINEAR && d->interp != RT3D_PARABOLIC)
        return fail(RT3D_EINVAL, "bad interp %d", d->interp);
    if (d->precision != RT3D_FP64 && d->precision != RT3D_FP32_FS_FP64_ALI &&
        d->precision != RT3D_FP32_FS_FF_REFINE)
        return fail(RT3D_EINVAL, "bad precision %d", d->precision);
    if (d->nlambda > 1) return fail(RT3D_EINVAL, "nlambda > 1 is not supported by this call");
    if (d->accel != RT3D_ACCEL_NONE && d->accel != RT3D_ACCEL_KRYLOV)
        return fail(RT3D_EINVAL, "bad accel %d", d->accel);
    if (d->cache != RT3D_CACHE_DEVICE && d->cache != RT3D_CACHE_HOST_STREAMED &&
        d->cache != RT3D_CACHE_HOST_MAPPED && d->cache != RT3D_CACHE_HOST_CHORDS)
        return fail(RT3D_EINVAL, "bad cache mode %d", d->cache);
    if (d->cache != RT3D_CACHE_DEVICE && d->geometry != RT3D_SPHERICAL)
        return fail(RT3D_EINVAL, "a host-resident cache needs the spherical grid");
    if (d->stream_bytes < 0) return fail(RT3D_EINVAL, "negative stream_bytes");
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
    g->ff_refine = d.precision == RT3D_FP32_FS_FF_REFINE;
    g->parab = d.interp == RT3D_PARABOLIC;
    g->a64 = g->fs64;
    g->sph = d.geometry == RT3D_SPHERICAL;
    g->cache = d.cache;
    if (g->sph) g->per = Periodic{false, false, true};

    // Direction set in FP64 on the host (midpoints in mu and phi, Sec. 3.1).
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
            if (!g->sph && !(std::fabs(m) > 0.0))
                return fail(RT3D_EINVAL, "direction %d has mu = 0 (use an even ntheta)", o);
        }
    }
    if (g->sph) return sph_build(g);
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
    TRY(g->alloc(&t.mu, nO));
    TRY(g->alloc(&t.code, total));
    TRY(g->alloc(&t.len64, total));
    TRY(g->alloc(&t.len32, total));
    TRY(g->alloc(&t.cw64, total));
    TRY(g->alloc(&t.cw32, total));
    TRY(g->alloc(&t.win, total));
    TRY(g->alloc(&t.rec32, total));
    TRY(g->alloc(&t.rec64, total));
    const bool quad = !g->fs64 && 4LL * g->nx * g->ny * g->nz <= (1LL << 29) - 1;
    if (quad) TRY(g->alloc(&t.rec4, total));
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
    CK(cudaMemcpyAsync(t.mu, g->mu.data(), sizeof(double) * nO, cudaMemcpyHostToDevice, s));
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
    tp.rec32 = t.rec32;
    tp.rec64 = t.rec64;
    tp.layer_sum = d_ls;
    tp.err = d_err;
    CK(launch_trace(tp, s));
    if (quad) CK(launch_quad_rec(t, g->nx, g->ny, t.rec4, s));
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

    return alloc_work(g);
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
    CKL(launch_pack(g->nx, g->ny, g->nz, g->chi, 1.0, g->chi /*S placeholder*/, g->chiS32, false, g->stream));
    CKL(launch_pack(g->nx, g->ny, g->nz, g->chi, 1.0, g->chi, g->chiS64, true, g->stream));
    return RT3D_OK;
}

// One ALI iteration on the grid's state (g->J): S from J, FS of the grid's
// FS precision (fp64 flag), Lambda* if not valid, Jacobi, J += dJ.
rt3d_status ali_iteration(rt3d_grid *g, const FsParams &fp, bool fp64, int max_sweeps,
                          double sweep_tol, double *rel) {
    const int N = (int)g->N;
    CKL(launch_source(g->nx, g->ny, g->nz, g->J, g->eps, g->B, fp64 ? g->chiS64 : g->chiS32, fp64, false, g->stream));
    const bool build = !g->lstar_valid;
    TRY(run_fs(g, fp, fp64, build));
    if (build) {
        CKL(launch_os_prep(g->nx, g->ny, g->nz, g->lstar, g->eps, g->a, g->a64, g->inv_diag,
                          g->stream, g->per, g->os_kind == kOsGaussSeidel, g->diag));
        CK(cudaMemcpyAsync(g->chi_ref, g->chi, sizeof(double) * N, cudaMemcpyDeviceToDevice,
                           g->stream));
        CK(cudaMemcpyAsync(g->eps_ref, g->eps, sizeof(double) * N, cudaMemcpyDeviceToDevice,
                           g->stream));
        g->lstar_valid = true;
    }
    TRY(os_solve_dev(g, g->Jfs, g->J, nullptr, os_cap(g, max_sweeps), sweep_tol));
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
    CKL(launch_source(g->nx, g->ny, g->nz, v, g->eps, nullptr, fp64 ? g->chiS64 : g->chiS32, fp64, true, g->stream));
    TRY(run_fs(g, fphom, fp64, false));
    CKL(launch_sub(n, v, g->Jfs, out, g->stream));
    return RT3D_OK;
}

#ifndef RT3D_PRECOND_SWEEPS
#define RT3D_PRECOND_SWEEPS 50
#endif
#ifndef RT3D_PRECOND_TOL
#define RT3D_PRECOND_TOL 1e-3
#endif

// z = M^-1 v by Jacobi sweeps (the OS solve of Eq. alo): at most
// RT3D_PRECOND_SWEEPS sweeps, stopped at a change of RT3D_PRECOND_TOL relative
// to the iterate (the paper's OS solve; the same settings as the ALI step)
rt3d_status precond(rt3d_grid *g, const double *v, double *z) {
    TRY(os_solve_dev(g, nullptr, nullptr, v, os_cap(g, RT3D_PRECOND_SWEEPS), RT3D_PRECOND_TOL));
    CKL(launch_copy_buf((int)g->N, g->dJ_dev, g->st, z, g->stream));
    return RT3D_OK;
}

// One FGMRES cycle (right preconditioning, classical Gram-Schmidt applied
// twice) for A x = r from x = 0. Stops when the residual estimate falls to
// eta |r| or after kKrylov steps. Returns the achieved reduction and the
// number of operator applications. (Scaling the system by diag|J|, so that
// the 2-norm weighs residuals relative to J, was measured to need more
// formal solutions on the 129^3 field workload, 253 against 167.)
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

#ifndef RT3D_KRYLOV_ETA
#define RT3D_KRYLOV_ETA 1e-5
#endif
#ifndef RT3D_KRYLOV_ETA0
#define RT3D_KRYLOV_ETA0 RT3D_KRYLOV_ETA
#endif

// Krylov-accelerated solve with iterative refinement. A round: residual
// r = J_FS(S(J)) - J of the current J, then (unless it certifies J) one
// FGMRES cycle on A delta = r with A in the grid's FS precision, J += delta.
// Residuals: FP32 before the first converged cycle in the mixed modes, then
// FP64; with float-float refinement (RT3D_FP32_FS_FF_REFINE) from the
// float-float formal solution, and an FP64 one only when the float-float
// estimate meets tol. The error after a round is estimated as gain * (next
// residual), gain = |delta|/|r| of the previous round; only an FP64 residual
// that meets tol certifies J.
rt3d_status krylov_solve(rt3d_grid *g, const FsParams &fp, const FsParams &fp64p,
                         const FsParams &fphom, double tol, int max_iter, rt3d_solve_stats &s,
                         bool *conv_out) {
    const int n = (int)g->N;
    const bool mixed = !g->fs64;
    bool res64 = !mixed;
    bool conv = false;
    double gain = -1.0, est = 1.0, res = 0.0;
    int it = 0, rounds32 = 0;
    // Reduction asked of one FGMRES cycle (eta0 for the cycle on the FP32
    // residual of the starting J). An FP64 formal solution costs about 40
    // FP32 ones on this GPU, so every cycle is driven deep (the FP32
    // operator's rounding still allows that) to keep the number of FP64
    // residuals of the refinement at two or three; a cycle whose estimated
    // error is already near tol is asked only for the reduction it needs,
    // with a margin of 100: eta = max(RT3D_KRYLOV_ETA, min(0.1, 0.01 tol/est)).
    const double eta = RT3D_KRYLOV_ETA, eta0 = RT3D_KRYLOV_ETA0;
    // residual kinds: 0 FP32, 1 FP64, 2 float-float
    auto residual = [&](int kind, double *res_out) -> rt3d_status {
        const bool build = !g->lstar_valid;
        if (kind == 2) {
            TRY(run_fs_ff(g, fp64p, g->chi, g->J, g->eps, g->B));
            ++s.fs_ff;
        } else {
            const bool f64 = kind == 1;
            CKL(launch_source(g->nx, g->ny, g->nz, g->J, g->eps, g->B, f64 ? g->chiS64 : g->chiS32,
                              f64, false, g->stream));
            TRY(run_fs(g, f64 ? fp64p : fp, f64, build));
            if (f64) ++s.fs_fp64;
            else ++s.fs_fp32;
            if (build) {
                CKL(launch_os_prep(g->nx, g->ny, g->nz, g->lstar, g->eps, g->a, g->a64, g->inv_diag,
                                   g->stream, g->per, g->os_kind == kOsGaussSeidel, g->diag));
                CK(cudaMemcpyAsync(g->chi_ref, g->chi, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                                   g->stream));
                CK(cudaMemcpyAsync(g->eps_ref, g->eps, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                                   g->stream));
                g->lstar_valid = true;
            }
        }
        TRY(reset_scalar(g, offsetof(OsState, res), sizeof(unsigned long long)));
        CKL(launch_residual(n, g->Jfs, g->J, g->r64, g->st, g->stream));
        TRY(read_scalar_d(g, offsetof(OsState, res), res_out));
        if (!(*res_out == *res_out)) return fail(RT3D_ENUMERIC, "NaN in the residual");
        return RT3D_OK;
    };
    auto record = [&](int kind, double r, double e) {
        const int ri = s.rounds < 16 ? s.rounds : -1;
        ++s.rounds;
        if (ri >= 0) {
            s.round_fp64[ri] = kind;
            s.round_res[ri] = r;
            s.round_est[ri] = e;
            s.round_fs[ri] = 0;
        }
        return ri;
    };
    // Float-float residuals are accurate to about 1e-12 of J; where the
    // problem amplifies that floor above tol (eps near 1e-8 in optically
    // thick media) a float-float residual stops falling between rounds, and
    // the refinement then takes its residuals from the FP64 formal solution.
    bool ff_ok = true;
    double res_ff_prev = -1.0;
    for (int round = 0; round < 60 && it < max_iter; ++round) {
        // the first residual also builds Lambda* (FP32 or FP64 kind)
        int kind = res64 ? ((g->ff_refine && ff_ok && g->lstar_valid) ? 2 : 1) : 0;
        TRY(residual(kind, &res));
        // gain < 0: unknown (first round, or a residual relative to J = 0)
        est = (kind != 0 && gain >= 0.0) ? gain * res : -1.0;
        int ri = record(kind, res, est);
        if (kind == 2) {
            const bool stalled = res_ff_prev > 0.0 && res > 0.1 * res_ff_prev;
            res_ff_prev = res;
            if (stalled && !(est >= 0.0 && est <= tol)) {
                ff_ok = false;  // this and later rounds: FP64 residuals
                kind = 1;
                TRY(residual(1, &res));
                est = gain >= 0.0 ? gain * res : -1.0;
                ri = record(1, res, est);
            }
        }
        if (kind == 2 && est >= 0.0 && est <= tol) {
            // float-float estimate met: the FP64 formal solution decides
            kind = 1;
            TRY(residual(1, &res));
            est = gain * res;
            ri = record(1, res, est);
        }
        if (kind == 1) s.residual64 = res;
        if (kind == 1 && est >= 0.0 && est <= tol) {
            conv = true;
            break;
        }
        double eta_k = res64 ? eta : eta0;
        if (est > tol) eta_k = std::max(eta_k, std::min(0.1, 0.01 * tol / est));
        double achieved = 0.0;
        int steps = 0;
        TRY(fgmres(g, fphom, g->fs64, g->r64, g->delta, eta_k, max_iter - it, &achieved, &steps));
        if (ri >= 0) s.round_fs[ri] = steps;
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

// Batched workspace for nl wavelengths (grows; never shrinks).
rt3d_status batch_setup(rt3d_grid *g, int nl) {
    if (g->bl_cap >= nl) return RT3D_OK;
    const size_t N = (size_t)g->N, nf = (size_t)g->nx * g->ny, L = (size_t)nl;
    TRY(g->alloc(&g->bchi, L * N));
    TRY(g->alloc(&g->beps, L * N));
    TRY(g->alloc(&g->bB, L * N));
    TRY(g->alloc(&g->bJ, L * N));
    TRY(g->alloc(&g->br, L * N));
    TRY(g->alloc(&g->bbuf0, L * N));
    TRY(g->alloc(&g->bbuf1, L * N));
    TRY(g->alloc(&g->bb32_0, L * N));
    TRY(g->alloc(&g->bb32_1, L * N));
    TRY(g->alloc(&g->binv, L * N));
    TRY(g->alloc(&g->bJrep, 4 * L * N));
    TRY(g->alloc(&g->bchiS, 4 * L * N));
    TRY(g->alloc(&g->ba, L * os_coef_count((long long)N)));
    TRY(g->alloc(&g->btop, L * nf));
    TRY(g->alloc(&g->bbot, L * nf));
    TRY(g->alloc(&g->bgrad, L * nf));
    BatchState &b = g->bsh;
    TRY(g->alloc(&b.active, L));
    TRY(g->alloc(&b.alist, L));
    TRY(g->alloc(&b.state, L));
    TRY(g->alloc(&b.done, L));
    TRY(g->alloc(&b.count, L));
    TRY(g->alloc(&b.iters, L));
    TRY(g->alloc(&b.dmax, L * (kBatchSweeps + 1)));
    TRY(g->alloc(&b.jmax, L * (kBatchSweeps + 1)));
    TRY(g->alloc(&b.rel, L));
    TRY(g->alloc(&b.hist, L * kHist));
    TRY(g->alloc(&b.est, L));
    b.nactive = 0;
    TRY(g->alloc(&g->bsd, 1));
    if (!g->bstream) {
        CK(cudaStreamCreateWithFlags(&g->bstream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&g->bev0, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&g->bev1, cudaEventDisableTiming));
    }
    g->bl_cap = nl;
    return RT3D_OK;
}

// Line-transfer workspace (allocated on first use; the weight buffer grows to
// the largest nl seen, the smaller one staying allocated until destroy) and
// the upload of the negated weights -wphi[l].
rt3d_status line_setup(rt3d_grid *g, const std::vector<double> &negw) {
    const size_t N = (size_t)g->N;
    const int nl = (int)negw.size();
    if (!g->lbar) {
        TRY(g->alloc(&g->lbar, 27 * N));
        TRY(g->alloc(&g->jbar_fs, N));
        TRY(g->alloc(&g->lptr, 28));
        std::vector<double *> tab(28);
        tab[0] = g->Jfs;
        for (int d = 0; d < 27; ++d) tab[1 + d] = g->lstar + (size_t)d * N;
        CK(cudaMemcpyAsync(g->lptr, tab.data(), sizeof(double *) * 28, cudaMemcpyHostToDevice,
                           g->stream));
        CK(cudaStreamSynchronize(g->stream));  // tab is host memory of this frame
    }
    if (nl > g->lcoef_cap) {
        TRY(g->alloc(&g->lcoef, (size_t)nl));
        g->lcoef_cap = nl;
    }
    CK(cudaMemcpyAsync(g->lcoef, negw.data(), sizeof(double) * nl, cudaMemcpyHostToDevice,
                       g->stream));
    CK(cudaStreamSynchronize(g->stream));  // negw is the caller's host vector
    return RT3D_OK;
}

// One ALI iteration of the line problem on g->J (= Jbar): for every
// wavelength l, (chi scale[l], S) packed with S = (1 - eps) Jbar + eps B, its
// FP64 formal solution added into jbar_fs with weight wphi[l] (and, when
// build, its Lambda* band into lbar); then the OS solve with the averaged band
// and Jbar += dJ. *rel = max |dJ| / |Jbar_new|.
// Jbar_FS = sum_l wphi[l] J_FS,l of the source S = (1 - eps) x + eps B
// (homogeneous: (1 - eps) x, with fp a homogeneous parameter set) into
// g->jbar_fs; with build also Lbar* = sum_l wphi[l] Lambda*_l into g->lbar.
rt3d_status line_fs(rt3d_grid *g, const FsParams &fp, bool fp64, const std::vector<double> &scale,
                    const double *x, bool homogeneous, bool build, int *fs_count) {
    const size_t N = (size_t)g->N;
    const int n = (int)N;
    void *chiS = fp64 ? (void *)g->chiS64 : (void *)g->chiS32;
    CK(cudaMemsetAsync(g->jbar_fs, 0, sizeof(double) * N, g->stream));
    if (build) CK(cudaMemsetAsync(g->lbar, 0, sizeof(double) * 27 * N, g->stream));
    for (int l = 0; l < (int)scale.size(); ++l) {
        CKL(launch_pack(g->nx, g->ny, g->nz, g->chi, scale[l], g->chi /*S placeholder*/, chiS,
                        fp64, g->stream));
        CKL(launch_source(g->nx, g->ny, g->nz, x, g->eps, homogeneous ? nullptr : g->B, chiS, fp64,
                          homogeneous, g->stream));
        TRY(run_fs(g, fp, fp64, build));
        ++*fs_count;
        // jbar_fs -= (-wphi[l]) Jfs
        CKL(launch_multi_axpy(n, g->jbar_fs, g->lptr, g->lcoef + l, 1, g->stream));
        if (build)
            for (int d = 0; d < 27; ++d)
                CKL(launch_multi_axpy(n, g->lbar + (size_t)d * N, g->lptr + 1 + d, g->lcoef + l,
                                      1, g->stream));
    }
    return RT3D_OK;
}

rt3d_status line_iteration(rt3d_grid *g, const FsParams &fp, bool fp64,
                           const std::vector<double> &scale, bool build, double *rel,
                           int *fs_count) {
    const int n = (int)g->N;
    TRY(line_fs(g, fp, fp64, scale, g->J, false, build, fs_count));
    if (build)
        CKL(launch_os_prep(g->nx, g->ny, g->nz, g->lbar, g->eps, g->a, g->a64, g->inv_diag,
                           g->stream, g->per, g->os_kind == kOsGaussSeidel, g->diag));
    TRY(os_solve_dev(g, g->jbar_fs, g->J, nullptr, os_cap(g, 50), 1e-3));
    TRY(reset_scalar(g, offsetof(OsState, rel), sizeof(unsigned long long)));
    CKL(launch_ali_update(n, g->J, g->dJ_dev, g->st, nullptr, g->stream));
    TRY(read_scalar_d(g, offsetof(OsState, rel), rel));
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
    info->fs_shape.block = g->fs_shape.block;
    info->fs_shape.rays_per_thread = g->fs_shape.rays_per_thread;
    info->fs_shape.widen = g->fs_shape.widen;
    info->fs_shape.branchless = g->fs_shape.branchless;
    for (int i = 0; i < RT3D_FS_TUNE_SHAPES; ++i) info->fs_tune_ms[i] = g->fs_tune_ms[i];
    info->sm_count = device_sm_count();
    info->cache = g->cache;
    info->host_bytes = g->host_bytes;
    info->cache_chunks = g->sph ? (int)g->c_angle.size() - 1 : 1;
    return RT3D_OK;
}

rt3d_status rt3d_grid_set_os_solver(rt3d_grid *g, int solver) {
    if (!g) return fail(RT3D_EINVAL, "NULL grid");
    if (solver != RT3D_OS_JACOBI && solver != RT3D_OS_GAUSS_SEIDEL && solver != RT3D_OS_BICGSTAB)
        return fail(RT3D_EINVAL, "OS solver %d not available", solver);
    const int old = g->os_kind;
    g->os_kind = solver == RT3D_OS_GAUSS_SEIDEL ? kOsGaussSeidel
                 : solver == RT3D_OS_BICGSTAB   ? kOsBicgstab
                                                : kOsJacobi;
    // a band in use keeps working: its coefficients in the new solver's layout
    if (g->lstar_valid && (old == kOsGaussSeidel) != (g->os_kind == kOsGaussSeidel)) {
        CKL(launch_os_prep(g->nx, g->ny, g->nz, g->lstar, g->eps, g->a, g->a64, g->inv_diag,
                           g->stream, g->per, g->os_kind == kOsGaussSeidel, g->diag));
        CK(cudaStreamSynchronize(g->stream));
    }
    return RT3D_OK;
}

rt3d_status rt3d_grid_invalidate_lstar(rt3d_grid *g) {
    if (!g) return fail(RT3D_EINVAL, "NULL grid");
    g->lstar_valid = false;
    return RT3D_OK;
}

rt3d_status rt3d_fs_tune_shape(int i, rt3d_fs_shape *out) {
    if (!out || i < 0 || i >= RT3D_FS_TUNE_SHAPES) return fail(RT3D_EINVAL, "bad candidate index or NULL");
    out->block = kFsShapes[i].block;
    out->rays_per_thread = kFsShapes[i].rays_per_thread;
    out->widen = kFsShapes[i].widen;
    out->branchless = kFsShapes[i].branchless;
    return RT3D_OK;
}

rt3d_status rt3d_grid_set_fs_shape(rt3d_grid *g, const rt3d_fs_shape *shape) {
    if (!g) return fail(RT3D_EINVAL, "NULL grid");
    if (!shape) {
        g->fs_shape = FsShape{0, 0, 0, 0};
        return RT3D_OK;
    }
    const FsShape sh{shape->block, shape->rays_per_thread, shape->widen, shape->branchless};
    if (!fs_shape_valid(sh))
        return fail(RT3D_EINVAL, "shape (%d, %d, %d, %d) not available", sh.block, sh.rays_per_thread,
                    sh.widen, sh.branchless);
    if (sh.rays_per_thread == 4 && !g->tpl.rec4)
        return fail(RT3D_EINVAL, "four characteristics per thread need an FP32 Cartesian grid of "
                                 "at most 2^27 voxels");
    g->fs_shape = sh;
    return RT3D_OK;
}

rt3d_status rt3d_grid_sph_ray(const rt3d_grid *gc, int angle, int index, int *K, int32_t *vox,
                              double *len, int *launch, int *kind) {
    rt3d_grid *g = const_cast<rt3d_grid *>(gc);
    if (!g || !K) return fail(RT3D_EINVAL, "NULL argument");
    if (!g->sph) return fail(RT3D_EINVAL, "not a spherical grid");
    if (angle < 0 || angle >= g->nO) return fail(RT3D_EINVAL, "angle %d out of range", angle);
    if (index < 0 || index >= g->s_nrays_angle[angle])
        return fail(RT3D_EINVAL, "ray %d out of range", index);
    const long long r = g->s_ray_base[angle] + index;
    long long off = 0;
    int k = 0, ln = 0, kd = 0;
    CK(cudaMemcpyAsync(&off, g->s_ray_off + r, sizeof off, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(&k, g->s_ray_len + r, sizeof k, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(&ln, g->s_ray_launch + r, sizeof ln, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(&kd, g->s_ray_kind + r, sizeof kd, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (*K < k) {
        *K = k;
        return fail(RT3D_EINVAL, "capacity below %d points", k);
    }
    *K = k;
    std::vector<float4> rec(vox ? k : 0);
    if (g->cache != RT3D_CACHE_DEVICE) {
        // host records (or chords); the offset is relative to the angle's chunk
        off += g->s_angle_chunk_seg[angle];
        if (vox && g->h_rec) std::memcpy(rec.data(), g->h_rec + off, sizeof(float4) * k);
        if (vox && !g->h_rec) {
            CK(cudaMemcpyAsync(rec.data(), g->s_rec + off, sizeof(float4) * k,
                               cudaMemcpyDeviceToHost, g->stream));
            CK(cudaStreamSynchronize(g->stream));
        }
        if (len) std::memcpy(len, g->h_len64 + off, sizeof(double) * k);
    } else {
        if (vox) CK(cudaMemcpyAsync(rec.data(), g->s_rec + off, sizeof(float4) * k, cudaMemcpyDeviceToHost, g->stream));
        if (len) CK(cudaMemcpyAsync(len, g->s_len64 + off, sizeof(double) * k, cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
    }
    for (int i = 0; vox && i < k; ++i) {
        int rep;
        std::memcpy(&rep, &rec[i].x, sizeof rep);
        vox[i] = sph_cell_of_rep(rep, g->nx, g->ny);
    }
    if (launch) *launch = ln;
    if (kind) *kind = kd;
    return RT3D_OK;
}

rt3d_status rt3d_grid_template(const rt3d_grid *gc, int angle, int *K, int32_t *vox,
                               double *len) {
    rt3d_grid *g = const_cast<rt3d_grid *>(gc);
    if (!g || !K) return fail(RT3D_EINVAL, "NULL argument");
    if (g->sph) return fail(RT3D_EINVAL, "spherical grids have no per-angle template");
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
    CKL(launch_pack(g->nx, g->ny, g->nz, dchi, 1.0, dS, g->fs64 ? g->chiS64 : g->chiS32, g->fs64, g->stream));
    FsParams fp;
    TRY(fs_params(g, bc, g->fs64, false, &fp));
    TRY(run_fs(g, fp, g->fs64, lstar_out != nullptr));
    TRY(deliver(g, J_out, g->Jfs, N));
    if (lstar_out) TRY(deliver(g, lstar_out, g->lstar, 27 * N));
    CK(cudaStreamSynchronize(g->stream));
    return RT3D_OK;
}

rt3d_status rt3d_formal_solution_ff(rt3d_grid *g, const double *chi, const double *S,
                                    const rt3d_bc *bc, double *J_out) {
    if (!g || !chi || !S || !J_out) return fail(RT3D_EINVAL, "NULL argument");
    const size_t N = (size_t)g->N;
    const double *dchi = nullptr, *dS = nullptr;
    TRY(stage_in(g, chi, N, g->chi, &dchi));
    TRY(stage_in(g, S, N, g->S, &dS));
    FsParams fp;
    TRY(fs_params(g, bc, false, false, &fp));
    TRY(run_fs_ff(g, fp, dchi, dS, nullptr, nullptr));
    TRY(deliver(g, J_out, g->Jfs, N));
    CK(cudaStreamSynchronize(g->stream));
    return RT3D_OK;
}

rt3d_status rt3d_diffusion_bc(rt3d_grid *g, int nl, const double *chi, const double *B,
                              double *I_face, double *grad) {
    if (!g || !chi || !B || !I_face || !grad) return fail(RT3D_EINVAL, "NULL argument");
    if (nl < 1) return fail(RT3D_EINVAL, "nlambda %d < 1", nl);
    if (!is_device_ptr(chi) || !is_device_ptr(B) || !is_device_ptr(I_face) || !is_device_ptr(grad))
        return fail(RT3D_EINVAL, "chi, B, I_face and grad must be memory of the grid's device");
    if (g->sph) {
        const double rc0 = g->s_rc_h[0], rc1 = g->nx > 1 ? g->s_rc_h[1] : rc0;
        CKL(launch_sph_diffusion_bc(g->nx, g->ny, g->nz, nl, rc0, rc1, g->desc.r_in, chi, B,
                                    I_face, grad, g->stream));
        return RT3D_OK;
    }
    CKL(launch_diffusion_bc(g->nx, g->ny, g->nz, nl, chi, B, I_face, grad, g->stream));
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
    CKL(launch_os_prep(g->nx, g->ny, g->nz, g->lstar, g->eps, g->a, g->a64, g->inv_diag, g->stream,
                        g->per, g->os_kind == kOsGaussSeidel, g->diag));
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
    g->fs_ms[0] = g->fs_ms[1] = g->fs_ms[2] = g->fs_ms[3] = 0.0;
    g->fs_lstar32 = 0;
    g->launches = 0;
    TRY(reset_scalar(g, offsetof(OsState, sweeps_total), sizeof(unsigned long long)));
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
        s.fs32_ms = g->fs_ms[0] + g->fs_ms[3];
        s.fs32_lstar_ms = g->fs_ms[3];
        s.fs_lstar = g->fs_lstar32;
        s.fs64_ms = g->fs_ms[1];
        s.fsff_ms = g->fs_ms[2];
        {
            unsigned long long sw = 0;
            CK(cudaMemcpyAsync(&sw, &g->st->sweeps_total, sizeof sw, cudaMemcpyDeviceToHost, g->stream));
            CK(cudaStreamSynchronize(g->stream));
            s.jacobi_sweeps = (int)std::min<unsigned long long>(sw, (unsigned long long)INT32_MAX);
        }
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
            CKL(launch_source(g->nx, g->ny, g->nz, g->J, g->eps, g->B, g->chiS64, true, false, g->stream));
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
            TRY(os_solve_dev(g, nullptr, nullptr, g->r64, os_cap(g, max_sweeps), sweep_tol));
            CKL(launch_copy_buf(n, g->dJ_dev, g->st, g->delta, g->stream));
            double drel = 1.0, dacc = 1.0;
            Progress dprog;
            const bool fs32 = mixed;
            for (int inner = 0; inner < 1000 && it < max_iter; ++inner) {
                CKL(launch_source(g->nx, g->ny, g->nz, g->delta, g->eps, nullptr, fs32 ? g->chiS32 : g->chiS64, !fs32,
                                  true, g->stream));
                TRY(run_fs(g, fphom, !fs32, false));
                if (fs32) ++s.fs_fp32;
                else ++s.fs_fp64;
                ++it;
                // r = Lambda_hom((1-eps) delta) + r64 - delta
                TRY(os_solve_dev(g, g->Jfs, g->delta, g->r64, os_cap(g, max_sweeps), sweep_tol));
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
        CKL(launch_source(g->nx, g->ny, g->nz, g->J, g->eps, g->B, g->chiS64, true, false, g->stream));
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
    s.fs32_ms = g->fs_ms[0] + g->fs_ms[3];
    s.fs32_lstar_ms = g->fs_ms[3];
    s.fs_lstar = g->fs_lstar32;
    s.fs64_ms = g->fs_ms[1];
    s.fsff_ms = g->fs_ms[2];
    {
        unsigned long long sw = 0;
        CK(cudaMemcpyAsync(&sw, &g->st->sweeps_total, sizeof sw, cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
        s.jacobi_sweeps = (int)std::min<unsigned long long>(sw, (unsigned long long)INT32_MAX);
    }
    s.launches = g->launches;
    s.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (stats) *stats = s;
    if (!conv) return fail(RT3D_ENOTCONVERGED, "not converged after %d iterations (est %.3g)", it, est);
    return RT3D_OK;
}

rt3d_status rt3d_line_solve(rt3d_grid *g, int nl, const double *chi, const double *scale,
                            const double *wphi, const double *eps, const double *B,
                            const rt3d_bc *bc, double *Jbar_inout, double tol, int max_iter,
                            rt3d_line_stats *stats) {
    const auto t_start = std::chrono::steady_clock::now();
    if (!g || !chi || !scale || !wphi || !eps || !B || !Jbar_inout)
        return fail(RT3D_EINVAL, "NULL argument");
    if (g->sph) return fail(RT3D_EINVAL, "line transfer needs the Cartesian grid");
    if (nl < 1 || nl > 65536) return fail(RT3D_EINVAL, "nlambda %d", nl);
    if (!(tol > 0.0) || max_iter < 1) return fail(RT3D_EINVAL, "bad tol or max_iter");
    if (ptr_kind(scale) != 0 || ptr_kind(wphi) != 0)
        return fail(RT3D_EINVAL, "scale and wphi must be host arrays");
    std::vector<double> sc(nl), negw(nl);
    double wsum = 0.0;
    for (int l = 0; l < nl; ++l) {
        if (!(scale[l] > 0.0) || !std::isfinite(scale[l]))
            return fail(RT3D_EINVAL, "scale[%d] = %g", l, scale[l]);
        if (!(wphi[l] >= 0.0) || !std::isfinite(wphi[l]))
            return fail(RT3D_EINVAL, "wphi[%d] = %g", l, wphi[l]);
        sc[l] = scale[l];
        negw[l] = -wphi[l];
        wsum += wphi[l];
    }
    if (!(wsum > 0.0)) return fail(RT3D_EINVAL, "the profile weights sum to zero");
    const size_t N = (size_t)g->N;
    rt3d_line_stats s{};
    s.est_error = -1.0;
    g->fs_ms[0] = g->fs_ms[1] = g->fs_ms[2] = g->fs_ms[3] = 0.0;
    g->fs_lstar32 = 0;
    g->launches = 0;
    TRY(reset_scalar(g, offsetof(OsState, sweeps_total), sizeof(unsigned long long)));
    TRY(line_setup(g, negw));
    g->lstar_valid = false;  // the grid's Lambda* and OS coefficients become the line's
    TRY(load_problem(g, chi, eps, B));
    CK(cudaMemcpyAsync(g->J, Jbar_inout, N * sizeof(double), cudaMemcpyDefault, g->stream));
    FsParams fp64p, fp32p, fphom;
    TRY(fs_params(g, bc, true, false, &fp64p));
    const bool mixed = !g->fs64;
    if (mixed) {
        TRY(fs_params(g, bc, false, false, &fp32p));
        TRY(fs_params(g, nullptr, false, true, &fphom));
    }
    // Phase 1: the line ALI, in FP32 formal solutions on the mixed grids
    // down to their rounding floor (estimate below 1e-6, or no decrease)
    Progress prog;
    double rel = 1.0;
    bool conv = false;
    int it = 0;
    const double switch_at = mixed ? std::max(tol, 1e-6) : tol;
    while (it < max_iter) {
        const int before = s.fs_lambda;
        TRY(line_iteration(g, mixed ? fp32p : fp64p, !mixed, sc, it == 0, &rel, &s.fs_lambda));
        if (mixed) s.fs_lambda32 += s.fs_lambda - before;
        ++it;
        if (!(rel == rel)) return fail(RT3D_ENUMERIC, "NaN in the line ALI change at iteration %d", it);
        prog.add(rel);
        if (it >= 2) {
            s.est_error = prog.error_estimate();
            if (s.est_error <= switch_at) {
                conv = !mixed;
                break;
            }
        }
        if (mixed && prog.stagnated()) break;
    }
    s.rel_change = rel;
    // Phase 2 (mixed grids), as the continuum solve's: defect correction with
    // FP64 residuals r64 = Jbar_FS64(S(Jbar)) - Jbar and corrections delta
    // from the homogeneous problem (1 - Lbar(1 - eps)) delta = r64 iterated
    // with FP32 formal solutions; the error after Jbar += delta is about
    // |delta| times delta's relative accuracy; a last FP64 residual
    // certifies the returned Jbar.
    const int n = (int)N;
    if (mixed && it < max_iter) {
        for (int round = 0; round < 8 && it < max_iter; ++round) {
            TRY(line_fs(g, fp64p, true, sc, g->J, false, false, &s.fs_lambda));
            TRY(reset_scalar(g, offsetof(OsState, res), sizeof(unsigned long long)));
            CKL(launch_residual(n, g->jbar_fs, g->J, g->r64, g->st, g->stream));
            double res = 0.0;
            TRY(read_scalar_d(g, offsetof(OsState, res), &res));
            s.residual64 = res;
            if (!(res == res)) return fail(RT3D_ENUMERIC, "NaN in the FP64 line residual");
            if (conv) break;  // that was the certification of the corrected Jbar
            // delta_0 = M^-1 r64, then the ALI on delta with homogeneous FP32
            // solutions, to the relative accuracy that brings the estimated
            // error (about |delta| times that accuracy) to half of tol
            TRY(os_solve_dev(g, nullptr, nullptr, g->r64, os_cap(g, 50), 1e-3));
            CKL(launch_copy_buf(n, g->dJ_dev, g->st, g->delta, g->stream));
            const double err_now = s.est_error > 0.0 ? s.est_error : 1.0;
            const double target = std::min(0.1, std::max(1e-4, 0.5 * tol / err_now));
            double drel = 1.0, dacc = 1.0;
            Progress dprog;
            for (int inner = 0; inner < 1000 && it < max_iter; ++inner) {
                const int before = s.fs_lambda;
                TRY(line_fs(g, fphom, false, sc, g->delta, true, false, &s.fs_lambda));
                s.fs_lambda32 += s.fs_lambda - before;
                ++it;
                // r = Lbar_hom((1 - eps) delta) + r64 - delta
                TRY(os_solve_dev(g, g->jbar_fs, g->delta, g->r64, os_cap(g, 50), 1e-3));
                TRY(reset_scalar(g, offsetof(OsState, rel), sizeof(unsigned long long)));
                CKL(launch_ali_update(n, g->delta, g->dJ_dev, g->st, nullptr, g->stream));
                TRY(read_scalar_d(g, offsetof(OsState, rel), &drel));
                if (!(drel == drel)) return fail(RT3D_ENUMERIC, "NaN in the line defect correction");
                dprog.add(drel);
                dacc = std::max(dprog.error_estimate(), drel);
                if (dacc <= target) break;
                if (dprog.stagnated()) break;
            }
            // Jbar += delta; size of the correction relative to Jbar
            TRY(reset_scalar(g, offsetof(OsState, rel), sizeof(unsigned long long)));
            CKL(launch_axpy_rel(n, g->J, g->delta, g->st, g->stream));
            double crel = 0.0;
            TRY(read_scalar_d(g, offsetof(OsState, rel), &crel));
            s.est_error = crel * dacc;
            s.rel_change = crel;
            if (s.est_error <= tol) conv = true;
        }
    }
    s.iterations = it;
    TRY(deliver(g, Jbar_inout, g->J, N));
    CK(cudaStreamSynchronize(g->stream));
    TRY(collect_events(g));
    s.fs64_ms = g->fs_ms[1];
    s.fs32_ms = g->fs_ms[0] + g->fs_ms[3];
    {
        unsigned long long sw = 0;
        CK(cudaMemcpyAsync(&sw, &g->st->sweeps_total, sizeof sw, cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
        s.jacobi_sweeps = (int)std::min<unsigned long long>(sw, (unsigned long long)INT32_MAX);
    }
    s.launches = g->launches;
    s.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (stats) *stats = s;
    if (!conv)
        return fail(RT3D_ENOTCONVERGED, "line ALI not converged after %d iterations (est %.3g)",
                    it, s.est_error);
    return RT3D_OK;
}


rt3d_status rt3d_solve_batched(rt3d_grid *g, int nl, const double *chi, const double *eps,
                               const double *B, const rt3d_bc *bc, double *J_inout, double tol,
                               int max_iter, int *status_out, rt3d_batch_stats *stats) {
    const auto t_start = std::chrono::steady_clock::now();
    if (!g || !chi || !eps || !B || !J_inout) return fail(RT3D_EINVAL, "NULL argument");
    if (nl < 1 || nl > 65535) return fail(RT3D_EINVAL, "n_lambda %d outside 1..65535", nl);
    if (g->sph) return fail(RT3D_EINVAL, "batched wavelengths need a Cartesian grid");
    if (!(tol > 0.0) || max_iter < 1) return fail(RT3D_EINVAL, "bad tol or max_iter");
    const size_t N = (size_t)g->N, nf = (size_t)g->nx * g->ny, L = (size_t)nl;
    rt3d_batch_stats bs{};
    bs.nlambda = nl;
    g->fs_ms[0] = g->fs_ms[1] = g->fs_ms[2] = g->fs_ms[3] = 0.0;
    g->fs_lstar32 = 0;
    g->launches = 0;
    TRY(batch_setup(g, nl));
    cudaStream_t s = g->stream;
    CK(cudaMemcpyAsync(g->bchi, chi, L * N * sizeof(double), cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(g->beps, eps, L * N * sizeof(double), cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(g->bB, B, L * N * sizeof(double), cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(g->bJ, J_inout, L * N * sizeof(double), cudaMemcpyDefault, s));
    const bool tf = bc && bc->I_top_face, bf = bc && bc->I_bottom_face;
    const bool gf = bc && bc->I_bottom_grad;
    if (tf) CK(cudaMemcpyAsync(g->btop, bc->I_top_face, L * nf * sizeof(double), cudaMemcpyDefault, s));
    if (bf) CK(cudaMemcpyAsync(g->bbot, bc->I_bottom_face, L * nf * sizeof(double), cudaMemcpyDefault, s));
    if (gf) CK(cudaMemcpyAsync(g->bgrad, bc->I_bottom_grad, L * nf * sizeof(double), cudaMemcpyDefault, s));

    // Lambda* of every wavelength (FP32 formal solution with Lambda*, once),
    // folded into its OS coefficients.
    for (int l = 0; l < nl; ++l) {
        float2 *cl = g->bchiS + 4 * (size_t)l * N;
        CKL(launch_pack(g->nx, g->ny, g->nz, g->bchi + l * N, 1.0, g->bB + l * N, cl, false, s));
        FsParams p{};
        p.nx = g->nx;
        p.ny = g->ny;
        p.nz = g->nz;
        p.nangles = g->nO;
        p.order = g->tpl.order;
        p.toff = g->tpl.toff;
        p.tlen = g->tpl.tlen;
        p.up = g->tpl.up;
        p.mu = g->tpl.mu;
        p.code = g->tpl.code;
        p.len = g->tpl.len32;
        p.cw = g->tpl.cw32;
        p.win = g->tpl.win;
        p.rec32 = g->tpl.rec32;
        p.chiS = cl;
        p.J = g->Jfs;
        p.lstar = g->lstar;
        p.homogeneous = 1;
        CK(cudaMemsetAsync(g->Jfs, 0, sizeof(double) * N, s));
        CK(cudaMemsetAsync(g->lstar, 0, sizeof(double) * 27 * N, s));
        CKL(launch_fs(p, false, g->parab, true, s));
        CKL(launch_os_prep(g->nx, g->ny, g->nz, g->lstar, g->beps + l * N, g->ba + l * os_coef_count((long long)N),
                           false, g->binv + l * N, s, g->per));
        ++bs.fs_lambda32;
    }
    g->lstar_valid = false;  // the grid's single-wavelength Lambda* was overwritten

    // device state
    std::vector<int> ones(L, 1);
    BatchState &h = g->bsh;
    CK(cudaMemcpyAsync(h.active, ones.data(), L * sizeof(int), cudaMemcpyHostToDevice, s));
    std::vector<int> iota(L);
    for (size_t l = 0; l < L; ++l) iota[l] = (int)l;
    CK(cudaMemcpyAsync(h.alist, iota.data(), L * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(h.state, 0, L * sizeof(int), s));
    CK(cudaMemsetAsync(h.iters, 0, L * sizeof(int), s));
    CK(cudaMemsetAsync(g->bJrep, 0, 4 * L * N * sizeof(double), s));
    h.nactive = nl;
    CK(cudaMemcpyAsync(g->bsd, &h, sizeof(BatchState), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));

    BatchFsParams bp{};
    bp.nx = g->nx;
    bp.ny = g->ny;
    bp.nz = g->nz;
    bp.nangles = g->nO;
    bp.order = g->tpl.order;
    bp.toff = g->tpl.toff;
    bp.tlen = g->tpl.tlen;
    bp.up = g->tpl.up;
    bp.mu = g->tpl.mu;
    bp.rec32 = g->tpl.rec32;
    bp.chiS = g->bchiS;
    bp.Jrep = g->bJrep;
    bp.top_face = tf ? g->btop : nullptr;
    bp.bot_face = bf ? g->bbot : nullptr;
    bp.bot_grad = gf ? g->bgrad : nullptr;
    bp.I_top = bc ? bc->I_top : 0.0;
    bp.I_bot = bc ? bc->I_bottom : 0.0;
    bp.bs = g->bsd;

    // Batched autotuner: every candidate shape with one characteristic per
    // thread is timed once on this batch's first source (CUDA events on the
    // batch stream), the fastest goes into the graph; kept for later calls.
    if (g->bfs_shape.block == 0) {
        CK(cudaEventRecord(g->bev0, s));
        CK(cudaStreamWaitEvent(g->bstream, g->bev0, 0));
        CKL(launch_b_source(bp, nl, g->bJ, g->beps, g->bB, g->bstream));
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        float best = 0.0f;
        int pick = -1;
        for (int i = 0; i < RT3D_FS_TUNE_SHAPES; ++i) {
            if (kFsShapes[i].rays_per_thread != 1) continue;
            CK(cudaEventRecord(e0, g->bstream));
            CKL(launch_b_fs(bp, nl, kFsShapes[i], g->parab, g->bstream));
            CK(cudaEventRecord(e1, g->bstream));
            CK(cudaMemsetAsync(g->bJrep, 0, 4 * L * N * sizeof(double), g->bstream));
            CK(cudaEventSynchronize(e1));
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            g->bfs_tune_ms[i] = ms;
            if (pick < 0 || ms < best) {
                best = ms;
                pick = i;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        CK(cudaStreamSynchronize(g->bstream));
        g->bfs_shape = kFsShapes[pick];
    }
    bs.fs_shape = rt3d_fs_shape{g->bfs_shape.block, g->bfs_shape.rays_per_thread,
                                g->bfs_shape.widen, g->bfs_shape.branchless};
    for (int i = 0; i < RT3D_FS_TUNE_SHAPES; ++i) bs.fs_tune_ms[i] = g->bfs_tune_ms[i];

    // capture one iteration into a CUDA graph on the batch stream
    const int iter_cap = max_iter;
    const double switch_tol = g->fs64 ? tol : std::max(tol, 1e-6);
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // one iteration over a wavelength extent of nlaunch (>= the active count)
    auto capture = [&](int nlaunch) -> rt3d_status {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        CK(cudaStreamBeginCapture(g->bstream, cudaStreamCaptureModeThreadLocal));
        cudaError_t le = launch_batch_iteration(bp, nl, nlaunch, g->bJ, g->beps, g->bB, g->ba,
                                                g->binv, g->br, g->bbuf0, g->bbuf1, g->bb32_0,
                                                g->bb32_1, kBatchSweeps, 1e-3, switch_tol,
                                                iter_cap, g->parab, g->bfs_shape, g->bstream);
        cudaError_t ce = cudaStreamEndCapture(g->bstream, &graph);
        if (le != cudaSuccess || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            graph = nullptr;
            return fail(RT3D_ECUDA, "batch graph capture failed: %s",
                        cudaGetErrorString(le != cudaSuccess ? le : ce));
        }
        CK(cudaGraphInstantiate(&exec, graph, 0));
        return RT3D_OK;
    };
    int nlaunch = nl;
    TRY(capture(nlaunch));
    const long long per_iter = 7 + kBatchSweeps;
    CK(cudaEventRecord(g->bev0, s));
    CK(cudaStreamWaitEvent(g->bstream, g->bev0, 0));
    float fs_ms_total = 0.0f;
    cudaEvent_t t0, t1;
    CK(cudaEventCreate(&t0));
    CK(cudaEventCreate(&t1));
    CK(cudaEventRecord(t0, g->bstream));
    int replays = 0, nactive = nl;
    while (nactive > 0 && replays < iter_cap) {
        const int burst = std::min(4, iter_cap - replays);
        for (int i = 0; i < burst; ++i) CK(cudaGraphLaunch(exec, g->bstream));
        replays += burst;
        CK(cudaMemcpyAsync(&nactive, &g->bsd->nactive, sizeof(int), cudaMemcpyDeviceToHost,
                           g->bstream));
        CK(cudaStreamSynchronize(g->bstream));
        // retired wavelengths leave the launches: a smaller extent once a
        // quarter of the launched ones has retired
        if (nactive > 0 && 4 * nactive <= 3 * nlaunch) {
            nlaunch = nactive;
            TRY(capture(nlaunch));
            ++bs.recaptures;
        }
    }
    CK(cudaEventRecord(t1, g->bstream));
    CK(cudaEventSynchronize(t1));
    CK(cudaEventElapsedTime(&fs_ms_total, t0, t1));
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    g->launches += per_iter * replays;
    bs.graph_replays = replays;
    bs.batch_ms = fs_ms_total;
    CK(cudaEventRecord(g->bev1, g->bstream));
    CK(cudaStreamWaitEvent(s, g->bev1, 0));

    std::vector<int> iters(L), state(L);
    CK(cudaMemcpyAsync(iters.data(), h.iters, L * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(state.data(), h.state, L * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int l = 0; l < nl; ++l) bs.fs_batched += iters[l];
    bs.fs_lambda32 += bs.fs_batched;
    bs.iterations = replays;

    // FP64 refinement and certification of every wavelength with the
    // single-wavelength Krylov solver, started from the batched J.
    int nconv = 0;
    double max_est = 0.0, max_res = 0.0;
    for (int l = 0; l < nl; ++l) {
        int st_l = state[l];
        if (st_l == 3) {
            if (status_out) status_out[l] = RT3D_ENUMERIC;
            continue;
        }
        CK(cudaMemcpyAsync(g->chi, g->bchi + l * N, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(g->eps, g->beps + l * N, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(g->B, g->bB + l * N, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(g->J, g->bJ + l * N, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CKL(launch_pack(g->nx, g->ny, g->nz, g->chi, 1.0, g->chi, g->chiS32, false, s));
        CKL(launch_pack(g->nx, g->ny, g->nz, g->chi, 1.0, g->chi, g->chiS64, true, s));
        g->lstar_valid = false;
        rt3d_bc bl{};
        bl.I_top = bc ? bc->I_top : 0.0;
        bl.I_bottom = bc ? bc->I_bottom : 0.0;
        bl.I_top_face = tf ? g->btop + l * nf : nullptr;
        bl.I_bottom_face = bf ? g->bbot + l * nf : nullptr;
        bl.I_bottom_grad = gf ? g->bgrad + l * nf : nullptr;
        FsParams fp, fp64k, fphomk;
        TRY(fs_params(g, &bl, g->fs64, false, &fp));
        TRY(fs_params(g, &bl, true, false, &fp64k));
        TRY(fs_params(g, nullptr, g->fs64, true, &fphomk));
        rt3d_solve_stats sl{};
        bool kconv = false;
        TRY(krylov_solve(g, fp, fp64k, fphomk, tol, max_iter, sl, &kconv));
        CK(cudaMemcpyAsync(g->bJ + l * N, g->J, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
        bs.fs_lambda32 += sl.fs_fp32;
        bs.fs_lambda64 += sl.fs_fp64;
        bs.fs_lambda_ff += sl.fs_ff;
        max_est = std::max(max_est, sl.est_error);
        max_res = std::max(max_res, sl.residual64);
        if (kconv) ++nconv;
        if (status_out) status_out[l] = kconv ? RT3D_OK : RT3D_ENOTCONVERGED;
    }
    g->lstar_valid = false;
    CK(cudaMemcpyAsync(J_inout, g->bJ, L * N * sizeof(double), cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
    TRY(collect_events(g));
    bs.converged = nconv;
    bs.max_est_error = max_est;
    bs.max_residual64 = max_res;
    bs.fs32_ms = g->fs_ms[0] + g->fs_ms[3] + bs.batch_ms;
    bs.fs64_ms = g->fs_ms[1];
    bs.fsff_ms = g->fs_ms[2];
    bs.launches = g->launches;
    bs.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (stats) *stats = bs;
    if (nconv < nl)
        return fail(RT3D_ENOTCONVERGED, "%d of %d wavelengths not converged", nl - nconv, nl);
    return RT3D_OK;
}

}  // extern "C"
