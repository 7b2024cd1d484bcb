// Tracker for the Cartesian box periodic in x and y (Sec. 4: "setting up the
// geometric paths through the grid for all solid angles"), run once per grid
// to fill the geometry cache (Sec. 4.1).
//
// One thread per solid angle traces the characteristic that starts at the
// centre (1/2, 1/2) of inflow-face cell (0,0): top face (z = nz) for mu < 0,
// bottom face (z = 0) for mu > 0. The m-th crossing of an x plane lies at
// parameter (m - 1/2)/|d_x|, of a y plane at (m - 1/2)/|d_y|, of a z plane at
// m/|mu|: each one IEEE division (__ddiv_rn), so the cache is reproducible bit
// for bit. Equal parameters advance all tied axes in one step (no zero-length
// chord). A chord is the difference of consecutive parameters (__dsub_rn).
//
// Per point the thread also stores the J weight w l_k / (sum of l over the
// layer of the point; every voxel of a layer sees each step of the layer once,
// so that sum is the per-voxel chord sum) and the passage-local Lambda*
// window: ring positions k-7 .. k+1 whose points form the run, ending at k+1,
// of voxels inside the 3x3x3 neighbourhood of point k.
#include "rt3d_internal.cuh"

namespace rt3d {

namespace {

__device__ __forceinline__ int wrap_diff(int a, int b, int n) {
    int d = a - b;
    if (d < 0) d += n;  // 0..n-1
    if (d == 0) return 0;
    if (d == 1) return 1;
    if (d == n - 1) return -1;
    return 2;  // not a neighbour
}

__global__ void trace_kernel(TraceParams p) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= p.nangles) return;
    const double dxv = p.dir[3 * o + 0], dyv = p.dir[3 * o + 1], dzv = p.dir[3 * o + 2];
    const double ax = fabs(dxv), ay = fabs(dyv), az = fabs(dzv);
    const long long base = p.toff[o];
    const int cap = p.cap[o];
    if (!(az > 0.0)) {
        atomicCAS(p.err, 0, 1);
        p.tlen[o] = 0;
        return;
    }
    const int sx = dxv > 0.0 ? 1 : -1, sy = dyv > 0.0 ? 1 : -1, sz = dzv > 0.0 ? 1 : -1;
    int x = 0, y = 0, z = dzv > 0.0 ? 0 : p.nz - 1;
    long long mx = 1, my = 1, mz = 1;
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    double tx = ax > 0.0 ? __ddiv_rn((double)mx - 0.5, ax) : inf;
    double ty = ay > 0.0 ? __ddiv_rn((double)my - 0.5, ay) : inf;
    double tz = __ddiv_rn((double)mz, az);
    double tprev = 0.0;
    int k = 0;
    for (;;) {
        double tn = tx < ty ? tx : ty;
        if (tz < tn) tn = tz;
        if (k >= cap) {
            atomicCAS(p.err, 0, 2);
            p.tlen[o] = 0;
            return;
        }
        p.code[base + k] = step_code(x, y, z);
        p.len64[base + k] = __dsub_rn(tn, tprev);
        ++k;
        tprev = tn;
        if (tx == tn) {
            ++mx;
            tx = __ddiv_rn((double)mx - 0.5, ax);
            x += sx;
            if (x >= p.nx) x -= p.nx;
            if (x < 0) x += p.nx;
        }
        if (ty == tn) {
            ++my;
            ty = __ddiv_rn((double)my - 0.5, ay);
            y += sy;
            if (y >= p.ny) y -= p.ny;
            if (y < 0) y += p.ny;
        }
        if (tz == tn) {
            if (mz == p.nz) break;
            ++mz;
            tz = __ddiv_rn((double)mz, az);
            z += sz;
        }
    }
    const int K = k;
    p.tlen[o] = K;

    // Chord sum of every layer, then the J weight of every point.
    double *ls = p.layer_sum + (long long)o * p.nz;
    for (int zz = 0; zz < p.nz; ++zz) ls[zz] = 0.0;
    for (int i = 0; i < K; ++i) ls[p.code[base + i] >> 22] += p.len64[base + i];
    const double w = p.wt[o];
    for (int i = 0; i < K; ++i) {
        const double l = p.len64[base + i];
        const double c = w * (l / ls[p.code[base + i] >> 22]);
        p.cw64[base + i] = c;
        p.cw32[base + i] = (float)c;
        p.len32[base + i] = (float)l;
        const uint32_t ci = p.code[base + i];
        const long long orep = rep_index(ci & 0x7ff, (ci >> 11) & 0x7ff, ci >> 22, p.nx, p.ny);
        p.rec32[base + i] = make_float4(__int_as_float((int)orep), (float)c, (float)(0.5 * l), (float)(0.5 * l));
        p.rec64[base + i] = make_double2(0.5 * l, c);
    }

    // Passage-local Lambda* windows.
    for (int i = 0; i < K; ++i) {
        const uint32_t ci = p.code[base + i];
        const int xi = ci & 0x7ff, yi = (ci >> 11) & 0x7ff, zi = ci >> 22;
        const int jend = (i + 1 < K) ? i + 1 : i;
        uint64_t wcode = 0;
        for (int r = 0; r < kWin; ++r) wcode |= (uint64_t)kWinNone << (5 * r);
        for (int j = jend; j >= 0; --j) {
            const uint32_t cj = p.code[base + j];
            const int ddx = wrap_diff(cj & 0x7ff, xi, p.nx);
            const int ddy = wrap_diff((cj >> 11) & 0x7ff, yi, p.ny);
            const int ddz = (int)(cj >> 22) - zi;
            if (ddx > 1 || ddy > 1 || ddz < -1 || ddz > 1) break;
            const int r = j - i + 7;  // ring position
            if (r < 0) {
                atomicCAS(p.err, 0, 3);  // window longer than the ring
                break;
            }
            const unsigned dcode = (unsigned)((ddx + 1) + 3 * (ddy + 1) + 9 * (ddz + 1));
            wcode &= ~((uint64_t)31 << (5 * r));
            wcode |= (uint64_t)dcode << (5 * r);
        }
        p.win[base + i] = wcode;
    }
}

}  // namespace

cudaError_t launch_trace(const TraceParams &p, cudaStream_t s) {
    const int threads = 64;
    const int blocks = (p.nangles + threads - 1) / threads;
    trace_kernel<<<blocks, threads, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace rt3d
