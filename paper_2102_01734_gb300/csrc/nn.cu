// Learned warm start: the layers of a small 3D U-Net that predicts log J of
// the converged solution from (log chi, log eps, B, log J_start). Not in the
// paper; the ALI/Krylov solve started from its prediction is certified by the
// same FP64 residual as any other start.
//
// Activations are BF16, channel-last [S][V][C] (S samples, V = nx*ny*nz
// voxels, x fastest, C a multiple of 16). Convolutions are 3x3x3, periodic in
// x and y, zero-padded in z (the geometry of the radiative-transfer box),
// computed as implicit GEMMs on the tensor cores: BF16 operands, FP32
// accumulation (nvcuda::wmma 16x16x16 tiles). Weights are stored per
// offset d = (dz+1)*9 + (dy+1)*3 + (dx+1) as Wt[d][Ci][Co] (BF16), with an
// FP32 master copy for the optimiser.
#include <cuda_bf16.h>
#include <mma.h>

#include "rt3d_internal.cuh"
#include "../../include/rt3d_nn.h"

namespace rt3d {

namespace {

using bf16 = __nv_bfloat16;
namespace wm = nvcuda::wmma;

struct Geo {
    int nx, ny, nz;
};

__device__ __forceinline__ int neighbour(int x, int y, int z, int dx, int dy, int dz, Geo g) {
    const int zz = z + dz;
    if (zz < 0 || zz >= g.nz) return -1;
    int xx = x + dx, yy = y + dy;
    xx += (xx < 0) ? g.nx : ((xx >= g.nx) ? -g.nx : 0);
    yy += (yy < 0) ? g.ny : ((yy >= g.ny) ? -g.ny : 0);
    return xx + g.nx * (yy + g.ny * zz);
}

// Y[s][v][co] = act(b[co] + sum_{d, ci} Wt[d][ci][co] X[s][v + sign*d][ci]).
// One warp computes 16 voxels x CO output channels; the 16 x 16 input tile of
// each (offset, channel block) is gathered into shared memory (16-byte rows),
// the weights are read as 16 x 16 B tiles. sign = -1 gives the data gradient
// when called with the transposed weights.
template <int CO>
__global__ void __launch_bounds__(128) conv_kernel(const bf16 *__restrict__ X,
                                                   const bf16 *__restrict__ Wt,
                                                   const float *__restrict__ bias,
                                                   bf16 *__restrict__ Y, float *__restrict__ Yf,
                                                   Geo g, int Ci, int relu, int sign) {
    __shared__ __align__(32) bf16 As[4][16][16];
    __shared__ __align__(32) float Cs[4][16][CO];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int V = g.nx * g.ny * g.nz;
    const int s = blockIdx.y;
    const int v0 = (blockIdx.x * 4 + warp) * 16;
    const bf16 *Xs = X + (long long)s * V * Ci;
    wm::fragment<wm::accumulator, 16, 16, 16, float> acc[CO / 16];
#pragma unroll
    for (int j = 0; j < CO / 16; ++j) wm::fill_fragment(acc[j], 0.0f);
    const int r = lane >> 1, h = lane & 1;  // tile row and 8-channel half of this lane
    const int v = v0 + r;
    const bool live = v < V;
    int x = 0, y = 0, z = 0;
    if (live) {
        x = v % g.nx;
        y = (v / g.nx) % g.ny;
        z = v / (g.nx * g.ny);
    }
    if (v0 < V) {
        for (int d = 0; d < 27; ++d) {
            const int dz = sign * (d / 9 - 1), dy = sign * ((d / 3) % 3 - 1), dx = sign * (d % 3 - 1);
            const int u = live ? neighbour(x, y, z, dx, dy, dz, g) : -1;
            for (int c0 = 0; c0 < Ci; c0 += 16) {
                uint4 val = make_uint4(0u, 0u, 0u, 0u);
                if (u >= 0) val = *reinterpret_cast<const uint4 *>(Xs + (long long)u * Ci + c0 + 8 * h);
                *reinterpret_cast<uint4 *>(&As[warp][r][8 * h]) = val;
                __syncwarp();
                wm::fragment<wm::matrix_a, 16, 16, 16, bf16, wm::row_major> a;
                wm::load_matrix_sync(a, &As[warp][0][0], 16);
#pragma unroll
                for (int j = 0; j < CO / 16; ++j) {
                    wm::fragment<wm::matrix_b, 16, 16, 16, bf16, wm::row_major> b;
                    wm::load_matrix_sync(b, Wt + ((long long)d * Ci + c0) * CO + j * 16, CO);
                    wm::mma_sync(acc[j], a, b, acc[j]);
                }
                __syncwarp();
            }
        }
    }
#pragma unroll
    for (int j = 0; j < CO / 16; ++j)
        wm::store_matrix_sync(&Cs[warp][0][j * 16], acc[j], CO, wm::mem_row_major);
    __syncwarp();
    for (int i = lane; i < 16 * CO; i += 32) {
        const int rr = i / CO, c = i % CO;
        const int vv = v0 + rr;
        if (vv >= V) continue;
        float o = Cs[warp][rr][c] + (bias ? bias[c] : 0.0f);
        if (relu) o = fmaxf(o, 0.0f);
        if (Y) Y[((long long)s * V + vv) * CO + c] = __float2bfloat16(o);
        if (Yf) Yf[((long long)s * V + vv) * CO + c] = o;
    }
}

// dW[d][ci][co] += sum_v X[v + d][ci] dY[v][co] over the voxels of this block
// (grid-stride over 64-voxel chunks, FP32 atomics once at the end). Each warp
// owns up to four (ci tile, co tile) pairs; (Ci/16)(Co/16) <= 16.
__global__ void __launch_bounds__(128) conv_wgrad_kernel(const bf16 *__restrict__ X,
                                                         const bf16 *__restrict__ dY,
                                                         float *__restrict__ dW, Geo g, int Ci,
                                                         int Co) {
    __shared__ __align__(32) bf16 Xt[64 * 96];  // [64][Ci] gathered neighbours, Ci <= 96
    const int warp = threadIdx.x >> 5;
    const int V = g.nx * g.ny * g.nz;
    const int d = blockIdx.y, s = blockIdx.z;
    const int dz = d / 9 - 1, dy = (d / 3) % 3 - 1, dx = d % 3 - 1;
    const bf16 *Xs = X + (long long)s * V * Ci;
    const bf16 *dYs = dY + (long long)s * V * Co;
    const int tci = Ci / 16, tco = Co / 16, npairs = tci * tco;
    wm::fragment<wm::accumulator, 16, 16, 16, float> acc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) wm::fill_fragment(acc[k], 0.0f);
    const int nchunk = (V + 63) / 64;
    const int vec = Ci / 8;  // 16-byte vectors per row
    for (int ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
        const int v0 = ch * 64;
        __syncthreads();
        for (int i = threadIdx.x; i < 64 * vec; i += blockDim.x) {
            const int rr = i / vec, q = i % vec;
            const int v = v0 + rr;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (v < V) {
                const int x = v % g.nx, y = (v / g.nx) % g.ny, z = v / (g.nx * g.ny);
                const int u = neighbour(x, y, z, dx, dy, dz, g);
                if (u >= 0) val = *reinterpret_cast<const uint4 *>(Xs + (long long)u * Ci + 8 * q);
            }
            *reinterpret_cast<uint4 *>(Xt + rr * Ci + 8 * q) = val;
        }
        __syncthreads();
        const int nsub = min(4, (V - v0 + 15) / 16);
        for (int k = 0; k < 4; ++k) {
            const int pair = warp + 4 * k;
            if (pair >= npairs) break;
            const int ti = pair / tco, to = pair % tco;
            for (int sub = 0; sub < nsub; ++sub) {
                // A = X_d^T: rows ci, cols v (column-major view of Xt)
                wm::fragment<wm::matrix_a, 16, 16, 16, bf16, wm::col_major> a;
                wm::load_matrix_sync(a, Xt + (sub * 16) * Ci + ti * 16, Ci);
                wm::fragment<wm::matrix_b, 16, 16, 16, bf16, wm::row_major> b;
                const int vb = v0 + sub * 16;
                if (vb + 16 <= V) {
                    wm::load_matrix_sync(b, dYs + (long long)vb * Co + to * 16, Co);
                } else {
                    // ragged tail: stage the valid rows, zeros elsewhere
                    __shared__ __align__(32) bf16 tail[4][16][16];
                    const int lane = threadIdx.x & 31;
                    for (int i = lane; i < 256; i += 32) {
                        const int rr = i / 16, c = i % 16;
                        tail[warp][rr][c] = (vb + rr < V) ? dYs[(long long)(vb + rr) * Co + to * 16 + c]
                                                           : __float2bfloat16(0.0f);
                    }
                    __syncwarp();
                    wm::load_matrix_sync(b, &tail[warp][0][0], 16);
                    __syncwarp();
                }
                wm::mma_sync(acc[k], a, b, acc[k]);
            }
        }
    }
    // flush: each warp's pairs through shared staging into FP32 atomics
    __shared__ __align__(32) float Cs[4][16][16];
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < 4; ++k) {
        const int pair = warp + 4 * k;
        if (pair >= npairs) break;
        const int ti = pair / tco, to = pair % tco;
        wm::store_matrix_sync(&Cs[warp][0][0], acc[k], 16, wm::mem_row_major);
        __syncwarp();
        for (int i = lane; i < 256; i += 32) {
            const int rr = i / 16, c = i % 16;
            atomicAdd(dW + ((long long)d * Ci + ti * 16 + rr) * Co + to * 16 + c, Cs[warp][rr][c]);
        }
        __syncwarp();
    }
}

// db[c] += sum_v dY[v][c]
__global__ void bias_grad_kernel(const bf16 *dY, float *db, long long rows, int C) {
    const int c = threadIdx.x % C;
    const int lanes = blockDim.x / C;
    float acc = 0.0f;
    for (long long v = blockIdx.x * lanes + threadIdx.x / C; v < rows; v += (long long)gridDim.x * lanes)
        acc += __bfloat162float(dY[v * C + c]);
    atomicAdd(db + c, acc);
}

// dYpre = dY * (Y > 0)
__global__ void relu_bwd_kernel(const bf16 *dY, const bf16 *Y, bf16 *out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = __bfloat162float(Y[i]) > 0.0f ? dY[i] : __float2bfloat16(0.0f);
}

// 2x2x2 average (periodic in x, y; a child beyond the top layer counts as 0)
__global__ void pool_kernel(const bf16 *X, bf16 *P, Geo g, Geo p, int C, int S) {
    const long long Vp = (long long)p.nx * p.ny * p.nz, V = (long long)g.nx * g.ny * g.nz;
    const long long n = Vp * C * S;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long vs = i / C;
        const int s = (int)(vs / Vp);
        const long long vp = vs % Vp;
        const int x = (int)(vp % p.nx), y = (int)((vp / p.nx) % p.ny), z = (int)(vp / ((long long)p.nx * p.ny));
        float acc = 0.0f;
        for (int a = 0; a < 2; ++a) {
            const int zz = 2 * z + a;
            if (zz >= g.nz) continue;
            for (int b = 0; b < 2; ++b)
                for (int e = 0; e < 2; ++e) {
                    const int xx = (2 * x + e) % g.nx, yy = (2 * y + b) % g.ny;
                    acc += __bfloat162float(X[((long long)s * V + xx + (long long)g.nx * (yy + (long long)g.ny * zz)) * C + c]);
                }
        }
        P[i] = __float2bfloat16(acc * 0.125f);
    }
}

// dX[v] = dP[parent(v)] / 8 (summed over the parents that wrap onto v)
__global__ void pool_bwd_kernel(const bf16 *dP, float *dX32, Geo g, Geo p, int C, int S) {
    const long long Vp = (long long)p.nx * p.ny * p.nz, V = (long long)g.nx * g.ny * g.nz;
    const long long n = Vp * C * S;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long vs = i / C;
        const int s = (int)(vs / Vp);
        const long long vp = vs % Vp;
        const int x = (int)(vp % p.nx), y = (int)((vp / p.nx) % p.ny), z = (int)(vp / ((long long)p.nx * p.ny));
        const float gval = __bfloat162float(dP[i]) * 0.125f;
        for (int a = 0; a < 2; ++a) {
            const int zz = 2 * z + a;
            if (zz >= g.nz) continue;
            for (int b = 0; b < 2; ++b)
                for (int e = 0; e < 2; ++e) {
                    const int xx = (2 * x + e) % g.nx, yy = (2 * y + b) % g.ny;
                    atomicAdd(dX32 + ((long long)s * V + xx + (long long)g.nx * (yy + (long long)g.ny * zz)) * C + c, gval);
                }
        }
    }
}

// U[v][c] = X[parent(v)][c] written into channels [coff, coff + C) of a
// Ctot-channel buffer; the backward pass sums the children of every parent.
__global__ void up_kernel(const bf16 *X, bf16 *U, Geo g, Geo p, int C, int Ctot, int coff, int S) {
    const long long V = (long long)g.nx * g.ny * g.nz, Vp = (long long)p.nx * p.ny * p.nz;
    const long long n = V * C * S;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long vs = i / C;
        const int s = (int)(vs / V);
        const long long v = vs % V;
        const int x = (int)(v % g.nx), y = (int)((v / g.nx) % g.ny), z = (int)(v / ((long long)g.nx * g.ny));
        const long long par = (x / 2) + (long long)p.nx * ((y / 2) + (long long)p.ny * (z / 2));
        U[((long long)s * V + v) * Ctot + coff + c] = X[((long long)s * Vp + par) * C + c];
    }
}

__global__ void up_bwd_kernel(const bf16 *dU, float *dX32, Geo g, Geo p, int C, int Ctot, int coff,
                              int S) {
    const long long V = (long long)g.nx * g.ny * g.nz, Vp = (long long)p.nx * p.ny * p.nz;
    const long long n = V * C * S;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long vs = i / C;
        const int s = (int)(vs / V);
        const long long v = vs % V;
        const int x = (int)(v % g.nx), y = (int)((v / g.nx) % g.ny), z = (int)(v / ((long long)g.nx * g.ny));
        const long long par = (x / 2) + (long long)p.nx * ((y / 2) + (long long)p.ny * (z / 2));
        atomicAdd(dX32 + ((long long)s * Vp + par) * C + c,
                  __bfloat162float(dU[((long long)s * V + v) * Ctot + coff + c]));
    }
}

// copy channels [coff, coff+C) of a Ctot-channel buffer to/from a C-channel one
__global__ void channel_copy_kernel(const bf16 *src, int Cs, int soff, bf16 *dst, int Cd, int doff,
                                    int C, long long rows) {
    const long long n = rows * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / C;
        const int c = (int)(i % C);
        dst[r * Cd + doff + c] = src[r * Cs + soff + c];
    }
}

__global__ void f32_to_bf16_kernel(const float *a, bf16 *b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16(a[i]);
}

__global__ void add_bf16_f32_kernel(const bf16 *a, const float *b, bf16 *out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16(__bfloat162float(a[i]) + b[i]);
}

// Features from the radiative-transfer arrays (FP64 [S][V]) into a 16-channel
// BF16 tensor: log10(chi)/3, log10(eps)/4, B - 1, ln(J0), 12 zero channels.
__global__ void features_kernel(const double *chi, const double *eps, const double *B,
                                const double *J0, bf16 *X, long long rows) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < rows;
         i += (long long)gridDim.x * blockDim.x) {
        float f[16] = {0};
        f[0] = (float)(log10(chi[i]) / 3.0);
        f[1] = (float)(log10(eps[i]) / 4.0);
        f[2] = (float)(B[i] - 1.0);
        f[3] = (float)log(fmax(J0[i], 1e-300));
        for (int c = 0; c < 16; ++c) X[i * 16 + c] = __float2bfloat16(f[c]);
    }
}

// Loss on channel 0 of the FP32 network output y, read as the correction
// ln J - ln J0: L = mean (y - ln(target/J0))^2; the gradient dY (BF16, 16
// channels, zeros beyond channel 0) and the summed squared error are written.
__global__ void mse_kernel(const float *Yf, const double *target, const double *J0, bf16 *dY,
                           float *sse, long long rows, float scale) {
    float acc = 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < rows;
         i += (long long)gridDim.x * blockDim.x) {
        const float e = Yf[i * 16] - (float)log(target[i] / J0[i]);
        acc += e * e;
        dY[i * 16] = __float2bfloat16(2.0f * e * scale);
        for (int c = 1; c < 16; ++c) dY[i * 16 + c] = __float2bfloat16(0.0f);
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(sse, acc);
}

// J = J0 exp(y) (FP64 out)
__global__ void apply_kernel(const float *Yf, const double *J0, double *J, long long rows) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < rows;
         i += (long long)gridDim.x * blockDim.x)
        J[i] = J0[i] * exp((double)Yf[i * 16]);
}

// Adam on an FP32 master copy, then the BF16 working copy Wt[d][ci][co] and
// its transpose WT[d][co][ci] (for the data gradient).
__global__ void adam_kernel(float *w, const float *gw, float *m, float *v, int n, float lr,
                            float b1, float b2, float eps, float c1, float c2, bf16 *Wt, bf16 *WT,
                            int Ci, int Co) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = gw[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        w[i] = wi;
        if (Wt) {
            Wt[i] = __float2bfloat16(wi);
            const int d = i / (Ci * Co), rem = i % (Ci * Co), ci = rem / Co, co = rem % Co;
            WT[((long long)d * Co + co) * Ci + ci] = __float2bfloat16(wi);
        }
    }
}

int gsz(long long n) {
    long long b = (n + 255) / 256;
    const long long cap = 16LL * device_sm_count();
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

}  // namespace rt3d

using namespace rt3d;

extern "C" {

static rt3d_status nn_err(cudaError_t e) {
    if (e == cudaSuccess) return RT3D_OK;
    set_last_error(cudaGetErrorString(e));
    return RT3D_ECUDA;
}

rt3d_status rt3d_nn_conv3d(const void *X, const void *Wt, const float *bias, void *Y, float *Yf,
                           int S, int nx, int ny, int nz, int Ci, int Co, int relu, int transpose,
                           void *stream) {
    if (Ci <= 0 || Ci % 16 || Ci > 96 || (Co != 16 && Co != 32 && Co != 48 && Co != 64 && Co != 96) ||
        S < 1) {
        set_last_error("conv3d: Ci must be a multiple of 16 up to 96 and Co one of 16/32/48/64/96");
        return RT3D_EINVAL;
    }
    const long long V = (long long)nx * ny * nz;
    if (V <= 0 || V * 64 >= (1LL << 31)) {
        set_last_error("conv3d: bad volume");
        return RT3D_EINVAL;
    }
    Geo g{nx, ny, nz};
    dim3 grid((unsigned)((V + 63) / 64), S);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bf16 *x = static_cast<const bf16 *>(X);
    const bf16 *w = static_cast<const bf16 *>(Wt);
    bf16 *y = static_cast<bf16 *>(Y);
    const int sign = transpose ? -1 : 1;
    if (Co == 16) conv_kernel<16><<<grid, 128, 0, s>>>(x, w, bias, y, Yf, g, Ci, relu, sign);
    else if (Co == 32) conv_kernel<32><<<grid, 128, 0, s>>>(x, w, bias, y, Yf, g, Ci, relu, sign);
    else if (Co == 48) conv_kernel<48><<<grid, 128, 0, s>>>(x, w, bias, y, Yf, g, Ci, relu, sign);
    else if (Co == 64) conv_kernel<64><<<grid, 128, 0, s>>>(x, w, bias, y, Yf, g, Ci, relu, sign);
    else conv_kernel<96><<<grid, 128, 0, s>>>(x, w, bias, y, Yf, g, Ci, relu, sign);
    return nn_err(cudaGetLastError());
}

rt3d_status rt3d_nn_conv3d_wgrad(const void *X, const void *dY, float *dW, float *db, int S, int nx,
                                 int ny, int nz, int Ci, int Co, void *stream) {
    if (Ci <= 0 || Ci % 16 || Ci > 96 || Co <= 0 || Co % 16 || (Ci / 16) * (Co / 16) > 16) {
        set_last_error("conv3d_wgrad: Ci <= 96 and (Ci/16)(Co/16) <= 16");
        return RT3D_EINVAL;
    }
    Geo g{nx, ny, nz};
    const long long V = (long long)nx * ny * nz;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int gx = (int)((V + 63) / 64);
    if (gx > 32) gx = 32;
    dim3 grid(gx, 27, S);
    conv_wgrad_kernel<<<grid, 128, 0, s>>>(static_cast<const bf16 *>(X), static_cast<const bf16 *>(dY),
                                            dW, g, Ci, Co);
    if (db) {
        const int threads = (256 / Co) * Co;
        bias_grad_kernel<<<gsz(V * S), threads, 0, s>>>(static_cast<const bf16 *>(dY), db, V * S, Co);
    }
    return nn_err(cudaGetLastError());
}

rt3d_status rt3d_nn_relu_bwd(const void *dY, const void *Y, void *out, long long n, void *stream) {
    relu_bwd_kernel<<<gsz(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const bf16 *>(dY), static_cast<const bf16 *>(Y), static_cast<bf16 *>(out), n);
    return nn_err(cudaGetLastError());
}

rt3d_status rt3d_nn_pool(const void *X, void *P, int S, int nx, int ny, int nz, int C, void *stream) {
    Geo g{nx, ny, nz}, p{(nx + 1) / 2, (ny + 1) / 2, (nz + 1) / 2};
    const long long n = (long long)p.nx * p.ny * p.nz * C * S;
    pool_kernel<<<gsz(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const bf16 *>(X), static_cast<bf16 *>(P), g, p, C, S);
    return nn_err(cudaGetLastError());
}

rt3d_status rt3d_nn_pool_bwd(const void *dP, float *dX32, int S, int nx, int ny, int nz, int C,
                             void *stream) {
    Geo g{nx, ny, nz}, p{(nx + 1) / 2, (ny + 1) / 2, (nz + 1) / 2};
    const long long n = (long long)p.nx * p.ny * p.nz * C * S;
    pool_bwd_kernel<<<gsz(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const bf16 *>(dP), dX32, g, p, C, S);
    return nn_err(cudaGetLastError());
}

rt3d_status rt3d_nn_upsample(const void *X, void *U, int S, int nx, int ny, int nz, int C, int Ctot,
                             int coff, void *stream) {
    Geo g{nx, ny, nz}, p{(nx + 1) / 2, (ny + 1) / 2, (nz + 1) / 2};
    const long long n = (long long)nx * ny * nz * C * S;
    up_kernel<<<gsz(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const bf16 *>(X), static_cast<bf16 *>(U), g, p, C, Ctot, coff, S);
    return nn_err(cudaGetLastError());
}

rt3d_status rt3d_nn_upsample_bwd(const void *dU, float *dX32, int S, int nx, int ny, int nz, int C,
                                 int Ctot, int coff, void *stream) {
    Geo g{nx, ny, nz}, p{(nx + 1) / 2, (ny + 1) / 2, (nz + 1) / 2};
    const long long n = (long long)nx * ny * nz * C * S;
    up_bwd_kernel<<<gsz(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const bf16 *>(dU), dX32, g, p, C, Ctot, coff, S);
    return nn_err(cudaGetLastError());
}

rt3d_status rt3d_nn_channel_copy(const void *src, int Cs, int soff, void *dst, int Cd, int doff, int C,
                                 long long rows, void *stream) {
    channel_copy_kernel<<<gsz(rows * C), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const bf16 *>(src), Cs, soff, static_cast<bf16 *>(dst), Cd, doff, C, rows);
    return nn_err(cudaGetLastError());
}

rt3d_status rt3d_nn_f32_to_bf16(const float *a, void *b, long long n, void *stream) {
    f32_to_bf16_kernel<<<gsz(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(a, static_cast<bf16 *>(b), n);
    return nn_err(cudaGetLastError());
}

rt3d_status rt3d_nn_add_bf16_f32(const void *a, const float *b, void *out, long long n, void *stream) {
    add_bf16_f32_kernel<<<gsz(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const bf16 *>(a), b, static_cast<bf16 *>(out), n);
    return nn_err(cudaGetLastError());
}

rt3d_status rt3d_nn_features(const double *chi, const double *eps, const double *B, const double *J0,
                             void *X, long long rows, void *stream) {
    features_kernel<<<gsz(rows), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        chi, eps, B, J0, static_cast<bf16 *>(X), rows);
    return nn_err(cudaGetLastError());
}

rt3d_status rt3d_nn_mse(const float *Yf, const double *target, const double *J0, void *dY, float *sse,
                        long long rows, float grad_scale, void *stream) {
    mse_kernel<<<gsz(rows), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        Yf, target, J0, static_cast<bf16 *>(dY), sse, rows, grad_scale);
    return nn_err(cudaGetLastError());
}

rt3d_status rt3d_nn_apply(const float *Yf, const double *J0, double *J, long long rows, void *stream) {
    apply_kernel<<<gsz(rows), 256, 0, static_cast<cudaStream_t>(stream)>>>(Yf, J0, J, rows);
    return nn_err(cudaGetLastError());
}

rt3d_status rt3d_nn_adam(float *w, const float *g, float *m, float *v, int n, float lr, float b1,
                         float b2, float eps, int step, void *Wt, void *WT, int Ci, int Co,
                         void *stream) {
    const float c1 = 1.0f / (1.0f - powf(b1, (float)step));
    const float c2 = 1.0f / (1.0f - powf(b2, (float)step));
    adam_kernel<<<gsz(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        w, g, m, v, n, lr, b1, b2, eps, c1, c2, static_cast<bf16 *>(Wt), static_cast<bf16 *>(WT), Ci, Co);
    return nn_err(cudaGetLastError());
}

}  // extern "C"
