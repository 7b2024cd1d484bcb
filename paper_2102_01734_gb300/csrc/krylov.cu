// Vector kernels of the Krylov-accelerated ALI (FGMRES on the scattering
// problem (1 - Lambda(1-eps)) J = Lambda(eps B) + J_bc, right-preconditioned
// by the OS operator [1 - Lambda*(1-eps)]^-1 of Eq. alo). All vectors are
// FP64 [N]; basis vectors are addressed through a device array of pointers.
#include "rt3d_internal.cuh"

namespace rt3d {

namespace {

__device__ __forceinline__ double block_sum(double x) {
    __shared__ double sm[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = x;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        r = lane < nw ? sm[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
    }
    __syncthreads();
    return r;  // valid in thread 0
}

// out[i] += <V[i], w> for i = blockIdx.y
__global__ void multi_dot_kernel(int n, const double *const *V, const double *w, double *out) {
    const double *v = V[blockIdx.y];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        acc = fma(v[i], w[i], acc);
    acc = block_sum(acc);
    if (threadIdx.x == 0) atomicAdd(out + blockIdx.y, acc);
}

// w -= sum_i coef[i] V[i]
__global__ void multi_axpy_kernel(int n, double *w, const double *const *V, const double *coef,
                                  int k) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < k; ++j) acc = fma(__ldg(coef + j), V[j][i], acc);
        w[i] -= acc;
    }
}

__global__ void scale_copy_kernel(int n, const double *src, double alpha, double *dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dst[i] = alpha * src[i];
}

__global__ void sub_kernel(int n, const double *a, const double *b, double *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = a[i] - b[i];
}

int blocks_for(int n, int threads, int cap) {
    int b = (n + threads - 1) / threads;
    return b < 1 ? 1 : (b > cap ? cap : b);
}

}  // namespace

cudaError_t launch_multi_dot(int n, const double *const *V, int k, const double *w, double *out,
                             cudaStream_t s) {
    dim3 grid(blocks_for(n, 256, 2 * device_sm_count()), k);
    multi_dot_kernel<<<grid, 256, 0, s>>>(n, V, w, out);
    return cudaGetLastError();
}

cudaError_t launch_multi_axpy(int n, double *w, const double *const *V, const double *coef, int k,
                              cudaStream_t s) {
    multi_axpy_kernel<<<blocks_for(n, 256, 8 * device_sm_count()), 256, 0, s>>>(n, w, V, coef, k);
    return cudaGetLastError();
}

cudaError_t launch_scale_copy(int n, const double *src, double alpha, double *dst, cudaStream_t s) {
    scale_copy_kernel<<<blocks_for(n, 256, 8 * device_sm_count()), 256, 0, s>>>(n, src, alpha, dst);
    return cudaGetLastError();
}

cudaError_t launch_sub(int n, const double *a, const double *b, double *out, cudaStream_t s) {
    sub_kernel<<<blocks_for(n, 256, 8 * device_sm_count()), 256, 0, s>>>(n, a, b, out);
    return cudaGetLastError();
}

}  // namespace rt3d
