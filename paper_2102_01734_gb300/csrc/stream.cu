// Build helper of the host-resident spherical cache (see stream.cuh).
#include "stream.cuh"

#include <algorithm>

namespace rt3d {

namespace {

__global__ void rebase_ray_off_kernel(long long *__restrict__ ray_off,
                                      const int *__restrict__ ray_angle,
                                      const long long *__restrict__ shift, long long nrays) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nrays; r += stride)
        ray_off[r] -= shift[ray_angle[r]];
}

}  // namespace

cudaError_t launch_rebase_ray_off(long long *ray_off, const int *ray_angle,
                                  const long long *shift, long long nrays, cudaStream_t s) {
    if (nrays <= 0) return cudaSuccess;
    const long long blocks = std::min<long long>((nrays + 255) / 256, 65536);
    rebase_ray_off_kernel<<<(unsigned)blocks, 256, 0, s>>>(ray_off, ray_angle, shift, nrays);
    return cudaGetLastError();
}

}  // namespace rt3d
