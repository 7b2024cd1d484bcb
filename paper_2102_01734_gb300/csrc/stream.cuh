// Host-resident spherical geometry cache (the SmallGPU residency of Sec. 4.3):
// device helpers of its build. Kept apart from rt3d_internal.cuh so that the
// formal-solution sources stay as they are.
#pragma once
#include <cuda_runtime.h>

namespace rt3d {

// ray_off[r] -= shift[ray_angle[r]] for r < nrays: the build writes segment
// offsets relative to the staging group, the formal solution wants them
// relative to the residency chunk of the ray's angle (shift = chunk start -
// group start, >= 0)
cudaError_t launch_rebase_ray_off(long long *ray_off, const int *ray_angle,
                                  const long long *shift, long long nrays, cudaStream_t s);

}  // namespace rt3d
