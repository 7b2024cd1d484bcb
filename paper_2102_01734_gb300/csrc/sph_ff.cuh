// Float-float formal solution without Lambda* on the spherical cache
// (fsff.cu). Kept apart from rt3d_internal.cuh so that the formal-solution
// sources stay as they are.
#pragma once
#include "rt3d_internal.cuh"

namespace rt3d {

// chiS: the replicated (chi, S) split into float-float (launch_pack_ff);
// contributions into the replicated FP64 Jrep (zero on entry; fold
// afterwards). Reads p.rec and p.len64 of every point.
cudaError_t launch_sph_fsff(const SphFsParams &p, const float4 *chiS, double *Jrep, bool parabolic,
                            cudaStream_t s);

}  // namespace rt3d
