// The LTE diffusion inner boundary on the spherical grid's core sphere
// (Sec. 3.2): the core-face arrays, and the entry intensity of every ray that
// starts on the core. Kept apart from rt3d_internal.cuh so that the
// formal-solution sources stay as they are.
#pragma once
#include <cuda_runtime.h>

namespace rt3d {

// Core faces (it + nt ip) of nl stacked grids ([nl][np][nt][nr] in, [nl][np][nt]
// out): dB/dtau = (B0 - B1) / (1/2 (chi0 + chi1) (rc1 - rc0)) between the two
// innermost shells (0 for nr = 1) and I_face = B0 + chi0 (rc0 - r_in) dB/dtau.
cudaError_t launch_sph_diffusion_bc(int nr, int nt, int np, int nl, double rc0, double rc1,
                                    double r_in, const double *chi, const double *B,
                                    double *I_face, double *grad, cudaStream_t s);

// Geometry of the entry intensities: per ray its launch cell, angle, entry
// kind (2: from the core) and core face; the cell-centre tables; the
// directions [nangles][3]
struct SphEntryParams {
    long long nrays;
    int nr, nt;
    double r_in;
    const int *ray_launch, *ray_angle, *ray_kind, *ray_face;
    const double *rc, *stc, *ctc, *cpc, *spc, *dir;
};

// I0[r] = face[f] + mu grad[f] for the rays that start on the core (f their
// core face, mu the cosine between the ray and the core's outward normal at
// the entry point; face NULL: the scalar I_face), 0 for the others;
// ident[r] = r (the face index through which the formal-solution kernels read
// I0 as a per-ray core face)
cudaError_t launch_sph_entry(const SphEntryParams &p, const double *face, double I_face,
                             const double *grad, double *I0, int *ident, cudaStream_t s);

}  // namespace rt3d
