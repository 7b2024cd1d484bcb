// The LTE diffusion inner boundary on the spherical grid (see sph_bc.cuh).
// The face arrays use the same operations in the same order as the CPU
// definition, without contraction, so they agree with it bit for bit.
#include "sph_bc.cuh"

#include <algorithm>

namespace rt3d {

namespace {

__global__ void sph_diffusion_bc_kernel(int nr, int nt, int np, int nl, double rc0, double rc1,
                                        double r_in, const double *__restrict__ chi,
                                        const double *__restrict__ B, double *__restrict__ I_face,
                                        double *__restrict__ grad) {
    const long long nf = (long long)nt * np, total = nf * nl;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long v0 = i * nr;  // (l, f) -> the innermost cell of that column
        if (nr < 2) {
            grad[i] = 0.0;
            I_face[i] = B[v0];
            continue;
        }
        const double dtau = __dmul_rn(__dmul_rn(0.5, __dadd_rn(chi[v0], chi[v0 + 1])),
                                      __dsub_rn(rc1, rc0));
        const double g = __ddiv_rn(__dsub_rn(B[v0], B[v0 + 1]), dtau);
        grad[i] = g;
        I_face[i] = __dadd_rn(B[v0], __dmul_rn(__dmul_rn(chi[v0], __dsub_rn(rc0, r_in)), g));
    }
}

__global__ void sph_entry_kernel(SphEntryParams p, const double *__restrict__ face, double I_face,
                                 const double *__restrict__ grad, double *__restrict__ I0,
                                 int *__restrict__ ident) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < p.nrays;
         r += (long long)gridDim.x * blockDim.x) {
        ident[r] = (int)r;
        if (p.ray_kind[r] != 2) {
            I0[r] = 0.0;
            continue;
        }
        const int v = p.ray_launch[r], o = p.ray_angle[r], f = p.ray_face[r];
        const int ir = v % p.nr, it = (v / p.nr) % p.nt, ip = v / (p.nr * p.nt);
        // the line through the launch cell's centre, and where it leaves the
        // core sphere (the larger root of |P + t d| = r_in)
        const double P0 = __dmul_rn(__dmul_rn(p.rc[ir], p.stc[it]), p.cpc[ip]);
        const double P1 = __dmul_rn(__dmul_rn(p.rc[ir], p.stc[it]), p.spc[ip]);
        const double P2 = __dmul_rn(p.rc[ir], p.ctc[it]);
        const double d0 = p.dir[3 * o], d1 = p.dir[3 * o + 1], d2 = p.dir[3 * o + 2];
        const double b = __dadd_rn(__dadd_rn(__dmul_rn(P0, d0), __dmul_rn(P1, d1)), __dmul_rn(P2, d2));
        const double pp = __dadd_rn(__dadd_rn(__dmul_rn(P0, P0), __dmul_rn(P1, P1)), __dmul_rn(P2, P2));
        const double dc = __dsub_rn(__dmul_rn(b, b), __dsub_rn(pp, __dmul_rn(p.r_in, p.r_in)));
        const double t0 = __dadd_rn(-b, __dsqrt_rn(fmax(dc, 0.0)));
        const double q0 = __dadd_rn(P0, __dmul_rn(t0, d0)), q1 = __dadd_rn(P1, __dmul_rn(t0, d1)),
                     q2 = __dadd_rn(P2, __dmul_rn(t0, d2));
        const double mu = __ddiv_rn(
            __dadd_rn(__dadd_rn(__dmul_rn(q0, d0), __dmul_rn(q1, d1)), __dmul_rn(q2, d2)), p.r_in);
        I0[r] = __dadd_rn(face ? face[f] : I_face, __dmul_rn(mu, grad[f]));
    }
}

}  // namespace

cudaError_t launch_sph_diffusion_bc(int nr, int nt, int np, int nl, double rc0, double rc1,
                                    double r_in, const double *chi, const double *B,
                                    double *I_face, double *grad, cudaStream_t s) {
    const long long total = (long long)nt * np * nl;
    const long long blocks = std::min<long long>((total + 255) / 256, 65536);
    sph_diffusion_bc_kernel<<<(unsigned)blocks, 256, 0, s>>>(nr, nt, np, nl, rc0, rc1, r_in, chi,
                                                            B, I_face, grad);
    return cudaGetLastError();
}

cudaError_t launch_sph_entry(const SphEntryParams &p, const double *face, double I_face,
                             const double *grad, double *I0, int *ident, cudaStream_t s) {
    if (p.nrays <= 0) return cudaSuccess;
    const long long blocks = std::min<long long>((p.nrays + 255) / 256, 65536);
    sph_entry_kernel<<<(unsigned)blocks, 256, 0, s>>>(p, face, I_face, grad, I0, ident);
    return cudaGetLastError();
}

}  // namespace rt3d
