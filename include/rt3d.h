/*
 * rt3d.h -- C ABI of the GB300 (sm_103a) long-characteristics 3D radiative
 * transfer library: formal solution, non-local Lambda* band and
 * operator-splitting (ALI) solver of Hauschildt & Baron, "A 3D radiative
 * transfer framework XII" (arXiv:2102.01734).
 *
 * Problem (Sec. 2.1, Eq. 1; Sec. 2.2, Eqs. frmsol, alisol, alodef, alo):
 *   n . grad I = chi (S - I),  J = Lambda S,  S = (1 - eps) J + eps B,
 *   [1 - Lambda*(1 - eps)] (J_new - J_old) = J_FS - J_old.
 *
 * Grid: a Cartesian box of nx * ny * nz unit voxels, periodic in x and y;
 * z = 0 is the inner (bottom) boundary layer, z = nz-1 the outer (top) one
 * (Sec. 3.1). Every voxel holds one value of each quantity (Sec. 2).
 *
 * Layouts. Every per-voxel array is double[N], N = nx*ny*nz, x fastest:
 * v = x + nx*(y + ny*z). Lambda* arrays are double[27][N] (offset-major):
 * element [d][v] = dJ_v / dS_{v+d}, with d = (dx+1) + 3(dy+1) + 9(dz+1),
 * dx,dy periodic, and 0 where v+d lies outside the box in z. Face arrays are
 * double[ny][nx] (index x + nx*y).
 *
 * Pointers. Every array argument may be host or device memory; the library
 * tells them apart with cudaPointerGetAttributes and stages host arrays
 * through device buffers owned by the grid (copies on the grid's stream).
 * The caller owns all arrays it passes; the library owns the grid, its
 * geometry cache and its work buffers. Calls on one grid are not thread
 * safe. All work is issued on the stream given in the descriptor; a call
 * returns after its results are complete (it synchronises that stream).
 *
 * Errors. Every entry point returns an rt3d_status and never aborts;
 * rt3d_last_error() gives a thread-local message for the last failure.
 */
#ifndef RT3D_H
#define RT3D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rt3d_grid rt3d_grid; /* opaque, library-owned */

typedef enum {
    RT3D_OK = 0,
    RT3D_EINVAL = 1,         /* bad descriptor, size or argument */
    RT3D_ENOMEM = 2,         /* device or host allocation failed */
    RT3D_ECUDA = 3,          /* a CUDA call failed */
    RT3D_ENOTCONVERGED = 4,  /* iteration cap reached; J holds the last iterate */
    RT3D_ETIMEOUT = 5,       /* reserved for a bounded device-side wait that ran out;
                                no kernel of this library spins on the device */
    RT3D_ENUMERIC = 6        /* NaN/Inf met in a residual or change */
} rt3d_status;

enum {
    RT3D_CARTESIAN_PERIODIC_XY = 0, /* n = (nx, ny, nz) unit voxels, periodic in x, y */
    RT3D_SPHERICAL = 1              /* n = (nr, ntheta, nphi) cells between r_in and r_out
                                       (log-spaced in r, uniform in theta and phi,
                                       periodic in phi); voxel v = ir + nr (it + nt ip) */
};
enum { RT3D_LINEAR = 0, RT3D_PARABOLIC = 1 };
enum {
    RT3D_ACCEL_NONE = 0,  /* ALI: J += [1 - Lambda*(1-eps)]^-1 (J_FS - J) */
    RT3D_ACCEL_KRYLOV = 1 /* FGMRES on (1 - Lambda(1-eps)) J = Lambda(eps B) + J_bc,
                             right-preconditioned by [1 - Lambda*(1-eps)]^-1 (the
                             same OS operator; same fixed point as the ALI) */
};
enum {
    RT3D_FP64 = 0,             /* formal solution and ALI in FP64 */
    RT3D_FP32_FS_FP64_ALI = 1, /* FP32 formal solution, FP64 ALI/residual, FP64 refinement */
    RT3D_FP32_FS_FF_REFINE = 2 /* as RT3D_FP32_FS_FP64_ALI, but the Krylov solve's
                                  refinement residuals come from the float-float
                                  formal solution (rt3d_formal_solution_ff) and only
                                  the residual that certifies J from an FP64 formal
                                  solution (the plain ALI's defect correction keeps
                                  FP64 residuals) */
};

/* Residency of the spherical geometry cache (Sec. 4.3: the LargeGPU mode keeps
 * the tracking caches on the GPU; the SmallGPU mode keeps them in host memory
 * and moves them to the GPU solid angle by solid angle). The ray tables
 * (offset, length, kind, core face: 20 bytes per ray, plus the launch voxel and
 * angle) stay on the device in every mode; these modes place the per-segment
 * records (24 bytes per segment, the bulk of the cache). */
enum {
    RT3D_CACHE_DEVICE = 0,        /* records in device memory, one launch per
                                     formal solution (LargeGPU) */
    RT3D_CACHE_HOST_STREAMED = 1, /* records in pinned host memory, cut at solid
                                     angle boundaries into chunks of at most
                                     stream_bytes; each formal solution copies
                                     chunk c into device buffer c % 2 on a copy
                                     stream while the kernel integrates chunk
                                     c - 1 (SmallGPU) */
    RT3D_CACHE_HOST_MAPPED = 2,   /* records in pinned, mapped host memory that
                                     the kernels read in place over the host link,
                                     one launch per chunk */
    RT3D_CACHE_HOST_CHORDS = 3    /* split by precision: the 16-byte records the
                                     FP32 kernels read stay on the device, the
                                     8-byte FP64 chords (read only by FP64 formal
                                     solutions) live in pinned host memory and are
                                     streamed as in RT3D_CACHE_HOST_STREAMED, in
                                     chunks of at most stream_bytes of chords */
};

typedef struct {
    int geometry;     /* RT3D_CARTESIAN_PERIODIC_XY or RT3D_SPHERICAL */
    int n[3];         /* Cartesian: nx, ny, nz with 4 <= nx, ny <= 2047,
                         1 <= nz <= 1023; spherical: nr, ntheta, nphi with
                         nr >= 1, ntheta >= 2, nphi >= 4, each <= 4096;
                         always 4 n[0] n[1] n[2] < 2^31 */
    int ntheta, nphi; /* direction set: mu_i = -1 + (2i+1)/ntheta,
                         phi_j = (2j+1) pi / nphi, weight 1/(ntheta nphi) */
    int interp;       /* RT3D_LINEAR or RT3D_PARABOLIC source interpolation */
    int precision;    /* RT3D_FP64, RT3D_FP32_FS_FP64_ALI or RT3D_FP32_FS_FF_REFINE */
    int nlambda;      /* reserved: must be 0 or 1 */
    void *cuda_stream;/* cudaStream_t to run on, or NULL for the legacy stream */
    int accel;        /* rt3d_solve iteration: RT3D_ACCEL_NONE (plain ALI, Eq. alo
                         with Jacobi OS solves) or RT3D_ACCEL_KRYLOV */
    double r_in, r_out; /* RT3D_SPHERICAL: core and outer radius (0 < r_in < r_out) */
    int cache;        /* RT3D_CACHE_*; anything but RT3D_CACHE_DEVICE needs
                         RT3D_SPHERICAL (the Cartesian cache is one template
                         per angle) */
    long long stream_bytes; /* host modes: the largest chunk of what is streamed
                         (24 bytes a segment; 8 in RT3D_CACHE_HOST_CHORDS), 0 for
                         1 GiB; a solid angle is never split, so a chunk holds
                         at least one angle. The streaming modes hold two
                         device buffers of the largest chunk; while
                         the grid is built, a staging buffer of up to 16 GiB (a
                         quarter of the free memory, at least one chunk) is
                         held as well */
} rt3d_grid_desc;

/* Boundary intensities (Sec. 3.1: I = 0 incoming at the outer boundary; the
 * inner boundary is given by the caller, e.g. I = B of the entered voxel, or
 * the LTE diffusion condition of the paper's test cases, Sec. 3.1 and 3.2).
 * A characteristic with mu < 0 enters through the top face, one with mu > 0
 * through the bottom face, at the centre of face cell (x0, y0). A non-NULL
 * face array (double[ny][nx], host or device) overrides the scalar. */
typedef struct {
    double I_top;
    double I_bottom;
    const double *I_top_face;
    const double *I_bottom_face;
    double I_irr;     /* RT3D_SPHERICAL: irradiation entering the outer sphere at
                         points with x > 0 along directions with d_x < 0 */
    const double *I_bottom_grad; /* nullable double[ny][nx] (spherical grids:
                         [nphi][ntheta]): the diffusion inner boundary, where a
                         characteristic with direction cosine mu > 0 enters with
                         I = I_bottom (or its face value) + mu I_bottom_grad, the
                         gradient being dB/dtau at the boundary with tau the vertical
                         (radial) optical depth growing inward (rt3d_diffusion_bc) */
} rt3d_bc;
/* On a spherical grid I_top (or I_top_face, unused) is the intensity entering
 * the outer sphere outside the irradiated part, I_bottom / I_bottom_face
 * ([nphi][ntheta], index it + nt ip) the intensity leaving the core into the
 * first cell of a characteristic; with I_bottom_grad a characteristic leaves
 * the core with I_bottom + mu I_bottom_grad, mu the cosine between it and the
 * core's outward normal at its entry point (computed per characteristic on
 * the device at every formal solution; 12 bytes per characteristic,
 * allocated on first use). */

typedef struct {
    int iterations;     /* ALI iterations of the main loop */
    int fs_fp32;        /* formal solutions done in FP32 */
    int fs_fp64;        /* formal solutions done in FP64 */
    int jacobi_sweeps;  /* Jacobi sweeps of all OS solves */
    double rel_change;  /* last max_v |dJ_v| / |J_v| */
    double residual64;  /* max_v |J_FS64(S(J))_v - J_v| / |J_v| of the returned J
                           (FP64 formal solution; 0 if not computed) */
    double est_error;   /* estimated max relative error of the returned J
                           (-1: not estimated, e.g. the cap was reached before
                           a refinement residual) */
    double seconds;     /* wall time of the call */
    double fs32_ms;     /* summed device time of the FP32 formal-solution kernels
                           (CUDA events on the grid's stream) */
    double fs64_ms;     /* same for the FP64 formal-solution kernels */
    long long launches; /* kernels launched by the call */
    int fs_ff;          /* float-float formal solutions (RT3D_FP32_FS_FF_REFINE) */
    double fsff_ms;     /* their summed device time */
    int rounds;         /* Krylov solve: refinement rounds (residual, then an
                           FGMRES cycle unless the residual certified J);
                           the first 16 are recorded below */
    int round_fp64[16];    /* the formal solution of the round's residual:
                              0 FP32, 1 FP64, 2 float-float */
    int round_fs[16];      /* formal solutions of the round's FGMRES cycle */
    double round_res[16];  /* the round's residual max_v |r_v| / |J_v| */
    double round_est[16];  /* estimated error at that residual (-1: none) */
    int fs_lstar;          /* FP32 formal solutions that built Lambda* (counted
                              in fs_fp32) */
    double fs32_lstar_ms;  /* their summed device time (included in fs32_ms) */
} rt3d_solve_stats;

/* Ray-bundle shape of the FP32 formal solution without Lambda* (not in the
 * paper, which maps characteristics to OpenACC gangs and vectors, Sec. 5). */
typedef struct {
    int block;            /* threads per block: 64, 128 or 256 */
    int rays_per_thread;  /* characteristics per thread: 1; 2 (face cells
                             (x, y) and (x, y + 1), y even, integrated together
                             in packed FP32x2 arithmetic); or 4 (face cells
                             (x, y .. y + 3), y a multiple of 4, two packed
                             pairs, the J contributions of successive points
                             summed in FP32 per voxel while the voxel stays
                             inside the block of voxels a warp's
                             characteristics occupy, then reduced in FP64;
                             FP32 grids of at most 2^27 voxels) */
    int widen;            /* FP32 contribution to FP64 for the reduction: 0 the
                             conversion instruction, 1 integer moves, 2 both
                             (one characteristic per thread: alternating from
                             point to point; two: the second by integer
                             moves; four: as 0) */
    int branchless;       /* 1: the parabolic correction is evaluated without
                             a branch (multiplied by its blend weight 0 where
                             the linear form applies); two characteristics
                             per thread always evaluate it so */
} rt3d_fs_shape;

#define RT3D_FS_TUNE_SHAPES 8

typedef struct {
    int nangles;              /* ntheta * nphi */
    int kmax;                 /* longest characteristic, points */
    long long segments;       /* ray-segment updates per formal solution:
                                 nx*ny * sum over angles of points per ray */
    long long device_bytes;   /* device memory held by the grid */
    rt3d_fs_shape fs_shape;   /* ray-bundle shape of the FP32 formal solution
                                 without Lambda* (block 0: not chosen yet) */
    float fs_tune_ms[RT3D_FS_TUNE_SHAPES]; /* kernel time of each candidate
                                 shape (rt3d_fs_tune_shape order) at the last
                                 autotuning; 0 if not tuned */
    int sm_count;             /* streaming multiprocessors of the grid's device
                                 (cudaDevAttrMultiProcessorCount), which sizes the
                                 library's capped launches */
    int cache;                /* RT3D_CACHE_* of the grid */
    long long host_bytes;     /* pinned host memory held by the grid (the
                                 per-segment records, or the FP64 chords, in the
                                 host modes) */
    int cache_chunks;         /* host modes: chunks of solid angles a formal
                                 solution goes through (1 on the device) */
} rt3d_grid_info;

/* Creates a grid: builds the direction set (host, FP64) and traces one
 * characteristic per solid angle on the device (Sec. 4, the tracker; the
 * geometry cache of Sec. 4.1). All nx*ny characteristics of an angle are
 * integer translates of that one. Returns RT3D_EINVAL for sizes outside the
 * limits above, a zero direction component along z (impossible with this
 * direction set), or a Lambda* window longer than 9 points. A spherical grid
 * builds its cache of long characteristics on the device (one warp per solid
 * angle); in the host cache modes each chunk of angles is built into a device
 * buffer and copied to pinned host memory. RT3D_ENOMEM when the device cache
 * does not fit the free device memory, or the host records would take more
 * than half of the host memory available to the process (MemAvailable, and
 * the cgroup limit where one is set). */
rt3d_status rt3d_grid_create(const rt3d_grid_desc *desc, rt3d_grid **out);

/* Releases the grid and all device memory it holds. NULL is ignored. */
void rt3d_grid_destroy(rt3d_grid *grid);

/* Solver of the OS step [1 - Lambda*(1 - eps)] dJ = r (Sec. 4: the OS
 * iteration by Jacobi, Gauss-Seidel or BiCGStab) used by every call of the
 * grid that solves it: rt3d_os_solve, rt3d_ali_step, rt3d_solve (its ALI, and
 * its Krylov preconditioner), rt3d_line_solve.
 *   RT3D_OS_JACOBI (default): Jacobi sweeps from dJ = r/diag.
 *   RT3D_OS_GAUSS_SEIDEL: eight-colour Gauss-Seidel sweeps from dJ = r/diag,
 *     colours c = (x&1) + 2(y&1) + 4(z&1) in order, every voxel of a colour
 *     from the values its neighbours hold before that colour's update; the
 *     same stop test as Jacobi, once per sweep of all colours.
 *   RT3D_OS_BICGSTAB: BiCGStab (van der Vorst 1992) from dJ = 0, stopped when
 *     ||A dJ - r||_2 <= tol ||r||_2, at a breakdown (omega = 0), or after the
 *     cap; its iterations are counted as sweeps, and a cap given in sweeps by
 *     the library (50 for the ALI and the preconditioner) allows half as
 *     many iterations (two matrix products each).
 * The batched solve (rt3d_solve_batched) and rt3d_os_solve_noalloc always use
 * Jacobi. RT3D_EINVAL for NULL or another value. */
#define RT3D_OS_JACOBI 0
#define RT3D_OS_GAUSS_SEIDEL 1
#define RT3D_OS_BICGSTAB 2
rt3d_status rt3d_grid_set_os_solver(rt3d_grid *grid, int solver);

/* Drops the grid's Lambda* band (Sec. 4: built in the first iteration of a
 * solve and kept while chi and eps are unchanged), so that the next solve or
 * ALI step builds it again from its own chi and eps. RT3D_EINVAL for NULL. */
rt3d_status rt3d_grid_invalidate_lstar(rt3d_grid *grid);

rt3d_status rt3d_grid_get_info(const rt3d_grid *grid, rt3d_grid_info *info);

/* Candidate i (0 <= i < RT3D_FS_TUNE_SHAPES) of the autotuner of the FP32
 * formal solution without Lambda*. RT3D_EINVAL for another i or out = NULL. */
rt3d_status rt3d_fs_tune_shape(int i, rt3d_fs_shape *out);

/* Sets the grid's ray-bundle shape of the FP32 formal solution without
 * Lambda*. shape = NULL: autotune at the next such formal solution (the
 * default for a new grid): every candidate of rt3d_fs_tune_shape that the
 * grid supports is launched once on that call's input, timed with CUDA
 * events on the grid's stream, and the fastest is kept (an unsupported
 * candidate records 0 ms in rt3d_grid_info). The result does not depend on the shape beyond
 * FP64 reduction order (both widenings are exact for normal FP32 values;
 * integer widening maps an FP32 zero or subnormal contribution to at most
 * 1.2e-38 in magnitude). RT3D_EINVAL for a shape outside the ranges of
 * rt3d_fs_shape, or four characteristics per thread on a grid that does
 * not support them. */
rt3d_status rt3d_grid_set_fs_shape(rt3d_grid *grid, const rt3d_fs_shape *shape);

/* The traced characteristic of solid angle `angle` from face cell (0,0):
 * points K (in/out: capacity on input), voxel indices vox[K] and FP64 chords
 * len[K], in host memory. Tracer rule: crossing parameters (m - 1/2)/|d_x|,
 * (m - 1/2)/|d_y| and m/|mu|, each one IEEE division; ties advance all tied
 * axes; chord = difference of consecutive crossing parameters. */
rt3d_status rt3d_grid_template(const rt3d_grid *grid, int angle, int *K, int32_t *vox,
                               double *len);

/* One characteristic of the spherical grid's cache: ray `index` (0-based) of
 * solid angle `angle`: points K (in/out capacity), cells vox[K], FP64 chords
 * len[K], the voxel that launched it, and its boundary kind (0 outer sphere,
 * 1 outer sphere irradiated, 2 core). Host memory. The same in every cache
 * residency (RT3D_CACHE_*). Returns RT3D_EINVAL past the last ray of the
 * angle. */
rt3d_status rt3d_grid_sph_ray(const rt3d_grid *grid, int angle, int index, int *K, int32_t *vox,
                              double *len, int *launch, int *kind);

/* Formal solution J = Lambda S (Eq. frmsol) over all solid angles, in the
 * grid's precision (FP64, or FP32 for RT3D_FP32_FS_FP64_ALI and
 * RT3D_FP32_FS_FF_REFINE; results are returned as double either way):
 *   J_v = sum_Omega w (sum_{k in v} l_k I_k) / (sum_{k in v} l_k),
 *   I_k = exp(-dtau) I_{k-1} + alpha S_{k-1} + beta S_k + gamma S_{k+1}.
 * chi > 0 (per unit length) and S: double[N]. J_out: double[N] (written).
 * lstar_out: nullable double[27][N]; when given, the passage-local Lambda*
 * band (Sec. 4, "non-local Lambda*") is built as well. bc: nullable (zero
 * incoming intensity). */
rt3d_status rt3d_formal_solution(rt3d_grid *grid, const double *chi, const double *S,
                                 const rt3d_bc *bc, double *J_out, double *lstar_out);

/* Bottom-face arrays of the LTE diffusion inner boundary (Sec. 3.1, 3.2
 * test cases) for nlambda stacked grids of the Cartesian grid's shape: per
 * column f = x + nx y and grid l,
 *   grad[l][f]   = (B[l][0][f] - B[l][1][f]) / (1/2 (chi[l][0][f] + chi[l][1][f])),
 *   I_face[l][f] = B[l][0][f] + 1/2 chi[l][0][f] grad[l][f],
 * the one-sided dB/dtau over the unit spacing of the two innermost layer
 * centres (trapezoidal optical depth) and B carried linearly to the bottom
 * face, half a voxel below the innermost centre, where the characteristics
 * enter; nz = 1 gives grad = 0 and I_face = B[l][0][f]. Pass them as
 * rt3d_bc's I_bottom_face and I_bottom_grad. chi, B: double[nlambda][N];
 * I_face, grad: double[nlambda][ny][nx], written. On a spherical grid the
 * faces are the core's, double[nlambda][nphi][ntheta] (index it + nt ip):
 * dB/dtau = (B0 - B1) / (1/2 (chi0 + chi1) (rc1 - rc0)) between the two
 * innermost shells (centres rc_i = sqrt(r_e[i] r_e[i+1])) and
 * I_face = B0 + chi0 (rc0 - r_in) dB/dtau, B carried down to the core sphere
 * (nr = 1: grad = 0). All four must be memory of the grid's device (or
 * managed memory); the kernel runs on the grid's stream, which the call does
 * not synchronise. RT3D_EINVAL for a NULL argument, nlambda < 1 or a pointer
 * that is not device memory. */
rt3d_status rt3d_diffusion_bc(rt3d_grid *grid, int nlambda, const double *chi, const double *B,
                              double *I_face, double *grad);

/* The formal solution without Lambda* in float-float arithmetic (not in the
 * paper: FP64-class accuracy, about 1e-13 relative, on the FP32 pipe; GB300's
 * FP64 rate is about 1/64 of its FP32 rate). Same arguments, layouts and
 * error behaviour as rt3d_formal_solution without lstar_out; grids of any
 * precision and geometry. The first call allocates the split replicated
 * (chi, S) (64 bytes per voxel) and, on a Cartesian grid, the split step
 * records (16 bytes per cached point); a spherical grid splits its FP64
 * chords per point instead (its records already hold the J weight as a
 * float-float pair) and reads them like the FP64 formal solution, in every
 * cache residency. */
rt3d_status rt3d_formal_solution_ff(rt3d_grid *grid, const double *chi, const double *S,
                                    const rt3d_bc *bc, double *J_out);

/* OS linear system of Eq. alo for the correction dJ = J_new - J_old:
 * [1 - Lambda*(1 - eps)] dJ = r, by the grid's OS solver (Sec. 4, OS
 * iteration; rt3d_grid_set_os_solver). Jacobi and Gauss-Seidel: dJ^0 = r /
 * diag; stop when max|dJ^{m+1} - dJ^m| <= tol * max|dJ^{m+1}| or after
 * max_sweeps (1..256) sweeps. BiCGStab: from dJ = 0, stop when
 * ||A dJ - r||_2 <= tol ||r||_2 or after max_sweeps iterations. lstar:
 * double[27][N] as written by rt3d_formal_solution; eps, r, dJ_out:
 * double[N]. sweeps_out (nullable, host) receives the sweeps (iterations). */
rt3d_status rt3d_os_solve(rt3d_grid *grid, const double *lstar, const double *eps,
                          const double *r, double *dJ_out, int max_sweeps, double tol,
                          int *sweeps_out);

/* One ALI iteration (Eqs. alisol, alo): S = (1-eps) J + eps B; J_FS =
 * Lambda S; Jacobi solve (<= 50 sweeps, relative tolerance 1e-3) of
 * [1 - Lambda*(1-eps)] dJ = J_FS - J; J += dJ. Lambda* is built on the first
 * call after grid creation or after chi or eps change (compared by
 * content). rel_change_out (nullable, host): max_v |dJ_v| / |J_v|. */
rt3d_status rt3d_ali_step(rt3d_grid *grid, const double *chi, const double *eps,
                          const double *B, const rt3d_bc *bc, double *J_inout,
                          double *rel_change_out);

/* Solves for J from J_inout until the estimated relative error of J is below
 * tol. chi, eps, B: double[N]; J_inout: double[N] (start, then the result).
 * RT3D_ACCEL_NONE (the paper's ALI, Eq. alo): iterations until the last
 * change times rho/(1-rho) (rho the observed contraction) is below tol; in
 * the mixed precisions FP32 iterations until the change stagnates, then
 * defect correction with FP64 formal solutions (residual r64 =
 * J_FS64(S(J)) - J, correction from the homogeneous FP32 ALI) until the FP64
 * residual certifies the result. RT3D_ACCEL_KRYLOV: refinement rounds, each
 * a residual r = J_FS(S(J)) - J and one FGMRES cycle on
 * (1 - Lambda(1-eps)) delta = r preconditioned by the OS solve, J += delta;
 * the error after a round is estimated as (|delta|/|r| of the previous round)
 * times the residual, and an FP64 residual meeting tol certifies J (FP32
 * residuals first in the mixed precisions; float-float ones with
 * RT3D_FP32_FS_FF_REFINE; FP64 throughout in RT3D_FP64). max_iter caps the
 * ALI iterations or the FGMRES steps. Returns RT3D_ENOTCONVERGED with
 * J_inout holding the last iterate when the cap is hit, RT3D_ENUMERIC when a
 * residual or change is not finite. stats: nullable (host). */
rt3d_status rt3d_solve(rt3d_grid *grid, const double *chi, const double *eps, const double *B,
                       const rt3d_bc *bc, double *J_inout, double tol, int max_iter,
                       rt3d_solve_stats *stats);

typedef struct {
    int nlambda;            /* wavelengths in the batch */
    int converged;          /* wavelengths certified converged */
    int iterations;         /* batched ALI iterations (graph replays) */
    int graph_replays;      /* replays of the captured iteration graph */
    long long fs_lambda32;  /* single-wavelength FP32 formal solutions done */
    long long fs_lambda64;  /* single-wavelength FP64 formal solutions done */
    double max_est_error;   /* largest estimated relative error of a returned J */
    double max_residual64;  /* largest certifying FP64 residual */
    double batch_ms;        /* device time of the batched iterations */
    double fs32_ms, fs64_ms;
    double seconds;
    long long launches;
    long long fs_lambda_ff; /* single-wavelength float-float formal solutions done */
    double fsff_ms;
    rt3d_fs_shape fs_shape; /* shape of the batched FP32 formal solution (autotuned
                               on the grid's first batched call, one
                               characteristic per thread) */
    float fs_tune_ms[RT3D_FS_TUNE_SHAPES]; /* its candidates' times (0: not
                               timed: two characteristics per thread) */
    int recaptures;         /* re-captures of the iteration graph with fewer
                               wavelengths (retired ones leave the launches) */
    long long fs_batched;   /* single-wavelength FP32 formal solutions inside the
                               batched iterations (of fs_lambda32; batch_ms is their
                               phase's device time) */
} rt3d_batch_stats;

/* Batched wavelengths (Sec. 4.1: the geometry is the same for all wavelength
 * points): n_lambda independent problems on the grid's geometry. chi, eps, B
 * and J_inout are double[n_lambda][N] (wavelength-major); face arrays of bc,
 * when given, are double[n_lambda][ny][nx]. Phase 1 iterates the ALI of all
 * wavelengths together in FP32 (one captured CUDA graph per iteration,
 * replayed; a wavelength retires on the device when its estimated error is
 * below max(tol, 1e-6) or its changes stagnate); phase 2 refines and certifies
 * every wavelength with rt3d_solve's Krylov scheme (float-float refinement
 * residuals with RT3D_FP32_FS_FF_REFINE, an FP64 residual certifying). The
 * batched formal solution's shape is autotuned on the grid's first batched
 * call (stats->fs_shape).
 * status_out (nullable, host int[n_lambda]) receives RT3D_OK,
 * RT3D_ENOTCONVERGED or RT3D_ENUMERIC per wavelength. Returns
 * RT3D_ENOTCONVERGED if any wavelength is not certified. Device memory grows
 * by about (8 * 8 + 4 * 26 + 4 * 16) n_lambda N bytes on first use. */
rt3d_status rt3d_solve_batched(rt3d_grid *grid, int nlambda, const double *chi,
                               const double *eps, const double *B, const rt3d_bc *bc,
                               double *J_inout, double tol, int max_iter, int *status_out,
                               rt3d_batch_stats *stats);

typedef struct {
    int iterations;         /* line ALI iterations done */
    int fs_lambda;          /* single-wavelength formal solutions done, FP32 and FP64
                               (those of the first iteration also build Lambda*) */
    int jacobi_sweeps;      /* Jacobi sweeps of all OS solves */
    double rel_change;      /* last max_v |dJbar_v| / |Jbar_v| */
    double est_error;       /* rel_change * rho / (1 - rho), rho the observed
                               contraction (-1 before the second iteration) */
    double seconds;         /* wall time of the call */
    double fs64_ms;         /* summed device time of the FP64 formal-solution kernels */
    long long launches;     /* kernels launched by the call */
    int fs_lambda32;        /* of fs_lambda, those in FP32 (mixed grids) */
    double fs32_ms;         /* summed device time of the FP32 formal-solution kernels */
    double residual64;      /* mixed grids: max_v |Jbar_FS64(S(Jbar))_v - Jbar_v| / |Jbar_v|
                               of the last FP64 residual (0 on an RT3D_FP64 grid) */
} rt3d_line_stats;

/* Line transfer (Sec. 2, with Eq. alisol: J weighted by the line profile
 * phi across the line, Jbar = int J_lambda phi_lambda dlambda). nlambda
 * wavelengths of one spectral line share the source function
 *   S = (1 - eps) Jbar + eps B,   Jbar = sum_l wphi[l] J_l,
 * where J_l is the formal solution (Eq. frmsol) with the opacity
 * scale[l] * chi and the boundary intensities bc (the same at every
 * wavelength). wphi[l] is the quadrature weight times the profile value
 * (normally summing to 1). Iterates the ALI of Eq. alo with the
 * profile-averaged band Lbar* = sum_l wphi[l] Lambda*_l, built in the call's
 * first iteration:
 *   Jbar_FS = sum_l wphi[l] Lambda_l S;  Jacobi solve (<= 50 sweeps,
 *   relative tolerance 1e-3) of [1 - Lbar*(1 - eps)] dJ = Jbar_FS - Jbar;
 *   Jbar += dJ,
 * until the last change times rho/(1 - rho) (rho the observed contraction,
 * from the second iteration on) is below tol, or for max_iter iterations
 * (max_iter = 1: exactly one iteration, returning RT3D_ENOTCONVERGED). On an
 * RT3D_FP64 grid every formal solution is FP64. On the mixed grids the
 * iterations use FP32 formal solutions (the first also building the band)
 * until the estimate falls below max(tol, 1e-6) or the changes stop
 * decreasing (the FP32 rounding floor); then, as in rt3d_solve, defect
 * correction: an FP64 residual r = Jbar_FS64(S(Jbar)) - Jbar, a correction
 * from the homogeneous problem (1 - Lbar(1 - eps)) delta = r by the same
 * iteration with FP32 formal solutions (iterated to the relative accuracy that
 * brings the estimate to tol/2, between 1e-4 and 0.1), Jbar += delta, until
 * |delta| times its estimated relative accuracy is below tol; a last FP64
 * residual certifies the result (residual64). The OS coefficients follow the grid's precision, which
 * changes only the convergence rate.
 * chi, eps, B: double[N] (host or device); scale, wphi: HOST double[nlambda]
 * with scale[l] > 0 and wphi[l] >= 0, finite, sum of wphi > 0;
 * 1 <= nlambda <= 65536;
 * Jbar_inout: double[N] (start, then the result). Cartesian grids only
 * (RT3D_EINVAL for a spherical grid). The call leaves the line's band in the
 * grid: the next rt3d_ali_step or rt3d_solve rebuilds the continuum Lambda*.
 * The first call allocates 28 N + 28 doubles. Returns RT3D_ENOTCONVERGED
 * with Jbar_inout holding the last iterate when max_iter is reached,
 * RT3D_ENUMERIC when a change is not finite. stats: nullable (host). */
rt3d_status rt3d_line_solve(rt3d_grid *grid, int nlambda, const double *chi,
                            const double *scale, const double *wphi, const double *eps,
                            const double *B, const rt3d_bc *bc, double *Jbar_inout,
                            double tol, int max_iter, rt3d_line_stats *stats);

/* Allocation-free Jacobi OS solve. No counterpart in the paper: this is a
 * library service for callers that cannot allocate device memory, such as a
 * host application whose device memory is entirely pre-reserved by its own
 * pool allocator, or a time-critical loop that must not call cudaMalloc or
 * cudaFree (both synchronise the device).
 *
 * Computes the same result as rt3d_os_solve on an RT3D_FP64 grid
 * ([1 - Lambda*(1-eps)] dJ = r by Jacobi sweeps from dJ^0 = r/diag, stop when
 * max|dJ^{m+1} - dJ^m| <= tol max|dJ^{m+1}| or after max_sweeps, 1..256)
 * without a grid and without allocating: the caller passes device arrays
 * lstar double[27][N] (layout of rt3d_formal_solution), eps, r and dJ_out
 * double[N], N = nx*ny*nz <= RT3D_NOALLOC_MAX_VOXELS (host pointers, larger
 * grids or nx, ny < 4 return RT3D_EINVAL). The only scratch is a fixed
 * file-scope device array of 2 * RT3D_NOALLOC_MAX_VOXELS doubles (1 MiB,
 * held by every GPU that loads the library until the process exits).
 * The arrays must be device memory of the current device (or managed
 * memory); another device's arrays return RT3D_EINVAL. The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current and keeps it for the process; make that first call
 * before any stream capture. A cudaDeviceReset (or another destruction of
 * the device's primary context) while the library is loaded is not
 * supported. All calls share the array: calls whose work overlaps on the
 * GPU race and must be serialised. Work runs on cuda_stream (NULL: legacy
 * stream); every call synchronises that stream before it returns (it reads
 * the sweep count back), and returns RT3D_EINVAL without launching anything
 * while the stream is being captured. sweeps_out (nullable, host) receives
 * the number of sweeps. */
#define RT3D_NOALLOC_MAX_VOXELS 65536
rt3d_status rt3d_os_solve_noalloc(int nx, int ny, int nz, const double *lstar,
                                  const double *eps, const double *r, double *dJ_out,
                                  int max_sweeps, double tol, int *sweeps_out,
                                  void *cuda_stream);

/* Message of the last failed call on this thread ("" if none). */
const char *rt3d_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RT3D_H */
