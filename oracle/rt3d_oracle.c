/*
 * rt3d_oracle.c -- plain, slow FP64 CPU oracle of the long-characteristics
 * formal solution, the non-local Lambda* band and the operator-splitting (ALI)
 * iteration described in Hauschildt & Baron, "A 3D radiative transfer
 * framework XII: many-core, vector and GPU methods" (arXiv:2102.01734):
 *   Sec. 2.1 (static RTE, Eq. 1), Sec. 2.2 (J = Lambda S, Eq. frmsol;
 *   Lambda iteration, Eq. alisol; operator splitting, Eqs. alodef and alo),
 *   Sec. 4 (tracker, formal solution, Lambda* in the first iteration, Jacobi
 *   OS solver) and the per-slot steps of the paper's Listing 1 (gather S and
 *   chi, dtau, alpha/beta/gamma, boundary fix-up, Lambda* data, Delta I).
 *
 * TEST INFRASTRUCTURE. Only the tests, __graft_entry__.smoke() and the CPU
 * legs of bench.py load this library. It shares no code, header or table with
 * the CUDA path; every formula below is written out independently.
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction,
 * so that traced crossing times are reproducible bit for bit).
 *
 * The paper refers the discretisation to its Papers I, III and IV and does not
 * print it. The readings used here (each also listed in the design notes):
 *  - voxel (x,y,z) is the unit cube [x,x+1)x[y,y+1)x[z,z+1); x,y periodic;
 *    z = 0 is the inner (bottom) boundary, z = nz the outer (top) one;
 *  - directions are midpoints, equally spaced in mu and phi, equal weights;
 *  - every solid angle has one characteristic per inflow-face voxel, starting
 *    at the face centre; points sit at chord midpoints;
 *  - dtau between consecutive points = 1/2 (chi_{k-1} l_{k-1} + chi_k l_k),
 *    with chi_0 l_0 = 0 and S_0 = S_1 at the boundary entry point;
 *  - linear / parabolic (Olson & Kunasz 1987) interpolation of S, linear on
 *    the last interval of a characteristic;
 *  - J_v = sum_Omega w_Omega (sum_{k in v} l_k I_k) / (sum_{k in v} l_k);
 *  - Lambda* row of v_k collects dI_k/dS_j over the passage-local window
 *    (the run of points ending at k+1 whose voxels lie in the 3x3x3
 *    neighbourhood of v_k).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------------------
 * Direction set: mu_i = -1 + (2i+1)/ntheta, phi_j = (2j+1) pi / nphi,
 * d = (sqrt((1-mu)(1+mu)) cos phi, sqrt((1-mu)(1+mu)) sin phi, mu),
 * w = 1/(ntheta nphi). "equally spaced in mu = cos(theta) and phi" (Sec. 3.1).
 * Angle index o = i * nphi + j.
 * ------------------------------------------------------------------------- */
void orc_directions(int nth, int nph, double *mu, double *phi, double *dir, double *w)
{
    for (int i = 0; i < nth; i++) {
        for (int j = 0; j < nph; j++) {
            int o = i * nph + j;
            double m = -1.0 + (double)(2 * i + 1) / (double)nth;
            double p = (double)(2 * j + 1) * M_PI / (double)nph;
            double s = sqrt((1.0 - m) * (1.0 + m));
            mu[o] = m;
            phi[o] = p;
            dir[3 * o + 0] = s * cos(p);
            dir[3 * o + 1] = s * sin(p);
            dir[3 * o + 2] = m;
            w[o] = 1.0 / (double)(nth * nph);
        }
    }
}

/* ---------------------------------------------------------------------------
 * Tracker for the Cartesian box periodic in x and y (Sec. 4: "setting up
 * the geometric paths through the grid for all solid angles").
 * Start at (x0+1/2, y0+1/2, z_in), z_in = nz if mu < 0 else 0. Crossing
 * parameters along the unit direction: the m-th x plane at (m - 1/2)/|d_x|,
 * likewise y, the m-th z plane at m/|mu|. Each is one IEEE division. Equal
 * crossing parameters advance all tied axes in one step. Chord = difference of
 * consecutive crossing parameters. Stops at the far z face.
 * Writes the wrapped linear voxel index v = x + nx (y + ny z) and the chord of
 * every point; returns the number of points K, or -1 (bad direction) or -2
 * (more than kmax points).
 * ------------------------------------------------------------------------- */
int orc_trace_cart(int nx, int ny, int nz, const double *d, int x0, int y0,
                   int kmax, int *vox, double *len)
{
    double ax = fabs(d[0]), ay = fabs(d[1]), az = fabs(d[2]);
    if (!(az > 0.0)) return -1;
    int sx = d[0] > 0.0 ? 1 : -1;
    int sy = d[1] > 0.0 ? 1 : -1;
    int sz = d[2] > 0.0 ? 1 : -1;
    int x = x0, y = y0, z = d[2] > 0.0 ? 0 : nz - 1;
    long mx = 1, my = 1, mz = 1;
    double tx = ax > 0.0 ? ((double)mx - 0.5) / ax : INFINITY;
    double ty = ay > 0.0 ? ((double)my - 0.5) / ay : INFINITY;
    double tz = (double)mz / az;
    double tprev = 0.0;
    int k = 0;
    for (;;) {
        double tn = tx < ty ? tx : ty;
        if (tz < tn) tn = tz;
        if (k >= kmax) return -2;
        vox[k] = x + nx * (y + ny * z);
        len[k] = tn - tprev;
        k++;
        tprev = tn;
        if (tx == tn) {
            mx++;
            tx = ((double)mx - 0.5) / ax;
            x += sx;
            if (x >= nx) x -= nx;
            if (x < 0) x += nx;
        }
        if (ty == tn) {
            my++;
            ty = ((double)my - 0.5) / ay;
            y += sy;
            if (y >= ny) y -= ny;
            if (y < 0) y += ny;
        }
        if (tz == tn) {
            if (mz == nz) break;
            mz++;
            tz = (double)mz / az;
            z += sz;
        }
    }
    return k;
}

/* Upper bound on the number of points of a characteristic (for buffers). */
int orc_kmax_cart(int nx, int ny, int nz, const double *d)
{
    (void)nx; (void)ny;
    double az = fabs(d[2]);
    double span = (double)nz / az;
    return nz + (int)(fabs(d[0]) * span) + (int)(fabs(d[1]) * span) + 8;
}

/* ---------------------------------------------------------------------------
 * Exponential integrals of the interval of optical depth u:
 *   e0 = 1 - exp(-u), e1 = u - e0, e2 = u^2 - 2 e1
 * (Olson & Kunasz 1987; e_n = int_0^u t^n exp(-(u - t)) dt). For u < 1/2 the
 * three are summed from their Taylor series to full FP64 precision, otherwise
 * evaluated in closed form with expm1.
 * ------------------------------------------------------------------------- */
void orc_e012(double u, double *e0, double *e1, double *e2)
{
    if (u < 0.5) {
        double term = u; /* u^n / n! at n = 1 */
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int n = 1; n <= 40; n++) {
            double sg = (n & 1) ? 1.0 : -1.0; /* (-1)^(n+1) */
            s0 += sg * term;
            if (n >= 2) s1 -= sg * term;
            if (n >= 3) s2 += 2.0 * sg * term;
            term = term * u / (double)(n + 1);
            if (term == 0.0) break;
        }
        *e0 = s0;
        *e1 = s1;
        *e2 = s2;
    } else {
        *e0 = -expm1(-u);
        *e1 = u - *e0;
        *e2 = u * u - 2.0 * *e1;
    }
}

/* Weight of the parabolic coefficients against the linear ones:
 * f = clamp(2 - 2u, 0, 1) * clamp(2 - q/2, 0, 1), q = u/w, i.e. the full
 * parabola for u <= 1/2 and u/w <= 2, the linear form for u >= 1 or
 * u/w >= 4, linear ramps in between. (Reading: with voxel-constant S the
 * plain parabola gives the downstream voxel a negative weight in optically
 * thick intervals and overshoots next to short intervals; then the OS
 * matrix 1 - Lambda*(1-eps) loses diagonal dominance at small eps and the
 * Jacobi/Gauss-Seidel solvers of Sec. 4 diverge.) */
double orc_parab_weight(double u, double w)
{
    if (!(w > 0.0)) return 0.0;
    double fu = 2.0 - 2.0 * u;
    if (fu > 1.0) fu = 1.0;
    if (fu < 0.0) fu = 0.0;
    double fq = 2.0 - 0.5 * (u / w);
    if (fq > 1.0) fq = 1.0;
    if (fq < 0.0) fq = 0.0;
    return fu * fq;
}

/* Interpolation coefficients of the interval (k-1 -> k) with optical depth u,
 * the next interval (k -> k+1) having w. E = exp(-u). Linear (parabolic == 0
 * or w <= 0): alpha = e0 - e1/u, beta = e1/u, gamma = 0. Parabolic: the
 * Lagrange parabola through the three points integrated over the interval,
 * blended with the linear coefficients by the weight f above:
 * c = c_lin + f (c_par - c_lin). u <= 0 (vacuum) gives E = 1 and zero
 * coefficients. */
void orc_coef(int parabolic, double u, double w, double *E, double *al, double *be, double *ga)
{
    if (!(u > 0.0)) {
        *E = 1.0;
        *al = *be = *ga = 0.0;
        return;
    }
    double e0, e1, e2;
    orc_e012(u, &e0, &e1, &e2);
    *E = exp(-u);
    double al_l = e0 - e1 / u, be_l = e1 / u;
    double f = parabolic ? orc_parab_weight(u, w) : 0.0;
    if (f == 0.0) {
        *al = al_l;
        *be = be_l;
        *ga = 0.0;
    } else {
        double al_p = e0 + (e2 - (w + 2.0 * u) * e1) / (u * (u + w));
        double be_p = ((u + w) * e1 - e2) / (u * w);
        double ga_p = (e2 - u * e1) / (w * (u + w));
        *al = al_l + f * (al_p - al_l);
        *be = be_l + f * (be_p - be_l);
        *ga = f * ga_p;
    }
}

/* ---------------------------------------------------------------------------
 * Formal solution along one characteristic of K points (Eq. 1 integrated
 * along the ray; the per-slot steps of Listing 1):
 *   I_k = E_k I_{k-1} + alpha_k S_{k-1} + beta_k S_k + gamma_k S_{k+1},
 * with u_k = 1/2 (chil[k-1] + chil[k]) (chil[-1] = 0), w_k = u_{k+1},
 * S_{-1} = S_0 (boundary entry point), linear form on the last interval.
 * chil[k] = chi_k l_k. Optional outputs: per-point E, alpha, beta, gamma.
 * ------------------------------------------------------------------------- */
void orc_ray_fs(int K, const double *chil, const double *S, double I0, int parabolic,
                double *I, double *E, double *al, double *be, double *ga)
{
    double Ic = I0;
    for (int k = 0; k < K; k++) {
        double u = 0.5 * ((k > 0 ? chil[k - 1] : 0.0) + chil[k]);
        int has_next = (k + 1 < K);
        double w = has_next ? 0.5 * (chil[k] + chil[k + 1]) : 0.0;
        double Sm = k > 0 ? S[k - 1] : S[0];
        double Sn = has_next ? S[k + 1] : 0.0;
        double e, a, b, g;
        orc_coef(parabolic && has_next, u, w, &e, &a, &b, &g);
        Ic = e * Ic + a * Sm + b * S[k] + g * Sn;
        I[k] = Ic;
        if (E) E[k] = e;
        if (al) al[k] = a;
        if (be) be[k] = b;
        if (ga) ga[k] = g;
    }
}

/* dI_k / dS_j for one characteristic, from the recurrence: every term
 * coef_m S_x that enters I_m reaches I_k attenuated by prod_{i=m+1..k} E_i.
 * Point 0 carries S twice (alpha_0 multiplies the entry value S_{-1} = S_0). */
static double orc_dIdS(int k, int j, const double *E, const double *al,
                       const double *be, const double *ga)
{
    double sum = 0.0;
    int mlo = j - 1 < 0 ? 0 : j - 1;
    int mhi = j + 1 < k ? j + 1 : k;
    for (int m = mlo; m <= mhi; m++) {
        double c = 0.0;
        if (m - 1 == j) c += al[m];
        if (m == 0 && j == 0) c += al[0];
        if (m == j) c += be[m];
        if (m + 1 == j) c += ga[m];
        if (c == 0.0) continue;
        double A = 1.0;
        for (int i = m + 1; i <= k; i++) A *= E[i];
        sum += c * A;
    }
    return sum;
}

/* 27-neighbourhood offset of voxel a seen from voxel b, periodic in x and y:
 * returns d = (dx+1) + 3 (dy+1) + 9 (dz+1) in 0..26, or -1 if a is not a
 * neighbour of b. Needs nx, ny >= 3. */
static int orc_nb_code(int nx, int ny, int a, int b)
{
    int xa = a % nx, ya = (a / nx) % ny, za = a / (nx * ny);
    int xb = b % nx, yb = (b / nx) % ny, zb = b / (nx * ny);
    int dx = ((xa - xb) % nx + nx) % nx;
    int dy = ((ya - yb) % ny + ny) % ny;
    int dz = za - zb;
    if (dx == nx - 1) dx = -1;
    else if (dx > 1) return -1;
    if (dy == ny - 1) dy = -1;
    else if (dy > 1) return -1;
    if (dz < -1 || dz > 1) return -1;
    return (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
}

/* Boundary intensity of ray (x0,y0) with direction cosine mu: top face for
 * mu < 0, bottom face for mu > 0; a face array (indexed x + nx y) overrides
 * the scalar. A bottom gradient array (nullable) gives the inner boundary the
 * LTE diffusion form of the test cases (Sec. 3.1, 3.2): I = I_bot + mu dB/dtau,
 * the first-order diffusion-limit intensity, with tau the vertical optical
 * depth increasing inward. */
static double orc_bc(int nx, double mu, int x0, int y0, double I_top, const double *I_top_face,
                     double I_bot, const double *I_bot_face, const double *I_bot_grad)
{
    const int f = x0 + nx * y0;
    if (mu < 0.0) return I_top_face ? I_top_face[f] : I_top;
    double I = I_bot_face ? I_bot_face[f] : I_bot;
    if (I_bot_grad) I += mu * I_bot_grad[f];
    return I;
}

/* ---------------------------------------------------------------------------
 * Face arrays of the LTE diffusion inner boundary (Sec. 3.1, 3.2 test cases)
 * for the bottom face z = 0, per column (x, y):
 *   grad   = dB/dtau = (B(x,y,0) - B(x,y,1)) / dtau,
 *   dtau   = 1/2 (chi(x,y,0) + chi(x,y,1)),
 * the one-sided difference over the innermost centre spacing (unit length,
 * trapezoidal optical depth; tau increases inward), and
 *   I_face = B(x,y,0) + 1/2 chi(x,y,0) grad,
 * B carried linearly from the innermost centre to the face half a voxel
 * below it, where the characteristics enter. A single layer (nz = 1) has no
 * gradient: grad = 0, I_face = B(x,y,0). Faces are indexed x + nx y.
 * ------------------------------------------------------------------------- */
void orc_diffusion_bc(int nx, int ny, int nz, const double *chi, const double *B,
                      double *I_face, double *grad)
{
    const long nf = (long)nx * ny;
    for (long f = 0; f < nf; f++) {
        if (nz < 2) {
            grad[f] = 0.0;
            I_face[f] = B[f];
            continue;
        }
        double dtau = 0.5 * (chi[f] + chi[nf + f]);
        grad[f] = (B[f] - B[nf + f]) / dtau;
        I_face[f] = B[f] + (0.5 * chi[f]) * grad[f];
    }
}

/* ---------------------------------------------------------------------------
 * Formal solution J = Lambda S (Eq. frmsol) on the periodic Cartesian
 * box for all solid angles, and optionally the 27-point Lambda* band:
 *   J_v = sum_Omega w (sum_{k in v} l_k I_k) / (sum_{k in v} l_k)
 *   L*[v][d] = sum_Omega w sum_{k in v} l_k/(sum l) sum_{j in window(k),
 *              v_j = v + d} dI_k/dS_j
 * Every characteristic is traced on its own. Arrays are x fastest:
 * v = x + nx (y + ny z); lstar (nullable) is [N][27] with
 * d = (dx+1) + 3(dy+1) + 9(dz+1). Returns 0, or < 0 on a tracing error.
 * OpenMP over solid angles with per-thread partial sums.
 * ------------------------------------------------------------------------- */
static int orc_fs_cart_core(int nx, int ny, int nz, int nth, int nph, int parabolic,
                            const double *chi, const double *S,
                            double I_top, const double *I_top_face, double I_bot,
                            const double *I_bot_face, const double *I_bot_grad, double *J,
                            double *lstar, int nthreads,
                            const int *angles, int nang)
{
    const long N = (long)nx * ny * nz;
    const int nO = nth * nph;
    double *mu = malloc(sizeof(double) * nO), *phi = malloc(sizeof(double) * nO);
    double *dir = malloc(sizeof(double) * 3 * nO), *wt = malloc(sizeof(double) * nO);
    orc_directions(nth, nph, mu, phi, dir, wt);
    if (nthreads < 1) nthreads = 1;
    int err = 0;
    double **Jp = calloc(nthreads, sizeof(double *));
    double **Lp = calloc(nthreads, sizeof(double *));
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *Jt = calloc(N, sizeof(double));
        double *Lt = lstar ? calloc(27 * N, sizeof(double)) : NULL;
        double *num = malloc(sizeof(double) * N), *den = malloc(sizeof(double) * N);
        double *numL = lstar ? malloc(sizeof(double) * 27 * N) : NULL;
        Jp[tid] = Jt;
        Lp[tid] = Lt;
        const int nloop = angles ? nang : nO;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int io = 0; io < nloop; io++) {
            const int o = angles ? angles[io] : io;
            const double *d = dir + 3 * o;
            int kmax = orc_kmax_cart(nx, ny, nz, d);
            int *vox = malloc(sizeof(int) * kmax);
            double *len = malloc(sizeof(double) * kmax), *chil = malloc(sizeof(double) * kmax);
            double *Sp = malloc(sizeof(double) * kmax), *I = malloc(sizeof(double) * kmax);
            double *E = malloc(sizeof(double) * kmax), *al = malloc(sizeof(double) * kmax);
            double *be = malloc(sizeof(double) * kmax), *ga = malloc(sizeof(double) * kmax);
            memset(num, 0, sizeof(double) * N);
            memset(den, 0, sizeof(double) * N);
            if (numL) memset(numL, 0, sizeof(double) * 27 * N);
            for (int y0 = 0; y0 < ny; y0++) {
                for (int x0 = 0; x0 < nx; x0++) {
                    int K = orc_trace_cart(nx, ny, nz, d, x0, y0, kmax, vox, len);
                    if (K < 0) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                        err = K;
                        continue;
                    }
                    for (int k = 0; k < K; k++) {
                        chil[k] = chi[vox[k]] * len[k];
                        Sp[k] = S[vox[k]];
                    }
                    double I0 = orc_bc(nx, d[2], x0, y0, I_top, I_top_face, I_bot, I_bot_face,
                                       I_bot_grad);
                    orc_ray_fs(K, chil, Sp, I0, parabolic, I, E, al, be, ga);
                    for (int k = 0; k < K; k++) {
                        num[vox[k]] += len[k] * I[k];
                        den[vox[k]] += len[k];
                        if (!numL) continue;
                        int vk = vox[k];
                        int jend = k + 1 < K ? k + 1 : k;
                        int j0 = jend;
                        while (j0 - 1 >= 0 && orc_nb_code(nx, ny, vox[j0 - 1], vk) >= 0) j0--;
                        /* the run must be contiguous through k: points k..jend are
                           always neighbours (consecutive DDA cells touch) */
                        for (int j = j0; j <= jend; j++) {
                            int dc = orc_nb_code(nx, ny, vox[j], vk);
                            if (dc < 0) continue;
                            numL[27 * (long)vk + dc] += len[k] * orc_dIdS(k, j, E, al, be, ga);
                        }
                    }
                }
            }
            for (long v = 0; v < N; v++) {
                if (den[v] > 0.0) Jt[v] += wt[o] * (num[v] / den[v]);
            }
            if (numL) {
                for (long v = 0; v < N; v++) {
                    if (!(den[v] > 0.0)) continue;
                    for (int c = 0; c < 27; c++) Lt[27 * v + c] += wt[o] * (numL[27 * v + c] / den[v]);
                }
            }
            free(vox); free(len); free(chil); free(Sp); free(I);
            free(E); free(al); free(be); free(ga);
        }
        free(num); free(den); free(numL);
    }
    for (long v = 0; v < N; v++) {
        double s = 0.0;
        for (int t = 0; t < nthreads; t++) s += Jp[t] ? Jp[t][v] : 0.0;
        J[v] = s;
    }
    if (lstar) {
        for (long i = 0; i < 27 * N; i++) {
            double s = 0.0;
            for (int t = 0; t < nthreads; t++) s += Lp[t] ? Lp[t][i] : 0.0;
            lstar[i] = s;
        }
    }
    for (int t = 0; t < nthreads; t++) { free(Jp[t]); free(Lp[t]); }
    free(Jp); free(Lp); free(mu); free(phi); free(dir); free(wt);
    return err;
}

int orc_fs_cart(int nx, int ny, int nz, int nth, int nph, int parabolic,
                const double *chi, const double *S,
                double I_top, const double *I_top_face, double I_bot, const double *I_bot_face,
                const double *I_bot_grad,
                double *J, double *lstar, int nthreads)
{
    return orc_fs_cart_core(nx, ny, nz, nth, nph, parabolic, chi, S, I_top, I_top_face, I_bot,
                            I_bot_face, I_bot_grad, J, lstar, nthreads, NULL, 0);
}

/* The same sums restricted to the listed solid angles (a bounded sample of a
 * large formal solution; J receives only their share). */
int orc_fs_cart_angles(int nx, int ny, int nz, int nth, int nph, int parabolic,
                       const double *chi, const double *S,
                       double I_top, const double *I_top_face, double I_bot,
                       const double *I_bot_face, const double *I_bot_grad, double *J, int nthreads,
                       const int *angles, int nang)
{
    return orc_fs_cart_core(nx, ny, nz, nth, nph, parabolic, chi, S, I_top, I_top_face, I_bot,
                            I_bot_face, I_bot_grad, J, NULL, nthreads, angles, nang);
}

/* ---------------------------------------------------------------------------
 * The same J_v and Lambda* row for ONE voxel v (for spot checks of large
 * grids). For every solid angle the characteristics through v are those
 * whose reference-ray step e lies in the layer of v, started from
 * (x_v - dx_e, y_v - dy_e); each is traced and integrated on its own, and all
 * of its points inside v are collected. Returns 0, or < 0 if the collected
 * chord sum of some angle is not 1/|mu| (a missing characteristic).
 * Optionally restricted to the solid angles [o_lo, o_hi).
 * ------------------------------------------------------------------------- */
int orc_fs_cart_voxel(int nx, int ny, int nz, int nth, int nph, int parabolic,
                      const double *chi, const double *S,
                      double I_top, const double *I_top_face, double I_bot, const double *I_bot_face,
                      const double *I_bot_grad,
                      long v, int o_lo, int o_hi, double *J_v, double *lstar_row)
{
    const int nO = nth * nph;
    double *mu = malloc(sizeof(double) * nO), *phi = malloc(sizeof(double) * nO);
    double *dir = malloc(sizeof(double) * 3 * nO), *wt = malloc(sizeof(double) * nO);
    orc_directions(nth, nph, mu, phi, dir, wt);
    int xv = (int)(v % nx), yv = (int)((v / nx) % ny), zv = (int)(v / ((long)nx * ny));
    double Jsum = 0.0;
    double Lrow[27];
    for (int c = 0; c < 27; c++) Lrow[c] = 0.0;
    int err = 0;
    if (o_lo < 0) o_lo = 0;
    if (o_hi > nO || o_hi <= 0) o_hi = nO;
    for (int o = o_lo; o < o_hi && !err; o++) {
        const double *d = dir + 3 * o;
        int kmax = orc_kmax_cart(nx, ny, nz, d);
        int *vox0 = malloc(sizeof(int) * kmax), *vox = malloc(sizeof(int) * kmax);
        double *len0 = malloc(sizeof(double) * kmax), *len = malloc(sizeof(double) * kmax);
        double *chil = malloc(sizeof(double) * kmax), *Sp = malloc(sizeof(double) * kmax);
        double *I = malloc(sizeof(double) * kmax), *E = malloc(sizeof(double) * kmax);
        double *al = malloc(sizeof(double) * kmax), *be = malloc(sizeof(double) * kmax);
        double *ga = malloc(sizeof(double) * kmax);
        int *seen = calloc((size_t)nx * ny, sizeof(int));
        int K0 = orc_trace_cart(nx, ny, nz, d, 0, 0, kmax, vox0, len0);
        double num = 0.0, den = 0.0, numL[27];
        for (int c = 0; c < 27; c++) numL[c] = 0.0;
        if (K0 < 0) err = K0;
        for (int e = 0; e < K0 && !err; e++) {
            if (vox0[e] / (nx * ny) != zv) continue;
            int dx = vox0[e] % nx, dy = (vox0[e] / nx) % ny;
            int x0 = ((xv - dx) % nx + nx) % nx, y0 = ((yv - dy) % ny + ny) % ny;
            if (seen[x0 + nx * y0]) continue;
            seen[x0 + nx * y0] = 1;
            int K = orc_trace_cart(nx, ny, nz, d, x0, y0, kmax, vox, len);
            if (K < 0) { err = K; break; }
            for (int k = 0; k < K; k++) {
                chil[k] = chi[vox[k]] * len[k];
                Sp[k] = S[vox[k]];
            }
            double I0 = orc_bc(nx, d[2], x0, y0, I_top, I_top_face, I_bot, I_bot_face, I_bot_grad);
            orc_ray_fs(K, chil, Sp, I0, parabolic, I, E, al, be, ga);
            for (int k = 0; k < K; k++) {
                if (vox[k] != v) continue;
                num += len[k] * I[k];
                den += len[k];
                if (!lstar_row) continue;
                int jend = k + 1 < K ? k + 1 : k;
                int j0 = jend;
                while (j0 - 1 >= 0 && orc_nb_code(nx, ny, vox[j0 - 1], (int)v) >= 0) j0--;
                for (int j = j0; j <= jend; j++) {
                    int dc = orc_nb_code(nx, ny, vox[j], (int)v);
                    if (dc < 0) continue;
                    numL[dc] += len[k] * orc_dIdS(k, j, E, al, be, ga);
                }
            }
        }
        if (!err) {
            double expect = 1.0 / fabs(d[2]);
            if (!(fabs(den - expect) <= 1e-9 * expect)) err = -3;
            Jsum += wt[o] * (num / den);
            for (int c = 0; c < 27; c++) Lrow[c] += wt[o] * (numL[c] / den);
        }
        free(vox0); free(vox); free(len0); free(len); free(chil); free(Sp);
        free(I); free(E); free(al); free(be); free(ga); free(seen);
    }
    *J_v = Jsum;
    if (lstar_row) for (int c = 0; c < 27; c++) lstar_row[c] = Lrow[c];
    free(mu); free(phi); free(dir); free(wt);
    return err;
}

/* Neighbour v + d of v (periodic in x, y), or -1 outside the box in z. */
static long orc_nb(int nx, int ny, int nz, long v, int c)
{
    int dx = c % 3 - 1, dy = (c / 3) % 3 - 1, dz = c / 9 - 1;
    int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long)nx * ny));
    x = (x + dx + nx) % nx;
    y = (y + dy + ny) % ny;
    z = z + dz;
    if (z < 0 || z >= nz) return -1;
    return x + (long)nx * (y + (long)ny * z);
}

/* ---------------------------------------------------------------------------
 * Operator-splitting linear system of Eq. alo written for the correction
 * Delta J = J_new - J_old:  [1 - Lambda*(1 - eps)] Delta J = r, r = J_FS - J_old,
 * solved by Jacobi iteration (Sec. 4, "OS iteration"):
 *   dJ^0 = r / diag,  dJ^{m+1}_v = (r_v + sum_{d != 13} L*[v][d] (1 - eps_{v+d})
 *                                  dJ^m_{v+d}) / diag_v,
 *   diag_v = 1 - L*[v][13] (1 - eps_v).
 * Stops when max|dJ^{m+1} - dJ^m| <= tol max|dJ^{m+1}| or after max_sweeps.
 * lstar is [N][27]. Returns the number of sweeps done.
 * ------------------------------------------------------------------------- */
int orc_os_jacobi(int nx, int ny, int nz, const double *lstar, const double *eps,
                  const double *r, double *dJ, int max_sweeps, double tol)
{
    const long N = (long)nx * ny * nz;
    double *nw = malloc(sizeof(double) * N);
    for (long v = 0; v < N; v++) dJ[v] = r[v] / (1.0 - lstar[27 * v + 13] * (1.0 - eps[v]));
    int m = 0;
    while (m < max_sweeps) {
        double dmax = 0.0, jmax = 0.0;
        for (long v = 0; v < N; v++) {
            double s = r[v];
            for (int c = 0; c < 27; c++) {
                if (c == 13) continue;
                long u = orc_nb(nx, ny, nz, v, c);
                if (u < 0) continue;
                s += lstar[27 * v + c] * (1.0 - eps[u]) * dJ[u];
            }
            nw[v] = s / (1.0 - lstar[27 * v + 13] * (1.0 - eps[v]));
        }
        for (long v = 0; v < N; v++) {
            double df = fabs(nw[v] - dJ[v]);
            if (df > dmax) dmax = df;
            if (fabs(nw[v]) > jmax) jmax = fabs(nw[v]);
            dJ[v] = nw[v];
        }
        m++;
        if (dmax <= tol * jmax) break;
    }
    free(nw);
    return m;
}

/* ---------------------------------------------------------------------------
 * Other solvers of the same OS system (the paper names Gauss-Seidel and
 * BiCGStab OS solvers besides Jacobi, Sec. 4), with the matrix
 *   A[v][v] = 1 - L*[v][13] (1 - eps_v),  A[v][u] = -L*[v][d] (1 - eps_u).
 *
 * Gauss-Seidel, colored = 0: voxels in index order, each update using the
 * newest values. colored = 1: eight colors by the parities of (x, y, z),
 * swept in order c = px + 2 py + 4 pz; within a color every update reads the
 * values from before that color's sweep (on a 27-point stencil two voxels of
 * one color are neighbours only across a periodic wrap of odd length).
 * Starts from dJ^0 = r / diag; the stop test of orc_os_jacobi. Returns the
 * sweeps done.
 * ------------------------------------------------------------------------- */
static double orc_os_row(int nx, int ny, int nz, const double *lstar, const double *eps,
                         const double *r, const double *x, long v)
{
    double s = r[v];
    for (int c = 0; c < 27; c++) {
        if (c == 13) continue;
        long u = orc_nb(nx, ny, nz, v, c);
        if (u < 0) continue;
        s += lstar[27 * v + c] * (1.0 - eps[u]) * x[u];
    }
    return s / (1.0 - lstar[27 * v + 13] * (1.0 - eps[v]));
}

int orc_os_gauss_seidel(int nx, int ny, int nz, const double *lstar, const double *eps,
                        const double *r, double *dJ, int max_sweeps, double tol, int colored)
{
    const long N = (long)nx * ny * nz;
    double *old = malloc(sizeof(double) * N);
    double *snap = malloc(sizeof(double) * N);
    for (long v = 0; v < N; v++) dJ[v] = r[v] / (1.0 - lstar[27 * v + 13] * (1.0 - eps[v]));
    int m = 0;
    while (m < max_sweeps) {
        memcpy(old, dJ, sizeof(double) * N);
        if (!colored) {
            for (long v = 0; v < N; v++) dJ[v] = orc_os_row(nx, ny, nz, lstar, eps, r, dJ, v);
        } else {
            for (int col = 0; col < 8; col++) {
                memcpy(snap, dJ, sizeof(double) * N);
                for (long v = 0; v < N; v++) {
                    int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long)nx * ny));
                    if ((x & 1) + 2 * (y & 1) + 4 * (z & 1) != col) continue;
                    dJ[v] = orc_os_row(nx, ny, nz, lstar, eps, r, snap, v);
                }
            }
        }
        double dmax = 0.0, jmax = 0.0;
        for (long v = 0; v < N; v++) {
            double df = fabs(dJ[v] - old[v]);
            if (df > dmax) dmax = df;
            if (fabs(dJ[v]) > jmax) jmax = fabs(dJ[v]);
        }
        m++;
        if (dmax <= tol * jmax) break;
    }
    free(old);
    free(snap);
    return m;
}

/* A x for the OS matrix above. */
static void orc_os_apply(int nx, int ny, int nz, const double *lstar, const double *eps,
                         const double *x, double *y)
{
    const long N = (long)nx * ny * nz;
    for (long v = 0; v < N; v++) {
        double s = (1.0 - lstar[27 * v + 13] * (1.0 - eps[v])) * x[v];
        for (int c = 0; c < 27; c++) {
            if (c == 13) continue;
            long u = orc_nb(nx, ny, nz, v, c);
            if (u < 0) continue;
            s -= lstar[27 * v + c] * (1.0 - eps[u]) * x[u];
        }
        y[v] = s;
    }
}

static double orc_dot(long n, const double *a, const double *b)
{
    double s = 0.0;
    for (long i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* BiCGStab (van der Vorst 1992) on A dJ = r from dJ = 0, without a
 * preconditioner; stops when ||r_k||_2 <= tol ||r||_2 or after max_iter
 * iterations (two products with A each). Returns the iterations done, or
 * -(iterations) on a breakdown (rho or omega zero). */
int orc_os_bicgstab(int nx, int ny, int nz, const double *lstar, const double *eps,
                    const double *r, double *dJ, int max_iter, double tol)
{
    const long N = (long)nx * ny * nz;
    double *res = malloc(sizeof(double) * N), *rh = malloc(sizeof(double) * N);
    double *p = calloc(N, sizeof(double)), *vv = calloc(N, sizeof(double));
    double *sv = malloc(sizeof(double) * N), *t = malloc(sizeof(double) * N);
    for (long i = 0; i < N; i++) {
        dJ[i] = 0.0;
        res[i] = r[i];
        rh[i] = r[i];
    }
    const double nr0 = sqrt(orc_dot(N, r, r));
    double rho = 1.0, alpha = 1.0, omega = 1.0;
    int k = 0, status = 0;
    if (!(nr0 > 0.0)) goto done;
    while (k < max_iter) {
        const double rho1 = orc_dot(N, rh, res);
        if (rho1 == 0.0) { status = -1; break; }
        const double beta = (rho1 / rho) * (alpha / omega);
        for (long i = 0; i < N; i++) p[i] = res[i] + beta * (p[i] - omega * vv[i]);
        orc_os_apply(nx, ny, nz, lstar, eps, p, vv);
        alpha = rho1 / orc_dot(N, rh, vv);
        for (long i = 0; i < N; i++) sv[i] = res[i] - alpha * vv[i];
        orc_os_apply(nx, ny, nz, lstar, eps, sv, t);
        const double tt = orc_dot(N, t, t);
        omega = tt > 0.0 ? orc_dot(N, t, sv) / tt : 0.0;
        for (long i = 0; i < N; i++) {
            dJ[i] += alpha * p[i] + omega * sv[i];
            res[i] = sv[i] - omega * t[i];
        }
        rho = rho1;
        k++;
        if (sqrt(orc_dot(N, res, res)) <= tol * nr0) break;
        if (omega == 0.0) { status = -1; break; }
    }
done:
    free(res); free(rh); free(p); free(vv); free(sv); free(t);
    return status < 0 ? -k : k;
}

/* ---------------------------------------------------------------------------
 * ALI iteration (Eqs. alisol, alodef, alo): from J,
 *   S = (1 - eps) J + eps B;  J_FS = Lambda S (Lambda* built in the first
 *   iteration);  r = J_FS - J;  Jacobi solve of [1 - L*(1-eps)] dJ = r;
 *   J += dJ;  rel = max_v |dJ_v| / |J_v|;
 * until rel < tol or max_iter iterations. J is updated in place. history
 * (nullable, max_iter) receives rel per iteration; lstar_out (nullable) the
 * Lambda* band. Returns the number of iterations (negative if not converged,
 * or on a tracing error -1000 + code).
 * ------------------------------------------------------------------------- */
int orc_ali_solve(int nx, int ny, int nz, int nth, int nph, int parabolic,
                  const double *chi, const double *eps, const double *B,
                  double I_top, const double *I_top_face, double I_bot, const double *I_bot_face,
                  const double *I_bot_grad,
                  double *J, double tol, int max_iter, int max_sweeps, double sweep_tol,
                  int nthreads, double *lstar_out, double *history)
{
    const long N = (long)nx * ny * nz;
    double *S = malloc(sizeof(double) * N), *Jfs = malloc(sizeof(double) * N);
    double *r = malloc(sizeof(double) * N), *dJ = malloc(sizeof(double) * N);
    double *L = lstar_out ? lstar_out : malloc(sizeof(double) * 27 * N);
    int it = 0, conv = 0, err = 0;
    for (it = 0; it < max_iter; it++) {
        for (long v = 0; v < N; v++) S[v] = (1.0 - eps[v]) * J[v] + eps[v] * B[v];
        err = orc_fs_cart(nx, ny, nz, nth, nph, parabolic, chi, S, I_top, I_top_face, I_bot,
                          I_bot_face, I_bot_grad, Jfs, it == 0 ? L : NULL, nthreads);
        if (err) break;
        for (long v = 0; v < N; v++) r[v] = Jfs[v] - J[v];
        orc_os_jacobi(nx, ny, nz, L, eps, r, dJ, max_sweeps, sweep_tol);
        double rel = 0.0;
        int bad = 0;
        for (long v = 0; v < N; v++) {
            J[v] += dJ[v];
            if (!isfinite(J[v])) bad = 1;
            if (dJ[v] == 0.0) continue;
            double q = fabs(dJ[v]) / fabs(J[v]);
            if (q > rel) rel = q;
        }
        if (history) history[it] = bad ? NAN : rel;
        if (bad) { err = -100; break; }
        if (rel < tol) { it++; conv = 1; break; }
    }
    free(S); free(Jfs); free(r); free(dJ);
    if (!lstar_out) free(L);
    if (err) return -1000000 + err;
    return conv ? it : -it;
}
