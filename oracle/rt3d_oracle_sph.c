/*
 * rt3d_oracle_sph.c -- plain FP64 CPU oracle of the long-characteristics
 * formal solution on the spherical (r, theta, phi) grid of the paper's SP test
 * case (Sec. 3.2: irradiated spherical atmospheres; Sec. 4: tracker and
 * formal solution). TEST INFRASTRUCTURE, shares no code with the CUDA path;
 * built with -ffp-contract=off so that every crossing parameter is plain
 * IEEE arithmetic.
 *
 * Readings (the paper gives no spherical discretisation):
 *  - cells: radial edges r_e[i] = r_in (r_out/r_in)^(i/nr), i = 0..nr; polar
 *    edges theta_e[j] = j pi / nt; azimuth edges phi_e[k] = 2 pi k / np
 *    (periodic). Voxel index v = ir + nr (it + nt ip).
 *  - the ray set of a solid angle: voxels visited in index order; a voxel not
 *    yet crossed by a ray of this angle launches the full line through its
 *    centre (sqrt(r_e[i] r_e[i+1]), mid theta, mid phi), traced back to its
 *    entry (outer sphere, or the core sphere r = r_in) and forward to its
 *    exit; every cell it crosses is marked.
 *  - crossings: spheres t = -b +- sqrt(b^2 - c); cones z^2 = cos^2(theta_e)
 *    |p|^2 with the sign of z equal to that of cos(theta_e) (the plane z = 0
 *    for theta_e = pi/2); half-planes of phi_e (linear, accepted where
 *    p . (cos phi_e, sin phi_e) > 0). Tangent roots (discriminant <= 0) do not
 *    cross. Equal parameters are merged.
 *  - the cell of an interval is found at its midpoint by comparisons only:
 *    r^2 against r_e^2, z|z| against cos(theta_e)|cos(theta_e)| r^2, and the
 *    sign of the cross product with the edge directions of phi.
 *  - points at chord midpoints, dtau, interpolation, J and the Lambda*
 *    window as on the Cartesian grid; entry through the core: I = B of the
 *    first cell, or the LTE diffusion condition I = I_face + mu dB/dtau
 *    (orc_diffusion_bc_sph); through the outer sphere: I = 0, or I_irr where
 *    the entry point has x > 0 and the direction d_x < 0 (irradiation from
 *    +x).
 *  - trig tables (cos/sin of the edges and centres) from libm on the host.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

void orc_directions(int nth, int nph, double *mu, double *phi, double *dir, double *w);
void orc_ray_fs(int K, const double *chil, const double *S, double I0, int parabolic,
                double *I, double *E, double *al, double *be, double *ga);

typedef struct {
    int nr, nt, np;
    double *re2;          /* r_e^2, nr+1 */
    double *re;           /* r_e, nr+1 */
    double *ct, *ctk;     /* cos(theta_e), cos|cos|, nt+1 */
    double *cpe, *spe;    /* cos/sin phi_e, np */
    double *rc, *stc, *ctc, *cpc, *spc; /* centres */
} orc_sph;

static void sph_init(orc_sph *g, int nr, int nt, int np, double r_in, double r_out)
{
    g->nr = nr; g->nt = nt; g->np = np;
    g->re = malloc(sizeof(double) * (nr + 1));
    g->re2 = malloc(sizeof(double) * (nr + 1));
    for (int i = 0; i <= nr; i++) {
        g->re[i] = r_in * pow(r_out / r_in, (double)i / (double)nr);
        g->re2[i] = g->re[i] * g->re[i];
    }
    g->re[0] = r_in; g->re2[0] = r_in * r_in;
    g->re[nr] = r_out; g->re2[nr] = r_out * r_out;
    g->ct = malloc(sizeof(double) * (nt + 1));
    g->ctk = malloc(sizeof(double) * (nt + 1));
    for (int j = 0; j <= nt; j++) {
        double c = cos((double)j * M_PI / (double)nt);
        if (2 * j == nt) c = 0.0;
        if (j == 0) c = 1.0;
        if (j == nt) c = -1.0;
        g->ct[j] = c;
        g->ctk[j] = c * fabs(c);
    }
    g->cpe = malloc(sizeof(double) * np);
    g->spe = malloc(sizeof(double) * np);
    for (int k = 0; k < np; k++) {
        double p = 2.0 * M_PI * (double)k / (double)np;
        g->cpe[k] = cos(p);
        g->spe[k] = sin(p);
    }
    g->rc = malloc(sizeof(double) * nr);
    for (int i = 0; i < nr; i++) g->rc[i] = sqrt(g->re[i] * g->re[i + 1]);
    g->stc = malloc(sizeof(double) * nt);
    g->ctc = malloc(sizeof(double) * nt);
    for (int j = 0; j < nt; j++) {
        double t = ((double)j + 0.5) * M_PI / (double)nt;
        g->stc[j] = sin(t);
        g->ctc[j] = cos(t);
    }
    g->cpc = malloc(sizeof(double) * np);
    g->spc = malloc(sizeof(double) * np);
    for (int k = 0; k < np; k++) {
        double p = 2.0 * M_PI * ((double)k + 0.5) / (double)np;
        g->cpc[k] = cos(p);
        g->spc[k] = sin(p);
    }
}

static void sph_free(orc_sph *g)
{
    free(g->re); free(g->re2); free(g->ct); free(g->ctk); free(g->cpe); free(g->spe);
    free(g->rc); free(g->stc); free(g->ctc); free(g->cpc); free(g->spc);
}

/* cell of point p (comparisons only) */
static int sph_cell(const orc_sph *g, const double *p)
{
    double r2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
    int ir = 0;
    while (ir + 1 < g->nr && g->re2[ir + 1] <= r2) ir++;
    double key = p[2] * fabs(p[2]);
    int it = 0;
    while (it + 1 < g->nt && g->ctk[it + 1] * r2 >= key) it++;
    int ip = 0;
    for (int k = 0; k < g->np; k++) {
        int k1 = (k + 1) % g->np;
        double c0 = g->cpe[k] * p[1] - g->spe[k] * p[0];
        double c1 = g->cpe[k1] * p[1] - g->spe[k1] * p[0];
        if (c0 >= 0.0 && c1 < 0.0) { ip = k; break; }
    }
    return ir + g->nr * (it + g->nt * ip);
}

static int cmp_d(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Traces the line P + t d between its entry and exit. Writes voxel indices
 * and chords; entry_core = 1 if the line enters through the core sphere;
 * pin receives the entry point. Returns K or -1 if cap is exceeded. */
int orc_sph_trace(const orc_sph *g, const double *P, const double *d, int cap, int *vox,
                  double *len, int *entry_core, double *pin)
{
    const double b = P[0] * d[0] + P[1] * d[1] + P[2] * d[2];
    const double P2 = P[0] * P[0] + P[1] * P[1] + P[2] * P[2];
    /* outer sphere */
    double disc = b * b - (P2 - g->re2[g->nr]);
    double sq = sqrt(disc);
    double t0 = -b - sq, t1 = -b + sq;
    *entry_core = 0;
    /* core sphere */
    double dc = b * b - (P2 - g->re2[0]);
    if (dc > 0.0) {
        double sc = sqrt(dc);
        double a = -b - sc, c = -b + sc;
        if (c <= 0.0 && c > t0) { t0 = c; *entry_core = 1; }
        if (a >= 0.0 && a < t1) t1 = a;
    }
    int ncap = 2 * (g->nr + 1) + 2 * (g->nt + 1) + g->np + 8;
    double *ts = malloc(sizeof(double) * ncap);
    int n = 0;
    for (int i = 1; i < g->nr; i++) {
        double di = b * b - (P2 - g->re2[i]);
        if (!(di > 0.0)) continue;
        double s = sqrt(di);
        double r1 = -b - s, r2 = -b + s;
        if (r1 > t0 && r1 < t1) ts[n++] = r1;
        if (r2 > t0 && r2 < t1) ts[n++] = r2;
    }
    for (int j = 1; j < g->nt; j++) {
        if (2 * j == g->nt) {
            if (d[2] != 0.0) {
                double t = -P[2] / d[2];
                if (t > t0 && t < t1) ts[n++] = t;
            }
            continue;
        }
        double c2 = g->ct[j] * g->ct[j];
        double A = d[2] * d[2] - c2;
        double Bh = P[2] * d[2] - c2 * b;
        double C = P[2] * P[2] - c2 * P2;
        double roots[2];
        int nr_ = 0;
        if (A == 0.0) {
            if (Bh != 0.0) roots[nr_++] = -C / (2.0 * Bh);
        } else {
            double dq = Bh * Bh - A * C;
            if (dq > 0.0) {
                double s = sqrt(dq);
                roots[nr_++] = (-Bh - s) / A;
                roots[nr_++] = (-Bh + s) / A;
            }
        }
        for (int q = 0; q < nr_; q++) {
            double t = roots[q];
            if (!(t > t0 && t < t1)) continue;
            double z = P[2] + t * d[2];
            if (z * g->ct[j] > 0.0) ts[n++] = t;
        }
    }
    for (int k = 0; k < g->np; k++) {
        double den = g->cpe[k] * d[1] - g->spe[k] * d[0];
        if (den == 0.0) continue;
        double t = (g->spe[k] * P[0] - g->cpe[k] * P[1]) / den;
        if (!(t > t0 && t < t1)) continue;
        double x = P[0] + t * d[0], y = P[1] + t * d[1];
        if (g->cpe[k] * x + g->spe[k] * y > 0.0) ts[n++] = t;
    }
    qsort(ts, n, sizeof(double), cmp_d);
    /* merge equal parameters, add the ends */
    double *all = malloc(sizeof(double) * (n + 2));
    int m = 0;
    all[m++] = t0;
    for (int i = 0; i < n; i++)
        if (ts[i] != all[m - 1]) all[m++] = ts[i];
    if (t1 != all[m - 1]) all[m++] = t1;
    int K = 0;
    for (int i = 0; i + 1 < m; i++) {
        if (K >= cap) { free(ts); free(all); return -1; }
        double mid = 0.5 * (all[i] + all[i + 1]);
        double p[3] = {P[0] + mid * d[0], P[1] + mid * d[1], P[2] + mid * d[2]};
        vox[K] = sph_cell(g, p);
        len[K] = all[i + 1] - all[i];
        K++;
    }
    pin[0] = P[0] + t0 * d[0];
    pin[1] = P[1] + t0 * d[1];
    pin[2] = P[2] + t0 * d[2];
    free(ts); free(all);
    return K;
}

int orc_sph_kcap(int nr, int nt, int np) { return 2 * (nr + 1) + 2 * (nt + 1) + np + 8; }

/* Ray set of solid angle o: the launching voxel of every ray, in order.
 * Returns the number of rays (launch[] must hold N entries). */
int orc_sph_rays(int nr, int nt, int np, double r_in, double r_out, int nth, int nph, int o,
                 int *launch)
{
    orc_sph g;
    sph_init(&g, nr, nt, np, r_in, r_out);
    int nO = nth * nph;
    double *mu = malloc(sizeof(double) * nO), *phi = malloc(sizeof(double) * nO);
    double *dir = malloc(sizeof(double) * 3 * nO), *w = malloc(sizeof(double) * nO);
    orc_directions(nth, nph, mu, phi, dir, w);
    long N = (long)nr * nt * np;
    char *hit = calloc(N, 1);
    int cap = orc_sph_kcap(nr, nt, np);
    int *vox = malloc(sizeof(int) * cap);
    double *len = malloc(sizeof(double) * cap);
    int nrays = 0;
    for (long v = 0; v < N; v++) {
        if (hit[v]) continue;
        int ir = (int)(v % nr), it = (int)((v / nr) % nt), ip = (int)(v / ((long)nr * nt));
        double P[3] = {g.rc[ir] * g.stc[it] * g.cpc[ip], g.rc[ir] * g.stc[it] * g.spc[ip],
                       g.rc[ir] * g.ctc[it]};
        int ec;
        double pin[3];
        int K = orc_sph_trace(&g, P, dir + 3 * o, cap, vox, len, &ec, pin);
        if (K < 0) { nrays = -1; break; }
        for (int k = 0; k < K; k++) hit[vox[k]] = 1;
        hit[v] = 1;
        launch[nrays++] = (int)v;
    }
    free(hit); free(vox); free(len); free(mu); free(phi); free(dir); free(w);
    sph_free(&g);
    return nrays;
}

/* Traces the ray launched by voxel v for direction o (exposed for tests). */
int orc_sph_trace_voxel(int nr, int nt, int np, double r_in, double r_out, const double *d, int v,
                        int cap, int *vox, double *len, int *entry_core, double *pin)
{
    orc_sph g;
    sph_init(&g, nr, nt, np, r_in, r_out);
    int ir = v % nr, it = (v / nr) % nt, ip = v / (nr * nt);
    double P[3] = {g.rc[ir] * g.stc[it] * g.cpc[ip], g.rc[ir] * g.stc[it] * g.spc[ip],
                   g.rc[ir] * g.ctc[it]};
    int K = orc_sph_trace(&g, P, d, cap, vox, len, entry_core, pin);
    sph_free(&g);
    return K;
}

static int sph_nb_code(int nr, int nt, int np, int a, int b)
{
    int ra = a % nr, ta = (a / nr) % nt, pa = a / (nr * nt);
    int rb = b % nr, tb = (b / nr) % nt, pb = b / (nr * nt);
    int dr = ra - rb, dt = ta - tb;
    int dp = ((pa - pb) % np + np) % np;
    if (dp == np - 1) dp = -1;
    else if (dp > 1) return -1;
    if (dr < -1 || dr > 1 || dt < -1 || dt > 1) return -1;
    return (dr + 1) + 3 * (dt + 1) + 9 * (dp + 1);
}

static double sph_dIdS(int k, int j, const double *E, const double *al, const double *be,
                       const double *ga)
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

/* The LTE diffusion inner boundary on the core sphere (Sec. 3.2: the SP test
 * case's inner boundary, as on the Cartesian grid), per core face (it, ip),
 * face index it + nt ip, from the two innermost shells v0 = nr (it + nt ip)
 * and v1 = v0 + 1:
 *   dB/dtau = (B(v0) - B(v1)) / (1/2 (chi(v0) + chi(v1)) (rc1 - rc0)),
 * the one-sided difference over the radial distance of the two cell centres
 * rc_i = sqrt(r_e[i] r_e[i+1]) (tau increases inward), and
 *   I_face = B(v0) + chi(v0) (rc0 - r_in) dB/dtau,
 * B carried linearly from the innermost centre down to the core sphere. One
 * shell (nr = 1): grad = 0, I_face = B(v0). A ray that enters from the core
 * in direction d at the point p of the core sphere starts with
 *   I = I_face + mu dB/dtau,  mu = p . d / r_in,
 * mu the cosine between the ray and the outward normal of the core. */
void orc_diffusion_bc_sph(int nr, int nt, int np, double r_in, double r_out, const double *chi,
                          const double *B, double *I_face, double *grad)
{
    orc_sph g;
    sph_init(&g, nr, nt, np, r_in, r_out);
    for (int ip = 0; ip < np; ip++)
        for (int it = 0; it < nt; it++) {
            const int f = it + nt * ip;
            const long v0 = (long)nr * f;
            if (nr < 2) {
                grad[f] = 0.0;
                I_face[f] = B[v0];
                continue;
            }
            const double dtau = 0.5 * (chi[v0] + chi[v0 + 1]) * (g.rc[1] - g.rc[0]);
            grad[f] = (B[v0] - B[v0 + 1]) / dtau;
            I_face[f] = B[v0] + chi[v0] * (g.rc[0] - r_in) * grad[f];
        }
    sph_free(&g);
}

/* Formal solution on the spherical grid for all solid angles (and the
 * 27-point Lambda* band over the index neighbourhood, periodic in phi):
 * J_v = sum_Omega w (sum_{k in v} l_k I_k) / (sum_{k in v} l_k). A ray that
 * enters from the core starts with core_face[f] + mu core_grad[f] (f the core
 * face of its first cell, mu the cosine at its entry point: the diffusion
 * condition above) when core_face is given, else with B of its first cell
 * (core_grad nullable: no gradient term); I_out is the incoming intensity at
 * the outer sphere (0 in the paper's set-up), I_irr the irradiation. lstar
 * nullable [N][27]. Returns 0 or < 0. */
int orc_fs_sph_bc(int nr, int nt, int np, double r_in, double r_out, int nth, int nph,
                  int parabolic, const double *chi, const double *S, const double *B,
                  const double *core_face, const double *core_grad, double I_out, double I_irr,
                  double *J, double *lstar)
{
    orc_sph g;
    sph_init(&g, nr, nt, np, r_in, r_out);
    const long N = (long)nr * nt * np;
    const int nO = nth * nph;
    double *mu = malloc(sizeof(double) * nO), *phi = malloc(sizeof(double) * nO);
    double *dir = malloc(sizeof(double) * 3 * nO), *w = malloc(sizeof(double) * nO);
    orc_directions(nth, nph, mu, phi, dir, w);
    int cap = orc_sph_kcap(nr, nt, np);
    int *vox = malloc(sizeof(int) * cap);
    double *len = malloc(sizeof(double) * cap), *chil = malloc(sizeof(double) * cap);
    double *Sp = malloc(sizeof(double) * cap), *I = malloc(sizeof(double) * cap);
    double *E = malloc(sizeof(double) * cap), *al = malloc(sizeof(double) * cap);
    double *be = malloc(sizeof(double) * cap), *ga = malloc(sizeof(double) * cap);
    double *num = malloc(sizeof(double) * N), *den = malloc(sizeof(double) * N);
    double *numL = lstar ? malloc(sizeof(double) * 27 * N) : NULL;
    char *hit = malloc(N);
    int err = 0;
    memset(J, 0, sizeof(double) * N);
    if (lstar) memset(lstar, 0, sizeof(double) * 27 * N);
    for (int o = 0; o < nO && !err; o++) {
        const double *d = dir + 3 * o;
        memset(num, 0, sizeof(double) * N);
        memset(den, 0, sizeof(double) * N);
        memset(hit, 0, N);
        if (numL) memset(numL, 0, sizeof(double) * 27 * N);
        for (long v = 0; v < N; v++) {
            if (hit[v]) continue;
            int ir = (int)(v % nr), it = (int)((v / nr) % nt), ip = (int)(v / ((long)nr * nt));
            double P[3] = {g.rc[ir] * g.stc[it] * g.cpc[ip], g.rc[ir] * g.stc[it] * g.spc[ip],
                           g.rc[ir] * g.ctc[it]};
            int ec;
            double pin[3];
            int K = orc_sph_trace(&g, P, d, cap, vox, len, &ec, pin);
            if (K < 0) { err = -2; break; }
            hit[v] = 1;
            for (int k = 0; k < K; k++) {
                hit[vox[k]] = 1;
                chil[k] = chi[vox[k]] * len[k];
                Sp[k] = S[vox[k]];
            }
            double I0;
            if (ec && core_face) {
                const int f = vox[0] / nr;  /* it + nt ip of the first cell */
                I0 = core_face[f];
                if (core_grad) {
                    const double mu = (pin[0] * d[0] + pin[1] * d[1] + pin[2] * d[2]) / r_in;
                    I0 += mu * core_grad[f];
                }
            } else if (ec) {
                I0 = B[vox[0]];
            } else {
                I0 = (pin[0] > 0.0 && d[0] < 0.0) ? I_irr : I_out;
            }
            orc_ray_fs(K, chil, Sp, I0, parabolic, I, E, al, be, ga);
            for (int k = 0; k < K; k++) {
                num[vox[k]] += len[k] * I[k];
                den[vox[k]] += len[k];
                if (!numL) continue;
                int vk = vox[k];
                int jend = k + 1 < K ? k + 1 : k;
                int j0 = jend;
                while (j0 - 1 >= 0 && sph_nb_code(nr, nt, np, vox[j0 - 1], vk) >= 0) j0--;
                for (int j = j0; j <= jend; j++) {
                    int dc = sph_nb_code(nr, nt, np, vox[j], vk);
                    if (dc < 0) continue;
                    numL[27 * (long)vk + dc] += len[k] * sph_dIdS(k, j, E, al, be, ga);
                }
            }
        }
        for (long v = 0; v < N; v++) {
            if (!(den[v] > 0.0)) { err = -3; continue; }
            J[v] += w[o] * (num[v] / den[v]);
            if (numL)
                for (int c = 0; c < 27; c++) lstar[27 * v + c] += w[o] * (numL[27 * v + c] / den[v]);
        }
    }
    free(vox); free(len); free(chil); free(Sp); free(I); free(E); free(al); free(be); free(ga);
    free(num); free(den); free(numL); free(hit); free(mu); free(phi); free(dir); free(w);
    sph_free(&g);
    return err;
}

int orc_fs_sph(int nr, int nt, int np, double r_in, double r_out, int nth, int nph,
               int parabolic, const double *chi, const double *S, const double *B,
               double I_out, double I_irr, double *J, double *lstar)
{
    return orc_fs_sph_bc(nr, nt, np, r_in, r_out, nth, nph, parabolic, chi, S, B, NULL, NULL,
                         I_out, I_irr, J, lstar);
}
