"""Pins of the spherical-grid oracle (paper Sec. 3.2 geometry; readings in
oracle/rt3d_oracle_sph.c): cells located independently with acos/atan2,
chord sums, entry points, coverage of every voxel by every solid angle, the
homogeneous-medium identity and the LTE closed form."""
import math

import numpy as np
import pytest

import oracle

R_IN, R_OUT = 1.0, 1.3


def _cell_by_angles(p, n):
    nr, nt, np_ = n
    r = math.sqrt(p[0] ** 2 + p[1] ** 2 + p[2] ** 2)
    ir = int(math.floor(nr * math.log(r / R_IN) / math.log(R_OUT / R_IN)))
    th = math.acos(max(-1.0, min(1.0, p[2] / r)))
    it = int(math.floor(th / math.pi * nt))
    ph = math.atan2(p[1], p[0]) % (2 * math.pi)
    ip = int(math.floor(ph / (2 * math.pi) * np_))
    # distance (in cell units) of the point from the nearest edge
    fr = nr * math.log(r / R_IN) / math.log(R_OUT / R_IN)
    ft, fp = th / math.pi * nt, ph / (2 * math.pi) * np_
    margin = min(abs(f - round(f)) for f in (fr, ft, fp))
    return min(max(ir, 0), nr - 1) + nr * (min(it, nt - 1) + nt * (ip % np_)), margin


@pytest.mark.parametrize("n", [(9, 7, 12), (5, 9, 16)])
def test_sph_trace_cells_chords_and_entry(n):
    nr, nt, np_ = n
    mu, phi, d, w = oracle.directions(4, 6)
    rng = np.random.default_rng(1)
    for o in range(0, 24, 3):
        for v in rng.integers(0, nr * nt * np_, 6):
            vox, ln, core, pin = oracle.sph_trace(n, d[o], int(v))
            assert np.all(ln > 0)
            r_in = np.linalg.norm(pin)
            assert abs(r_in - (R_IN if core else R_OUT)) < 1e-12
            # the launching voxel is on the ray; consecutive cells are neighbours
            assert int(v) in set(vox.tolist())
            ir, it, ip = vox % nr, (vox // nr) % nt, vox // (nr * nt)
            assert np.all(np.abs(np.diff(ir)) <= 1) and np.all(np.abs(np.diff(it)) <= 1)
            dp = np.diff(ip) % np_
            assert np.all((dp <= 1) | (dp == np_ - 1))
            # every interval's midpoint cell agrees with acos/atan2
            t = np.concatenate([[0.0], np.cumsum(ln)])
            for k in range(len(vox)):
                m = 0.5 * (t[k] + t[k + 1])
                p = pin + m * d[o]
                cell, margin = _cell_by_angles(p, n)
                if margin > 1e-7:
                    assert cell == vox[k], (o, v, k)


def test_sph_every_voxel_is_covered_and_homogeneous_identity():
    n = (6, 5, 8)
    shape = (8, 5, 6)
    chi = np.full(shape, 3.0)
    S = np.full(shape, 1.7)
    J = oracle.fs_sph(chi, S, S, 3, 6, True, I_out=1.7, I_irr=1.7)
    assert np.max(np.abs(J - 1.7)) < 1.7 * 4e-15
    rays = oracle.sph_rays(n, 3, 6, 4)
    assert 0 < len(rays) < np.prod(n)


def test_sph_lte_closed_form():
    """S = B = 1 everywhere, no incoming intensity at the outer sphere, I = 1
    from the core: along a ray entering from outside I = 1 - exp(-tau), from the
    core I = 1."""
    n = (5, 5, 8)
    nr, nt, np_ = n
    shape = (np_, nt, nr)
    rng = np.random.default_rng(3)
    chi = 10 ** rng.uniform(-1, 1, shape)
    ones = np.ones(shape)
    nth, nph = 2, 4
    J = oracle.fs_sph(chi, ones, ones, nth, nph, False, I_out=0.0, I_irr=0.0)
    mu, phi, d, w = oracle.directions(nth, nph)
    N = chi.size
    Jref = np.zeros(N)
    cflat = chi.reshape(-1)
    for o in range(nth * nph):
        num = np.zeros(N)
        den = np.zeros(N)
        for v in oracle.sph_rays(n, nth, nph, o):
            vox, ln, core, pin = oracle.sph_trace(n, d[o], int(v))
            if core:
                I = np.ones(len(vox))
            else:
                chil = cflat[vox] * ln
                tau = np.concatenate([[0.0], np.cumsum(chil)[:-1]]) + 0.5 * chil
                I = -np.expm1(-tau)
            np.add.at(num, vox, ln * I)
            np.add.at(den, vox, ln)
        Jref += w[o] * num / den
    assert np.max(np.abs(J.reshape(-1) - Jref) / Jref) < 1e-13


@pytest.mark.parametrize("parabolic", [False, True])
def test_sph_boundary_intensities_attenuate(parabolic):
    """S = 0 in every cell: the intensity along a characteristic is its entry
    intensity times exp(-tau) (tau from the entry to the chord midpoint), so J
    follows from the three boundary rules alone: B of the first cell through
    the core, I_irr where the entry point on the outer sphere has x > 0 and the
    direction d_x < 0, I_out elsewhere on the outer sphere. The entry point
    comes from the trace; the rule is applied here from its statement."""
    n = (5, 4, 8)
    nr, nt, np_ = n
    shape = (np_, nt, nr)
    rng = np.random.default_rng(4)
    chi = 10 ** rng.uniform(-1, 0.5, shape)
    B = 1 + rng.uniform(0, 1, shape)
    zero = np.zeros(shape)
    I_out, I_irr = 0.3, 2.0
    nth, nph = 2, 6
    J = oracle.fs_sph(chi, zero, B, nth, nph, parabolic, I_out=I_out, I_irr=I_irr)
    mu, phi, d, w = oracle.directions(nth, nph)
    N = chi.size
    Jref = np.zeros(N)
    cflat, bflat = chi.reshape(-1), B.reshape(-1)
    n_irr = 0
    for o in range(nth * nph):
        num = np.zeros(N)
        den = np.zeros(N)
        for v in oracle.sph_rays(n, nth, nph, o):
            vox, ln, core, pin = oracle.sph_trace(n, d[o], int(v))
            if core:
                I0 = bflat[vox[0]]
            elif pin[0] > 0.0 and d[o][0] < 0.0:
                I0 = I_irr
                n_irr += 1
            else:
                I0 = I_out
            chil = cflat[vox] * ln
            tau = np.concatenate([[0.0], np.cumsum(chil)[:-1]]) + 0.5 * chil
            np.add.at(num, vox, ln * I0 * np.exp(-tau))
            np.add.at(den, vox, ln)
        Jref += w[o] * num / den
    assert n_irr > 0
    assert np.max(np.abs(J.reshape(-1) - Jref) / Jref) < 1e-13


def _sph_band_vs_lambda(n, nth, nph, parabolic, seed=5):
    nr, nt, np_ = n
    shape = (np_, nt, nr)
    rng = np.random.default_rng(seed)
    chi = 10 ** rng.uniform(-1, 0.5, shape)
    zero = np.zeros(shape)
    _, L = oracle.fs_sph(chi, np.ones(shape), zero, nth, nph, parabolic, lstar=True)
    N = chi.size
    M = np.zeros((N, N))
    e = np.zeros(N)
    for u in range(N):
        e[:] = 0.0
        e[u] = 1.0
        M[:, u] = oracle.fs_sph(chi, e.reshape(shape), zero, nth, nph, parabolic).reshape(-1)
    diag, off = [], []
    for v in range(N):
        ir, it, ip = v % nr, (v // nr) % nt, v // (nr * nt)
        scale = np.max(np.abs(M[v]))
        for d in range(27):
            dr, dt, dp = d % 3 - 1, (d // 3) % 3 - 1, d // 9 - 1
            rr, tt, pp = ir + dr, it + dt, (ip + dp) % np_
            if not (0 <= rr < nr and 0 <= tt < nt):
                assert L[v, d] == 0.0
                continue
            u = rr + nr * (tt + nt * pp)
            (diag if d == 13 else off).append((L[v, d] - M[v, u]) / scale)
    return np.array(diag), np.array(off)


@pytest.mark.parametrize("parabolic", [False, True])
def test_sph_lambda_star_is_the_band_of_lambda_on_a_fine_grid(parabolic):
    """Lambda* (the passage-local window) against the brute-force Lambda built
    column by column: on cells small enough that no characteristic leaves a
    cell's 3x3x3 neighbourhood and comes back, the whole band is exact."""
    diag, off = _sph_band_vs_lambda((3, 12, 24), 2, 4, parabolic)
    assert np.max(np.abs(diag)) < 1e-14
    assert np.max(np.abs(off)) < 1e-14


def test_sph_lambda_star_on_coarse_cells():
    """On coarse cells (45 degrees in phi) a straight characteristic can leave a
    neighbourhood and re-enter it; the passage-local window then omits the
    later passage. The diagonal stays exact, and with linear interpolation
    (non-negative weights) no band entry exceeds Lambda's."""
    diag, off = _sph_band_vs_lambda((5, 4, 8), 2, 6, False)
    assert np.max(np.abs(diag)) < 1e-14
    assert np.max(off) < 1e-14
    assert np.min(off) < -1e-3  # the effect is real at this resolution


# ---- the LTE diffusion inner boundary on the core sphere (Sec. 3.2)

def _radial_centres(nr):
    re = R_IN * (R_OUT / R_IN) ** (np.arange(nr + 1) / nr)
    re[0], re[-1] = R_IN, R_OUT
    return np.sqrt(re[:-1] * re[1:])


def test_sph_diffusion_faces_exact_for_a_linear_profile():
    """B linear in the radial optical depth with chi constant along each
    radius: the one-sided difference is the exact dB/dtau and the carried
    value the exact B on the core sphere; one shell: no gradient."""
    n = (6, 5, 8)
    nr, nt, np_ = n
    rc = _radial_centres(nr)
    rng = np.random.default_rng(0)
    chic = 10 ** rng.uniform(-1, 1, (np_, nt))
    a = rng.uniform(0.5, 2, (np_, nt))
    b = rng.uniform(-1, 3, (np_, nt))
    chi = np.broadcast_to(chic[:, :, None], chi_shape := (np_, nt, nr)).copy()
    tau = chic[:, :, None] * (R_OUT - rc[None, None, :])
    B = a[:, :, None] + b[:, :, None] * tau
    I_face, grad = oracle.diffusion_bc_sph(chi, B)
    assert np.allclose(grad, b, rtol=1e-12, atol=1e-12)
    assert np.allclose(I_face, a + b * chic * (R_OUT - R_IN), rtol=1e-13, atol=1e-13)
    I1, g1 = oracle.diffusion_bc_sph(chi[:, :, :1], B[:, :, :1])
    assert np.array_equal(g1, np.zeros((np_, nt))) and np.array_equal(I1, B[:, :, 0])
    assert chi.shape == chi_shape
    # chi of the two innermost shells enters dB/dtau through their mean (a
    # swap leaves it), the carried face value through the innermost alone
    chi2 = 10 ** rng.uniform(-1, 1, chi.shape)
    sw = chi2.copy()
    sw[:, :, 0], sw[:, :, 1] = chi2[:, :, 1], chi2[:, :, 0]
    Ia, ga = oracle.diffusion_bc_sph(chi2, B)
    Ib, gb = oracle.diffusion_bc_sph(sw, B)
    assert np.allclose(ga, gb, rtol=1e-14, atol=0)
    assert np.allclose(Ia - B[:, :, 0], chi2[:, :, 0] * (rc[0] - R_IN) * ga, rtol=1e-13)
    assert np.allclose(Ib - B[:, :, 0], chi2[:, :, 1] * (rc[0] - R_IN) * gb, rtol=1e-13)
    assert not np.allclose(Ia, Ib, rtol=1e-6)


def test_sph_diffusion_gradient_term_brute_force():
    """Optically thin (chi = 1e-10), S = 0, I_face = 0: every ray keeps its
    entry intensity, so J of a cell is the chord-weighted mean over the rays
    of each angle of mu g for the rays from the core, with mu recomputed here
    from the impact parameter |p x d| of the entry point (not the oracle's
    dot product)."""
    n = (4, 3, 6)
    nr, nt, np_ = n
    nth, nph = 2, 4
    rng = np.random.default_rng(5)
    g = rng.uniform(0.5, 2.0, (np_, nt))
    chi = np.full((np_, nt, nr), 1e-10)
    zero = np.zeros(chi.shape)
    J = oracle.fs_sph(chi, zero, zero, nth, nph, False, core_face=np.zeros((np_, nt)),
                      core_grad=g)
    mu, phi, d, w = oracle.directions(nth, nph)
    N = nr * nt * np_
    Jb = np.zeros(N)
    ncore = 0
    for o in range(nth * nph):
        num, den = np.zeros(N), np.zeros(N)
        for v in oracle.sph_rays(n, nth, nph, o):
            vox, ln, core, pin = oracle.sph_trace(n, d[o], int(v))
            I0 = 0.0
            if core:
                p = np.linalg.norm(np.cross(pin, d[o]))
                m = math.sqrt(max(0.0, 1.0 - (p / R_IN) ** 2))
                f = vox[0] // nr
                I0 = m * g.reshape(-1)[f]
                ncore += 1
            np.add.at(num, vox, ln * I0)
            np.add.at(den, vox, ln)
        Jb += w[o] * num / den
    assert ncore > 0
    assert np.allclose(J.reshape(-1), Jb, rtol=1e-8, atol=1e-12)
    assert np.max(J) > 0.1


@pytest.mark.parametrize("nr", [12, 24])
def test_sph_diffusion_boundary_in_the_grey_lte_limit(nr):
    """Grey LTE atmosphere (S = B = 3/4 (tau + 2/3), chi ~ r^-12, innermost
    shell of optical thickness ~1): entering with I = B of the first cell
    leaves the innermost mean intensity 16 % below B; the diffusion condition
    brings it within 4 % (the remainder is the curvature of the shell), and
    closer with finer shells."""
    n = (nr, 4, 8)
    rc = _radial_centres(nr)
    chi = np.broadcast_to(12 * rc ** -12.0, (8, 4, nr)).copy()
    tau = rc ** -11.0 - R_OUT ** -11.0
    B = np.broadcast_to(0.75 * (tau + 2.0 / 3.0), (8, 4, nr)).copy()
    I_face, grad = oracle.diffusion_bc_sph(chi, B)
    Jd = oracle.fs_sph(chi, B, B, 4, 8, True, core_face=I_face, core_grad=grad)
    Jp = oracle.fs_sph(chi, B, B, 4, 8, True)
    dd = np.mean(Jd[:, :, 0] / B[:, :, 0] - 1)
    dp = np.mean(Jp[:, :, 0] / B[:, :, 0] - 1)
    assert dp < -0.15
    assert abs(dd) < 0.04 and abs(dd) < 0.25 * abs(dp)
    # the gradient term is what does it: the carried face value alone is not enough
    Jf = oracle.fs_sph(chi, B, B, 4, 8, True, core_face=I_face)
    assert np.mean(Jf[:, :, 0] / B[:, :, 0] - 1) < -0.1
