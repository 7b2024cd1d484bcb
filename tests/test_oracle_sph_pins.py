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
