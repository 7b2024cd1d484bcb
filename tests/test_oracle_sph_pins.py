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
