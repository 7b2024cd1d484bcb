"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms of the RTE (Sec. 2.1, Eq. 1), high-precision quadrature of the
interpolation integrals, brute-force geometry, the brute-force Lambda matrix
(Eq. frmsol, J = Lambda S) and the dense direct solve of the scattering
problem that the ALI iteration (Eqs. alisol, alodef, alo) converges to, the
sqrt(eps) surface law and the spectral radius of the Lambda iteration
(Sec. 2.2, lambda_max ~ (1-eps)(1-1/T)).
"""
from fractions import Fraction
import math

import mpmath
import numpy as np
import pytest

import oracle
from paper_2102_01734_gb300 import inputs

mpmath.mp.dps = 40


# ------------------------------------------------------------ direction set
def test_directions_midpoint_grid():
    mu, phi, d, w = oracle.directions(8, 16)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-15)
    # midpoints, equally spaced in mu and phi
    assert np.allclose(np.unique(mu), -1 + (2 * np.arange(8) + 1) / 8.0, atol=0)
    assert np.allclose(np.unique(phi), (2 * np.arange(16) + 1) * np.pi / 16, atol=1e-15)
    assert np.all(np.abs(d) > 1e-3)  # no axis-parallel component, mu != 0
    # the set is symmetric under mu -> -mu
    assert np.allclose(np.sort(mu), -np.sort(mu)[::-1])


# ---------------------------------------------------- exponential integrals
def _e012_exact(u):
    u = mpmath.mpf(u)
    e0 = -mpmath.expm1(-u)
    e1 = mpmath.quad(lambda t: t * mpmath.exp(-(u - t)), [0, u])
    e2 = mpmath.quad(lambda t: t * t * mpmath.exp(-(u - t)), [0, u])
    return e0, e1, e2


@pytest.mark.parametrize("u", [1e-12, 3e-7, 1e-4, 0.01, 0.2, 0.4999, 0.5, 0.7, 1.0, 3.3, 20.0,
                               150.0, 2500.0])
def test_e012_against_quadrature(u):
    got = oracle.e012(u)
    ref = _e012_exact(u)
    for g, r in zip(got, ref):
        assert abs(g - float(r)) <= 4e-15 * abs(float(r)), (u, g, float(r))


def _lagrange_integrals(u, w):
    """Integrals over [0,u] of exp(-(u-t)) times the three Lagrange basis
    parabolas through t = 0, u, u+w (mpmath quadrature)."""
    u, w = mpmath.mpf(u), mpmath.mpf(w)
    K = lambda f: mpmath.quad(lambda t: f(t) * mpmath.exp(-(u - t)), [0, u])
    a = K(lambda t: (t - u) * (t - u - w) / (u * (u + w)))
    b = K(lambda t: t * (t - u - w) / (u * (u - u - w)))
    g = K(lambda t: t * (t - u) / ((u + w) * w))
    return a, b, g


@pytest.mark.parametrize("u,w", [(1e-5, 2e-5), (0.01, 0.03), (0.3, 0.2), (0.45, 4.0),
                                 (0.5, 0.25), (0.2, 0.1)])
def test_parabolic_coefficients_integrate_the_parabola(u, w):
    """Optically thin intervals with spacing ratio u/w <= 2: the full
    Olson-Kunasz parabola."""
    E, a, b, g = oracle.coef(True, u, w)
    ra, rb, rg = _lagrange_integrals(u, w)
    scale = float(-mpmath.expm1(-u))  # e0: the size of the sum alpha+beta+gamma
    assert abs(E - math.exp(-u)) <= 1e-16 * max(1.0, math.exp(-u))
    for x, r in ((a, ra), (b, rb), (g, rg)):
        assert abs(x - float(r)) <= 1e-13 * scale, (u, w, x, float(r))
    assert abs(a + b + g - scale) <= 1e-14 * scale
    assert g < 0.0


def _linear_integrals(u):
    um = mpmath.mpf(u)
    ra = mpmath.quad(lambda t: (1 - t / um) * mpmath.exp(-(um - t)), [0, um])
    rb = mpmath.quad(lambda t: (t / um) * mpmath.exp(-(um - t)), [0, um])
    return ra, rb


@pytest.mark.parametrize("u,w", [(1.0, 1.0), (2.0, 1.5), (30.0, 45.0), (300.0, 100.0),
                                 (0.3, 0.05), (0.1, 0.02)])
def test_thick_or_skewed_intervals_use_the_linear_weights(u, w):
    """u >= 1 or u/w >= 4: the parabola is switched off, every weight of the
    interval is non-negative."""
    E, a, b, g = oracle.coef(True, u, w)
    ra, rb = _linear_integrals(u)
    scale = float(-mpmath.expm1(-u))
    assert g == 0.0
    assert abs(a - float(ra)) <= 1e-13 * scale and abs(b - float(rb)) <= 1e-13 * scale
    assert a >= 0.0 and b >= 0.0


def test_parabolic_weight_ramps_are_continuous():
    """No jump in the coefficients across the blend ramps (u = 1/2, 1 and
    u/w = 2, 4), and alpha+beta+gamma = e0 everywhere."""
    for u0, w0 in ((0.5, 1.0), (1.0, 1.0), (0.4, 0.2), (0.4, 0.1)):
        for du in (1e-9, -1e-9):
            c1 = np.array(oracle.coef(True, u0 + du, w0))
            c0 = np.array(oracle.coef(True, u0, w0))
            assert np.max(np.abs(c1 - c0)) < 1e-7
    rng = np.random.default_rng(1)
    for u, w in 10 ** rng.uniform(-4, 2, (200, 2)):
        E, a, b, g = oracle.coef(True, u, w)
        e0 = -math.expm1(-u)
        assert abs(a + b + g - e0) <= 1e-14 * e0
        f = oracle.parab_weight(u, w)
        assert 0.0 <= f <= 1.0
        assert (f == 0.0) == (g == 0.0)


@pytest.mark.parametrize("u", [1e-9, 0.02, 0.6, 7.0, 800.0])
def test_linear_coefficients_integrate_the_line(u):
    E, a, b, g = oracle.coef(False, u, 0.0)
    um = mpmath.mpf(u)
    ra = mpmath.quad(lambda t: (1 - t / um) * mpmath.exp(-(um - t)), [0, um])
    rb = mpmath.quad(lambda t: (t / um) * mpmath.exp(-(um - t)), [0, um])
    scale = float(-mpmath.expm1(-um))
    assert g == 0.0
    assert abs(a - float(ra)) <= 1e-13 * scale
    assert abs(b - float(rb)) <= 1e-13 * scale


def test_vacuum_interval():
    assert oracle.coef(True, 0.0, 1.0) == (1.0, 0.0, 0.0, 0.0)


# ------------------------------------------- exactness along a characteristic
def _analytic_I(tau, I_start, k0, k1, Sfun):
    """I at tau[k1] from I_start at tau[k0]: I0 e^{-dt} + int S e^{-(t1-t)} dt."""
    t0, t1 = mpmath.mpf(tau[k0]), mpmath.mpf(tau[k1])
    pts = [mpmath.mpf(t) for t in tau[k0:k1 + 1]]
    integ = mpmath.quad(lambda t: Sfun(t) * mpmath.exp(-(t1 - t)), pts)
    return I_start * mpmath.exp(-(t1 - t0)) + integ


@pytest.mark.parametrize("parabolic", [False, True])
def test_polynomial_source_is_integrated_exactly(parabolic):
    rng = np.random.default_rng(7)
    K = 14
    # chi*l per point; the parabolic case stays where the full parabola applies
    # (intervals <= 1/2, neighbouring intervals within a factor 2)
    chil = rng.uniform(0.16, 0.3, K) if parabolic else 10.0 ** rng.uniform(-3, 1.3, K)
    # point optical depths: tau_k = sum_{i<k} chil_i + chil_k / 2 (entry at 0)
    tau = np.concatenate([[0.0], np.cumsum(chil)[:-1]]) + 0.5 * chil
    tau_m = [mpmath.mpf(0)]
    acc = mpmath.mpf(0)
    for i in range(K):
        tau_m.append(acc + mpmath.mpf(chil[i]) / 2)
        acc += mpmath.mpf(chil[i])
    tau_m = tau_m[1:]
    c0, c1, c2 = 1.3, -0.21, (0.017 if parabolic else 0.0)
    Sfun = lambda t: c0 + c1 * t + c2 * t * t
    S = np.array([float(Sfun(mpmath.mpf(t))) for t in tau_m])
    I, E, al, be, ga = oracle.ray_fs(chil, S, 0.7, parabolic)
    # from point 1 on, every interval but the last one is interpolated exactly
    last = K - 2 if parabolic else K - 1
    ref = _analytic_I(tau_m, mpmath.mpf(I[0]), 0, last, Sfun)
    assert abs(I[last] - float(ref)) <= 1e-13 * abs(float(ref))


def test_homogeneous_constant_source_closed_form():
    """I = S (1 - e^-tau) + I0 e^-tau for constant S (the closed form of the
    transfer equation in a homogeneous medium)."""
    chil = np.full(40, 0.37)
    S = np.full(40, 2.0)
    for parabolic in (False, True):
        I, *_ = oracle.ray_fs(chil, S, 0.5, parabolic)
        tau = 0.37 * (np.arange(40) + 0.5)
        ref = 2.0 * (1 - np.exp(-tau)) + 0.5 * np.exp(-tau)
        assert np.max(np.abs(I - ref) / ref) < 1e-14


# --------------------------------------------------------------- the tracer
def _brute_trace(shape, d, x0, y0):
    """All plane crossings enumerated and sorted; the cell of every interval
    found from the exact (rational) midpoint of the interval."""
    nz, ny, nx = shape
    ax, ay, az = abs(d[0]), abs(d[1]), abs(d[2])
    T = nz / az
    ts = set()
    for a in (ax, ay):
        if a > 0:
            m = 1
            while True:
                t = (m - 0.5) / a
                if t >= T:
                    break
                ts.add(t)
                m += 1
    for m in range(1, nz + 1):
        ts.add(m / az)
    ts = sorted(ts)
    ts = [t for t in ts if t <= nz / az]
    prev = 0.0
    vox, ln = [], []
    for t in ts:
        mid = (Fraction(prev) + Fraction(t)) / 2
        px = Fraction(x0) + Fraction(1, 2) + mid * Fraction(d[0])
        py = Fraction(y0) + Fraction(1, 2) + mid * Fraction(d[1])
        pz = (Fraction(nz) if d[2] < 0 else Fraction(0)) + mid * Fraction(d[2])
        ix, iy, iz = math.floor(px) % nx, math.floor(py) % ny, math.floor(pz)
        vox.append(ix + nx * (iy + ny * iz))
        ln.append(t - prev)
        prev = t
    return np.array(vox), np.array(ln)


@pytest.mark.parametrize("nth,nph", [(6, 10), (2, 4), (4, 6)])
def test_tracer_against_brute_force(nth, nph):
    shape = (5, 6, 7)
    mu, phi, d, w = oracle.directions(nth, nph)
    for o in range(nth * nph):
        for (x0, y0) in ((0, 0), (3, 5), (6, 2)):
            vox, ln = oracle.trace_cart(shape, d[o], x0, y0)
            bv, bl = _brute_trace(shape, d[o], x0, y0)
            assert np.array_equal(vox, bv), (o, x0, y0)
            assert np.array_equal(ln, bl)
            assert np.all(ln > 0)


def test_chord_sum_per_voxel_is_one_over_mu():
    shape = (4, 5, 6)
    nz, ny, nx = shape
    mu, phi, d, w = oracle.directions(6, 8)
    for o in range(len(mu)):
        tot = np.zeros(nx * ny * nz)
        for y0 in range(ny):
            for x0 in range(nx):
                vox, ln = oracle.trace_cart(shape, d[o], x0, y0)
                np.add.at(tot, vox, ln)
        assert np.allclose(tot, 1.0 / abs(mu[o]), rtol=1e-13, atol=0)


# ----------------------------------------------------------- formal solution
def test_homogeneous_medium_constant_source():
    shape = (6, 5, 7)
    chi = np.full(shape, 0.7)
    S = np.full(shape, 2.5)
    for parabolic in (False, True):
        J = oracle.fs_cart(chi, S, 4, 8, parabolic, bc={"I_top": 2.5, "I_bottom": 2.5})
        assert np.max(np.abs(J - 2.5)) <= 2.5 * 2e-15


def test_vacuum_carries_the_boundary_intensities():
    """chi = 0 everywhere: intensities stay at their boundary values, so J is
    the direction average 1/2 (I_top + I_bottom) whatever S is (half of the
    midpoint directions enter at the top, half at the bottom)."""
    rng = np.random.default_rng(4)
    shape = (5, 6, 7)
    S = rng.uniform(0.5, 2.0, shape)
    for parabolic in (False, True):
        J = oracle.fs_cart(np.zeros(shape), S, 4, 8, parabolic, bc={"I_top": 0.3, "I_bottom": 1.7})
        assert np.max(np.abs(J - 1.0)) <= 1e-15


def test_lte_slab_closed_form():
    """S = B = 1, eps = 1, I_top = 0, I_bottom = B: along every point the
    intensity is B (1 - e^{-tau_top}) downwards and B upwards; J is the chord
    weighted average of these closed forms."""
    nz, ny, nx = 9, 4, 4
    chi1 = inputs.vertical_chi(nz)
    chi = np.broadcast_to(chi1[:, None, None], (nz, ny, nx)).copy()
    S = np.ones(chi.shape)
    nth, nph = 4, 6
    mu, phi, d, w = oracle.directions(nth, nph)
    Jref = np.zeros(nz)
    for o in range(nth * nph):
        vox, ln = oracle.trace_cart(chi.shape, d[o], 0, 0)
        z = vox // (nx * ny)
        if mu[o] > 0:
            I = np.ones(len(vox))
        else:
            chil = chi1[z] * ln
            tau = np.concatenate([[0.0], np.cumsum(chil)[:-1]]) + 0.5 * chil
            I = -np.expm1(-tau)
        num = np.bincount(z, ln * I, nz)
        den = np.bincount(z, ln, nz)
        Jref += w[o] * num / den
    for parabolic in (False, True):
        J = oracle.fs_cart(chi, S, nth, nph, parabolic, bc={"I_top": 0.0, "I_bottom": 1.0})
        assert np.max(np.abs(J - Jref[:, None, None]) / Jref[:, None, None]) < 1e-14
    # deep inside the optically thick LTE slab J -> B
    assert abs(J[0].mean() - 1.0) < 1e-12
    assert abs(J[1].mean() - 1.0) < 1e-4
    assert abs(J[-1].mean() - 0.5) < 0.05  # surface: only the upward half is bright


def test_translation_invariance():
    nz, ny, nx = 7, 5, 6
    chi = np.broadcast_to(inputs.vertical_chi(nz)[:, None, None], (nz, ny, nx)).copy()
    S = np.broadcast_to(np.linspace(0.3, 2.0, nz)[:, None, None], chi.shape).copy()
    J, L = oracle.fs_cart(chi, S, 4, 6, True, bc={"I_top": 0.1, "I_bottom": 2.0}, lstar=True)
    spread = np.max(np.ptp(J.reshape(nz, -1), axis=1) / J.reshape(nz, -1).mean(axis=1))
    assert spread < 1e-14
    Lr = L.reshape(nz, ny * nx, 27)
    assert np.max(np.ptp(Lr, axis=1)) < 1e-14


def test_linearity():
    rng = np.random.default_rng(3)
    shape = (5, 4, 6)
    chi = 10 ** rng.uniform(-2, 1, shape)
    S1, S2 = rng.uniform(0, 1, shape), rng.uniform(0, 1, shape)
    for parabolic in (False, True):
        J1 = oracle.fs_cart(chi, S1, 4, 6, parabolic)
        J2 = oracle.fs_cart(chi, S2, 4, 6, parabolic)
        J12 = oracle.fs_cart(chi, 2.0 * S1 - 0.5 * S2, 4, 6, parabolic)
        assert np.max(np.abs(J12 - (2.0 * J1 - 0.5 * J2))) < 1e-13 * np.max(np.abs(J12))


def test_voxel_route_matches_full_solution():
    rng = np.random.default_rng(5)
    shape = (6, 5, 7)
    chi = 10 ** rng.uniform(-2, 1.5, shape)
    S = rng.uniform(0.2, 2, shape)
    bc = {"I_top": 0.0, "I_bottom": rng.uniform(0.5, 1.5, (5, 7))}
    J, L = oracle.fs_cart(chi, S, 4, 6, True, bc=bc, lstar=True)
    for v in (0, 17, 101, chi.size - 1):
        Jv, row = oracle.fs_cart_voxel(chi, S, 4, 6, v, True, bc=bc, lstar=True)
        assert abs(Jv - J.reshape(-1)[v]) <= 1e-14 * abs(Jv)
        assert np.max(np.abs(row - L[v])) <= 1e-14 * np.max(np.abs(row))


# ---------------------------------------------------------------- Lambda*
def _band_of(M, shape):
    nz, ny, nx = shape
    N = M.shape[0]
    band = np.zeros((N, 27))
    for v in range(N):
        x, y, z = v % nx, (v // nx) % ny, v // (nx * ny)
        for c in range(27):
            dx, dy, dz = c % 3 - 1, (c // 3) % 3 - 1, c // 9 - 1
            if not 0 <= z + dz < nz:
                continue
            u = (x + dx) % nx + nx * ((y + dy) % ny + ny * (z + dz))
            band[v, c] = M[v, u]
    return band


@pytest.mark.parametrize("parabolic", [False, True])
def test_lstar_equals_band_of_brute_force_lambda(parabolic):
    """9x9x4 box, mu = +-1/2: a characteristic moves < 7 cells sideways, so it
    never re-enters a 3x3x3 neighbourhood and Lambda* is the exact band."""
    rng = np.random.default_rng(11)
    shape = (4, 9, 9)
    chi = 10 ** rng.uniform(-1.5, 0.7, shape)
    S = rng.uniform(0.5, 1.5, shape)
    J, L = oracle.fs_cart(chi, S, 2, 5, parabolic, lstar=True)
    M = oracle.lambda_matrix(chi, 2, 5, parabolic)
    # Lambda S reproduces the formal solution (zero boundary intensity)
    assert np.max(np.abs(M @ S.reshape(-1) - J.reshape(-1))) < 1e-13
    band = _band_of(M, shape)
    assert np.max(np.abs(band - L)) < 1e-13
    # Lambda* holds no entry outside the box in z
    z = np.arange(chi.size) // 81
    assert np.all(L[z == 0][:, :9] == 0) and np.all(L[z == 3][:, 18:] == 0)


@pytest.mark.parametrize("n,nth,nph", [((4, 4, 5), 4, 6), ((5, 4, 6), 4, 4)])
def test_lstar_on_wrapping_characteristics(n, nth, nph):
    """Small periodic boxes with shallow directions: characteristics wrap
    around x, y and re-enter a voxel's 3x3x3 neighbourhood, and the
    passage-local window leaves the later passage out. With the linear
    weights (all contributions non-negative) no band entry then exceeds the
    brute-force Lambda's, and some fall measurably below it."""
    nx, ny, nz = n
    shape = (nz, ny, nx)
    rng = np.random.default_rng(3)
    chi = 10 ** rng.uniform(-1, 0, shape)
    _, L = oracle.fs_cart(chi, np.ones(shape), nth, nph, False, lstar=True)
    M = oracle.lambda_matrix(chi, nth, nph, False)
    diff = (_band_of(M, shape) - L) / np.max(np.abs(M), axis=1, keepdims=True)
    assert np.min(diff) > -1e-14
    assert np.max(diff) > 0.05


# ----------------------------------------------------------------- the ALI
def test_os_jacobi_solves_the_band_system():
    rng = np.random.default_rng(2)
    shape = (5, 4, 6)
    chi = 10 ** rng.uniform(-1, 1, shape)
    S = np.ones(shape)
    _, L = oracle.fs_cart(chi, S, 4, 6, False, lstar=True)
    eps = 10 ** rng.uniform(-4, -1, shape)
    r = rng.standard_normal(shape)
    dJ, m = oracle.os_jacobi(L, eps, r, max_sweeps=5000, tol=1e-15)
    A = np.eye(chi.size) - _dense_from_band(L, shape) * (1 - eps.reshape(-1))[None, :]
    ref = np.linalg.solve(A, r.reshape(-1))
    assert np.max(np.abs(dJ.reshape(-1) - ref)) < 1e-12 * np.max(np.abs(ref))


def _os_band_system(seed, shape=(5, 4, 6), eps_range=(-4, -1)):
    rng = np.random.default_rng(seed)
    chi = 10 ** rng.uniform(-1, 1, shape)
    _, L = oracle.fs_cart(chi, np.ones(shape), 4, 6, False, lstar=True)
    eps = 10 ** rng.uniform(*eps_range, shape)
    r = rng.standard_normal(shape)
    A = np.eye(chi.size) - _dense_from_band(L, shape) * (1 - eps.reshape(-1))[None, :]
    return L, eps, r, np.linalg.solve(A, r.reshape(-1))


@pytest.mark.parametrize("colored", [False, True])
def test_os_gauss_seidel_solves_the_band_system(colored):
    L, eps, r, ref = _os_band_system(4)
    dJ, m = oracle.os_gauss_seidel(L, eps, r, max_sweeps=5000, tol=1e-15, colored=colored)
    assert 0 < m < 5000
    assert np.max(np.abs(dJ.reshape(-1) - ref)) < 1e-12 * np.max(np.abs(ref))


def test_os_gauss_seidel_takes_fewer_sweeps_than_jacobi():
    # For a diagonally dominant M-matrix-like system the Gauss-Seidel spectral
    # radius is below the Jacobi one (Stein-Rosenberg), so at the same stop
    # test it needs fewer sweeps; the eight-color order is a Gauss-Seidel
    # order too.
    L, eps, r, ref = _os_band_system(5)
    _, mj = oracle.os_jacobi(L, eps, r, max_sweeps=5000, tol=1e-10)
    _, mg = oracle.os_gauss_seidel(L, eps, r, max_sweeps=5000, tol=1e-10, colored=False)
    _, mc = oracle.os_gauss_seidel(L, eps, r, max_sweeps=5000, tol=1e-10, colored=True)
    assert mg < mj and mc < mj


def test_os_gauss_seidel_one_sweep_by_hand():
    # One lexicographic sweep on a tiny box, written out voxel by voxel from
    # the definition dJ_v = (r_v + sum_{u != v} L*[v][u](1-eps_u) dJ_u) / A_vv
    # with the voxels already visited taking their new values.
    rng = np.random.default_rng(6)
    shape = (3, 3, 3)
    chi = 10 ** rng.uniform(-1, 1, shape)
    _, L = oracle.fs_cart(chi, np.ones(shape), 2, 4, False, lstar=True)
    eps = 10 ** rng.uniform(-3, -1, shape)
    r = rng.standard_normal(shape)
    M = _dense_from_band(L, shape) * (1 - eps.reshape(-1))[None, :]
    n = M.shape[0]
    diag = 1 - np.diag(M)
    x = r.reshape(-1) / diag
    for v in range(n):
        x[v] = (r.reshape(-1)[v] + sum(M[v, u] * x[u] for u in range(n) if u != v)) / diag[v]
    dJ, m = oracle.os_gauss_seidel(L, eps, r, max_sweeps=1, tol=0.0, colored=False)
    assert m == 1
    assert np.max(np.abs(dJ.reshape(-1) - x)) < 1e-14 * np.max(np.abs(x))


def test_os_bicgstab_solves_the_band_system():
    L, eps, r, ref = _os_band_system(7, eps_range=(-6, -3))
    dJ, k = oracle.os_bicgstab(L, eps, r, max_iter=500, tol=1e-13)
    assert 0 < k < 500
    assert np.max(np.abs(dJ.reshape(-1) - ref)) < 1e-10 * np.max(np.abs(ref))


def test_os_bicgstab_exact_on_a_diagonal_system():
    # eps = 1 removes every coupling (A = I): the first step is exact and the
    # stabilising half-step has nothing left to do.
    L, _, r, _ = _os_band_system(8)
    eps = np.ones(r.shape)
    dJ, k = oracle.os_bicgstab(L, eps, r, max_iter=50, tol=1e-14)
    assert k == 1
    assert np.max(np.abs(dJ - r)) < 1e-14 * np.max(np.abs(r))


def _dense_from_band(L, shape):
    nz, ny, nx = shape
    N = L.shape[0]
    M = np.zeros((N, N))
    for v in range(N):
        x, y, z = v % nx, (v // nx) % ny, v // (nx * ny)
        for c in range(27):
            dx, dy, dz = c % 3 - 1, (c // 3) % 3 - 1, c // 9 - 1
            if not 0 <= z + dz < nz:
                continue
            u = (x + dx) % nx + nx * ((y + dy) % ny + ny * (z + dz))
            M[v, u] += L[v, c]
    return M


@pytest.mark.parametrize("parabolic", [False, True])
def test_ali_converges_to_the_direct_solution(parabolic):
    rng = np.random.default_rng(4)
    shape = (5, 4, 4)
    chi = 10 ** rng.uniform(-1, 1.3, shape)
    eps = 10 ** rng.uniform(-3, -1, shape)
    B = rng.uniform(0.5, 1.5, shape)
    bc = {"I_top": 0.0, "I_bottom": B[0]}
    J, it, hist, _ = oracle.ali_solve(chi, eps, B, 4, 6, parabolic, bc, tol=1e-14, max_iter=400)
    assert it > 0
    Jd = oracle.direct_solve(chi, eps, B, 4, 6, parabolic, bc)
    assert np.max(np.abs(J - Jd) / np.abs(Jd)) < 1e-12


def test_lambda_iteration_fixed_point():
    rng = np.random.default_rng(6)
    shape = (4, 3, 4)
    chi = 10 ** rng.uniform(-1, 0.5, shape)
    eps = np.full(shape, 0.5)
    B = rng.uniform(0.5, 1.5, shape)
    bc = {"I_top": 0.0, "I_bottom": B[0]}
    J = np.zeros(shape)
    for _ in range(200):  # Eq. alisol
        J = oracle.fs_cart(chi, (1 - eps) * J + eps * B, 4, 6, False, bc)
    Jd = oracle.direct_solve(chi, eps, B, 4, 6, False, bc)
    assert np.max(np.abs(J - Jd) / Jd) < 1e-12


def test_spectral_radius_of_lambda_iteration():
    """Power iteration on Lambda(1-eps) for a homogeneous slab of vertical
    optical thickness T. Sec. 2.2 quotes lambda_max ~ (1-eps)(1-1/T), an
    estimate that tends to 1 for large T. The fundamental slab mode of the
    continuum problem is sharper: cos(k tau) with k = pi / (T + 2 q) (q =
    0.7104, the Hopf extrapolation depth) and eigenvalue arctan(k)/k."""
    eps = 1e-3
    lams = []
    for T, nz in ((5.0, 10), (20.0, 20)):
        shape = (nz, 3, 3)
        chi = np.full(shape, T / nz)
        x = np.ones(shape)
        lam = 0.0
        for _ in range(300):
            y = (1 - eps) * oracle.fs_cart(chi, x, 8, 8, False)
            lam = np.linalg.norm(y) / np.linalg.norm(x)
            x = y / np.linalg.norm(y)
        k = math.pi / (T + 2 * 0.7104)
        assert abs(lam - (1 - eps) * math.atan(k) / k) < 0.01, (T, lam)
        assert (1 - eps) * (1 - 1 / T) < lam < 1 - eps
        lams.append(lam)
    assert lams[1] > lams[0]  # thicker slab: closer to unity


def test_P7_sqrt_eps_surface_law():
    """Homogeneous eps, B = 1: the surface source function of a thick
    scattering slab tends to sqrt(eps) B; the discretisation error shrinks as
    the layers refine."""
    errs = {}
    for eps in (1e-2, 1e-4):
        for nz in (33, 65):
            chi = np.broadcast_to(inputs.vertical_chi(nz)[:, None, None], (nz, 3, 3)).copy()
            e, B = np.full(chi.shape, eps), np.ones(chi.shape)
            J, it, _, _ = oracle.ali_solve(chi, e, B, 8, 16, False,
                                           {"I_top": 0.0, "I_bottom": 1.0}, tol=1e-9,
                                           max_iter=2000)
            assert it > 0
            S0 = (1 - eps) * J[-1, 0, 0] + eps
            errs[(eps, nz)] = abs(S0 / math.sqrt(eps) - 1)
    assert errs[(1e-2, 33)] < 0.05 and errs[(1e-2, 65)] < 0.02
    assert errs[(1e-4, 65)] < errs[(1e-4, 33)]
    assert errs[(1e-4, 65)] < 0.2


# ------------------------------------------- LTE diffusion inner boundary
def test_diffusion_entry_in_vacuum_closed_form():
    """chi = 0: every point keeps its characteristic's entry intensity. With
    I_top = 0 and uniform faces I_bottom = a, gradient g, the upward half of
    the midpoint directions (weight 1/2, sum of w mu = 1/4 exactly) gives
    J = a/2 + g/4 everywhere."""
    shape = (3, 5, 4)
    S = np.random.default_rng(2).uniform(0.5, 2.0, shape)
    a, g = 1.7, 0.9
    for parabolic in (False, True):
        J = oracle.fs_cart(np.zeros(shape), S, 8, 6, parabolic,
                           bc={"I_top": 0.0, "I_bottom": a, "I_bottom_grad": np.full((5, 4), g)})
        assert np.max(np.abs(J - (a / 2 + g / 4))) <= 1e-14


def test_diffusion_entry_per_column_by_brute_force():
    """chi = 0 with face arrays that differ per column: J_v is the chord
    weighted average over the characteristics crossing v of their entry
    values I_bottom(x0, y0) + mu g(x0, y0), rebuilt here from the traced
    characteristics (catches a transposed face index or a wrong mu)."""
    nz, ny, nx = 2, 3, 4
    rng = np.random.default_rng(5)
    face, grad = rng.uniform(0.5, 1.5, (ny, nx)), rng.uniform(-1.0, 1.0, (ny, nx))
    top = rng.uniform(0.0, 0.3, (ny, nx))
    nth, nph = 4, 4
    mu, phi, d, w = oracle.directions(nth, nph)
    Jref = np.zeros(nz * ny * nx)
    for o in range(nth * nph):
        num, den = np.zeros_like(Jref), np.zeros_like(Jref)
        for y0 in range(ny):
            for x0 in range(nx):
                vox, ln = oracle.trace_cart((nz, ny, nx), d[o], x0, y0)
                I0 = face[y0, x0] + mu[o] * grad[y0, x0] if mu[o] > 0 else top[y0, x0]
                np.add.at(num, vox, ln * I0)
                np.add.at(den, vox, ln)
        Jref += w[o] * num / den
    J = oracle.fs_cart(np.zeros((nz, ny, nx)), np.ones((nz, ny, nx)), nth, nph, False,
                       bc={"I_top": top, "I_bottom": face, "I_bottom_grad": grad})
    assert np.max(np.abs(J.reshape(-1) - Jref)) <= 1e-14


def test_diffusion_faces_of_a_linear_source():
    """B = a + b tau per column with tau the trapezoidal vertical optical depth
    of a random chi: the gradient is b, and the face value is B at the bottom
    face, whose optical depth from the top is the column's total sum of chi
    (unit voxels); nz = 1 gives no gradient."""
    rng = np.random.default_rng(8)
    chi = 10 ** rng.uniform(-1, 1, (6, 3, 5))
    a, b = rng.uniform(0.5, 2, (3, 5)), rng.uniform(0.1, 3, (3, 5))
    B = a + b * inputs.grey_tau(chi)
    I_face, grad = oracle.diffusion_bc(chi, B)
    assert np.max(np.abs(grad - b) / b) < 1e-12
    Bface = a + b * chi.sum(axis=0)
    assert np.max(np.abs(I_face - Bface) / Bface) < 1e-13
    I1, g1 = oracle.diffusion_bc(chi[:1], B[:1])
    assert np.all(g1 == 0.0) and np.array_equal(I1, B[0])


def test_diffusion_boundary_gives_j_equal_b_in_a_grey_lte_slab():
    """Grey LTE slab (S = B = 3/4 (tau + 2/3), 0.2 optical depth per voxel,
    bottom tau about 5): the diffusion intensity B + mu dB/dtau is the exact
    solution for a source linear in tau, so J = B near the inner boundary up
    to the discretisation, while the plain rule I = B leaves J short by about
    g/4 (the upward half carries no mu g)."""
    nz, ny, nx = 24, 4, 4
    chi = np.full((nz, ny, nx), 0.2)
    B = 0.75 * (inputs.grey_tau(chi) + 2.0 / 3.0)
    I_face, g = oracle.diffusion_bc(chi, B)
    assert np.allclose(g, 0.75, rtol=1e-13)
    for parabolic in (False, True):
        J_diff = oracle.fs_cart(chi, B, 8, 8, parabolic,
                                bc={"I_top": 0.0, "I_bottom": I_face, "I_bottom_grad": g})
        J_plain = oracle.fs_cart(chi, B, 8, 8, parabolic, bc={"I_top": 0.0, "I_bottom": B[0]})
        d_diff, d_plain = (J_diff[0] - B[0]).mean(), (J_plain[0] - B[0]).mean()
        assert abs(d_diff) < 0.01, d_diff
        assert abs(d_plain + 0.75 / 4) < 0.01, d_plain
