"""Spherical grid (paper Sec. 3.2 geometry): the CUDA geometry cache, formal
solution, Lambda* and converged solve against the FP64 CPU oracle."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N3 = (9, 7, 12)  # (nr, ntheta, nphi)


@pytest.fixture(scope="module")
def rt3d():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_01734_gb300 import build, rt3d as mod
    build.build()
    mod.load()
    return mod


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def radii(n):
    nr = n[0]
    re = 1.3 ** (np.arange(nr + 1) / nr)
    return np.sqrt(re[:-1] * re[1:])


def atmosphere(n, seed, tau_core=20.0):
    """chi = C r^-12 (times a mild random factor), shape (nphi, ntheta, nr)."""
    nr, nt, np_ = n
    rng = np.random.default_rng(seed)
    rc = radii(n)
    chi = np.broadcast_to(tau_core * 12 * rc ** -12.0, (np_, nt, nr)).copy()
    chi *= np.exp(0.3 * rng.standard_normal(chi.shape))
    B = 1.0 + 0.2 * rng.uniform(-1, 1, chi.shape)
    return chi, B


def test_sph_cache_bit_exact(rt3d):
    g = rt3d.Grid(N3, 2, 4, geometry=rt3d.SPHERICAL)
    mu, phi, d, w = oracle.directions(2, 4)
    for o in range(8):
        launch = oracle.sph_rays(N3, 2, 4, o)
        for i, v in enumerate(launch):
            r = g.sph_ray(o, i)
            assert r is not None, (o, i)
            vox, ln, lv, kind = r
            assert lv == v
            ovox, oln, core, pin = oracle.sph_trace(N3, d[o], int(v))
            assert np.array_equal(vox, ovox), (o, i)
            assert np.array_equal(ln.view(np.int64), oln.view(np.int64)), (o, i)
            okind = 2 if core else (1 if (pin[0] > 0 and d[o, 0] < 0) else 0)
            assert kind == okind
        assert g.sph_ray(o, len(launch)) is None
    info = g.info()
    assert info["segments"] > 0


@pytest.mark.parametrize("parabolic", [False, True])
def test_sph_fs_parity(rt3d, parabolic):
    chi, B = atmosphere(N3, 1)
    rng = np.random.default_rng(2)
    S = rng.uniform(0.5, 1.5, chi.shape)
    bc = {"I_top": 0.3, "I_bottom": B[:, :, 0].copy(), "I_irr": 10.0}
    Jo, Lo = oracle.fs_sph(chi, S, B, 3, 6, parabolic, I_out=0.3, I_irr=10.0, lstar=True)
    for prec, tol in ((rt3d.FP64, 1e-12), (rt3d.FP32_FS_FP64_ALI, 2e-5)):
        g = rt3d.Grid(N3, 3, 6, int(parabolic), prec, geometry=rt3d.SPHERICAL)
        dbc = {"I_top": 0.3, "I_bottom": dev(bc["I_bottom"]), "I_irr": 10.0}
        J, L = g.formal_solution(dev(chi), dev(S), dbc, lstar=True)
        err = np.max(np.abs(J.cpu().numpy() - Jo) / np.abs(Jo))
        assert err < tol, (prec, err)
        Lg = L.cpu().numpy().T
        lerr = np.max(np.abs(Lg - Lo) / np.max(np.abs(Lo), axis=1, keepdims=True))
        assert lerr < tol, (prec, lerr)
        # without Lambda* (FP32: the record kernel over rays sorted by length)
        for _ in range(2):
            J2 = g.formal_solution(dev(chi), dev(S), dbc)
            err = np.max(np.abs(J2.cpu().numpy() - Jo) / np.abs(Jo))
            assert err < tol, (prec, err)
        # float-float (any precision of grid)
        for _ in range(2):
            Jf = g.formal_solution_ff(dev(chi), dev(S), dbc)
            err = np.max(np.abs(Jf.cpu().numpy() - Jo) / np.abs(Jo))
            assert err < 1e-11, (prec, err)


def test_sph_solve_matches_direct_solution(rt3d):
    """Converged J against the dense solve of (1 - Lambda(1-eps)) J =
    Lambda(eps B) + J_bc, Lambda built column by column from the oracle."""
    n = (6, 5, 8)
    nr, nt, np_ = n
    chi, B = atmosphere(n, 3, tau_core=8.0)
    eps = np.full(chi.shape, 1e-2)
    core = B[:, :, 0].copy()
    N = chi.size
    nth, nph = 2, 6
    M = np.zeros((N, N))
    e = np.zeros(chi.shape)
    for u in range(N):
        e.reshape(-1)[:] = 0.0
        e.reshape(-1)[u] = 1.0
        M[:, u] = oracle.fs_sph(chi, e, np.zeros(chi.shape), nth, nph, True, 0.0, 0.0).reshape(-1)
    Jbc = oracle.fs_sph(chi, np.zeros(chi.shape), B, nth, nph, True, 0.0, 10.0).reshape(-1)
    ef = eps.reshape(-1)
    rhs = M @ (ef * B.reshape(-1)) + Jbc
    Jd = np.linalg.solve(np.eye(N) - M * (1 - ef)[None, :], rhs).reshape(chi.shape)
    for prec in (rt3d.FP64, rt3d.FP32_FS_FP64_ALI, rt3d.FP32_FS_FF_REFINE):
        for accel in (rt3d.ACCEL_NONE, rt3d.ACCEL_KRYLOV):
            g = rt3d.Grid(n, nth, nph, rt3d.PARABOLIC, prec, accel=accel,
                          geometry=rt3d.SPHERICAL)
            J = dev(B).clone()
            g.solve(dev(chi), dev(eps), dev(B), {"I_top": 0.0, "I_bottom": dev(core),
                                                 "I_irr": 10.0}, J, tol=1e-10, max_iter=4000)
            err = np.max(np.abs(J.cpu().numpy() - Jd) / np.abs(Jd))
            assert err < 1e-8, (prec, accel, err)
