"""The OS step's other solvers on the GPU (Sec. 4: the OS iteration by Jacobi,
Gauss-Seidel or BiCGStab) against the FP64 CPU oracle: the eight-colour
Gauss-Seidel sweep (same sweep count, iterates within 1e-12), BiCGStab (the
oracle's iteration count within one, the solution of the band system), and
the converged solve with each solver as the ALI's OS step and as the Krylov
preconditioner."""
import numpy as np
import pytest

import oracle
from paper_2102_01734_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt3d():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_01734_gb300 import build, rt3d as mod
    build.build()
    mod.load()
    return mod


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _band_problem(n, seed, parabolic):
    nx, ny, nz = n
    shape = (nz, ny, nx)
    rng = np.random.default_rng(seed)
    chi = 10 ** rng.uniform(-1, 1.5, shape)
    _, L = oracle.fs_cart(chi, np.ones(shape), 4, 6, parabolic, lstar=True)
    eps = 10 ** rng.uniform(-4, -1, shape)
    r = rng.standard_normal(shape)
    return L, eps, r


# odd nx and ny: same-colour neighbours across the periodic seam
CASES = [((11, 9, 7), 1, False), ((12, 10, 5), 2, True), ((5, 4, 3), 3, False), ((9, 7, 4), 4, True)]


@pytest.mark.parametrize("n,seed,parabolic", CASES)
def test_gauss_seidel_matches_oracle(rt3d, n, seed, parabolic):
    L, eps, r = _band_problem(n, seed, parabolic)
    g = rt3d.Grid(n, 4, 6, int(parabolic), rt3d.FP64)
    g.set_os_solver(rt3d.OS_GAUSS_SEIDEL)
    for max_sweeps, tol in ((7, 0.0), (50, 1e-6), (256, 1e-12)):
        dJo, mo = oracle.os_gauss_seidel(L, eps, r, max_sweeps=max_sweeps, tol=tol, colored=True)
        dJ, m = g.os_solve(dev(L.T), dev(eps), dev(r), max_sweeps=max_sweeps, tol=tol)
        assert m == mo, (max_sweeps, tol, m, mo)
        err = np.max(np.abs(dJ.cpu().numpy() - dJo)) / np.max(np.abs(dJo))
        assert err < 1e-12, (max_sweeps, tol, err)


@pytest.mark.parametrize("n,seed,parabolic", CASES)
def test_gauss_seidel_needs_fewer_sweeps_than_jacobi(rt3d, n, seed, parabolic):
    L, eps, r = _band_problem(n, seed, parabolic)
    g = rt3d.Grid(n, 4, 6, int(parabolic), rt3d.FP64)
    _, mj = g.os_solve(dev(L.T), dev(eps), dev(r), max_sweeps=256, tol=1e-10)
    g.set_os_solver(rt3d.OS_GAUSS_SEIDEL)
    _, mg = g.os_solve(dev(L.T), dev(eps), dev(r), max_sweeps=256, tol=1e-10)
    assert mg < mj, (mg, mj)


@pytest.mark.parametrize("n,seed,parabolic", CASES)
def test_bicgstab_matches_oracle(rt3d, n, seed, parabolic):
    L, eps, r = _band_problem(n, seed, parabolic)
    # the solution of the band system: the oracle's Jacobi iterated to rounding
    exact, _ = oracle.os_jacobi(L, eps, r, max_sweeps=20000, tol=1e-15)
    dJo, ko = oracle.os_bicgstab(L, eps, r, max_iter=200, tol=1e-10)
    assert ko > 0
    g = rt3d.Grid(n, 4, 6, int(parabolic), rt3d.FP64)
    g.set_os_solver(rt3d.OS_BICGSTAB)
    dJ, k = g.os_solve(dev(L.T), dev(eps), dev(r), max_sweeps=200, tol=1e-10)
    # the dot products are summed in another order than the oracle's, so the
    # iterates differ by rounding: the count may differ by one
    assert abs(k - ko) <= 1, (k, ko)
    a = dJ.cpu().numpy()
    scale = np.max(np.abs(exact))
    assert np.max(np.abs(a - exact)) < 1e-8 * scale
    assert np.max(np.abs(a - dJo)) < 1e-8 * scale


def test_solver_switch_keeps_the_band(rt3d):
    """A switch to Gauss-Seidel re-lays the coefficients of the band the grid
    holds: a Jacobi ALI step, the switch, and a second step give the J of a
    fresh Gauss-Seidel grid stepping once from the first step's J (same band,
    built again from the same chi and eps)."""
    n = (12, 10, 8)
    chi, eps, B, bc = inputs.cartesian_config(n, 1e-2, seed=9)
    bcd = {"I_top": 0.0, "I_bottom": dev(bc["I_bottom"])}
    g = rt3d.Grid(n, 4, 8, rt3d.PARABOLIC, rt3d.FP64)
    J = dev(B).clone()
    g.ali_step(dev(chi), dev(eps), dev(B), bcd, J)  # Jacobi; builds Lambda*
    J1 = J.clone()
    g.set_os_solver(rt3d.OS_GAUSS_SEIDEL)
    g.ali_step(dev(chi), dev(eps), dev(B), bcd, J)  # the band the grid holds
    h = rt3d.Grid(n, 4, 8, rt3d.PARABOLIC, rt3d.FP64)
    h.set_os_solver(rt3d.OS_GAUSS_SEIDEL)
    Jh = J1.clone()
    h.ali_step(dev(chi), dev(eps), dev(B), bcd, Jh)
    a, b = J.cpu().numpy(), Jh.cpu().numpy()
    assert np.max(np.abs(a - b) / np.abs(b)) < 1e-12


@pytest.mark.parametrize("solver", ["gs", "bicgstab"])
@pytest.mark.parametrize("accel", ["ali", "krylov"])
def test_solve_with_each_os_solver(rt3d, solver, accel):
    """Converged J with the solver as the ALI's OS step (ali) or as the
    FGMRES preconditioner (krylov), every precision, against the oracle's
    dense direct solve (eps = 1e-4, parabolic, field)."""
    n = (9, 8, 10)
    chi, eps, B, bc = inputs.cartesian_config(n, 1e-4, seed=4)
    Jo = oracle.direct_solve(chi, eps, B, 4, 8, True, bc)
    kind = rt3d.OS_GAUSS_SEIDEL if solver == "gs" else rt3d.OS_BICGSTAB
    acc = rt3d.ACCEL_NONE if accel == "ali" else rt3d.ACCEL_KRYLOV
    for prec in (rt3d.FP64, rt3d.FP32_FS_FP64_ALI, rt3d.FP32_FS_FF_REFINE):
        g = rt3d.Grid(n, 4, 8, rt3d.PARABOLIC, prec, accel=acc)
        g.set_os_solver(kind)
        J = dev(B).clone()
        st = g.solve(dev(chi), dev(eps), dev(B), {"I_top": 0.0, "I_bottom": dev(bc["I_bottom"])},
                     J, tol=1e-9, max_iter=20000)
        err = np.max(np.abs(J.cpu().numpy() - Jo) / np.abs(Jo))
        assert err < 1e-8, (prec, err, st["iterations"])
        assert st["jacobi_sweeps"] > 0
