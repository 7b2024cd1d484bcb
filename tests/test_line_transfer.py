"""Line transfer: the profile-averaged mean intensity of Sec. 2.

The wavelengths of a line share S = (1 - eps) Jbar + eps B with
Jbar = sum_l wphi[l] J_l; wavelength l sees the opacity scale[l] * chi.

CPU tests pin the oracle (against the continuum ALI it must reduce to and
against the dense solve of the line problem); GPU tests compare the C ABI's
line solve with the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2102_01734_gb300 import inputs


def _box(n, eps, seed):
    chi, epsa, B, bc = inputs.cartesian_config(n, eps, seed=seed)
    return chi, epsa, B, bc


def test_line_profile_quadrature():
    scale, wphi = inputs.line_profile(9, xmax=3.0, strength=2.0)
    assert abs(wphi.sum() - 1.0) < 1e-15
    assert np.allclose(wphi, wphi[::-1]) and np.allclose(scale, scale[::-1])
    assert scale[4] == 2.0 and np.argmax(wphi) == 4
    assert abs(scale[0] / 2.0 - np.exp(-9.0)) < 1e-18


def test_line_single_wavelength_is_the_continuum_ali():
    chi, eps, B, bc = _box((5, 4, 6), 1e-2, 2)
    Jc, itc, _, _ = oracle.ali_solve(chi, eps, B, 2, 4, True, bc, tol=1e-12, max_iter=2000)
    Jl, itl = oracle.line_ali_solve(chi, [1.0], [1.0], eps, B, 2, 4, True, bc, tol=1e-12,
                                    max_iter=2000)
    assert itc > 0 and itl == itc
    assert np.max(np.abs(Jl - Jc) / np.abs(Jc)) < 1e-13


def test_line_equal_opacities_reduce_to_the_continuum():
    # all wavelengths see the same opacity: Jbar is the continuum J whatever
    # the weights
    chi, eps, B, bc = _box((5, 4, 6), 1e-2, 3)
    Jc = oracle.direct_solve(chi, eps, B, 2, 4, False, bc)
    Jl = oracle.line_direct_solve(chi, [1.0, 1.0, 1.0], [0.2, 0.5, 0.3], eps, B, 2, 4, False,
                                  bc)
    assert np.max(np.abs(Jl - Jc) / np.abs(Jc)) < 1e-12


def test_line_duplicate_wavelengths_merge():
    chi, eps, B, bc = _box((5, 4, 6), 1e-2, 4)
    S = (1 - eps) * B + eps * B
    a = oracle.line_fs(chi, [1.0, 0.1, 0.1], [0.5, 0.2, 0.3], S, 2, 4, True, bc)
    b = oracle.line_fs(chi, [1.0, 0.1], [0.5, 0.5], S, 2, 4, True, bc)
    assert np.max(np.abs(a - b) / np.abs(b)) < 1e-14


@pytest.mark.parametrize("parabolic", [False, True])
def test_line_ali_converges_to_the_dense_solve(parabolic):
    chi, eps, B, bc = _box((5, 4, 6), 1e-2, 5)
    scale, wphi = inputs.line_profile(5, xmax=2.5, strength=3.0)
    Jx = oracle.line_direct_solve(chi, scale, wphi, eps, B, 2, 4, parabolic, bc)
    Jl, it = oracle.line_ali_solve(chi, scale, wphi, eps, B, 2, 4, parabolic, bc, tol=1e-13,
                                   max_iter=3000)
    assert it > 0
    assert np.max(np.abs(Jl - Jx) / np.abs(Jx)) < 1e-10
    # the wings (optically thin) leave Jbar far from the continuum solution
    Jc = oracle.direct_solve(chi * 3.0, eps, B, 2, 4, parabolic, bc)
    assert np.max(np.abs(Jl - Jc) / np.abs(Jc)) > 1e-3


def test_line_lambda_star_is_the_band_of_the_averaged_lambda():
    chi, _, _, _ = _box((9, 9, 4), 1e-2, 6)
    scale, wphi = inputs.line_profile(3, xmax=2.0)
    Lb = oracle.line_lambda_star(chi, scale, wphi, 2, 4, False)
    M = sum(w * oracle.lambda_matrix(chi * s, 2, 4, False) for s, w in zip(scale, wphi))
    nz, ny, nx = chi.shape
    for v in range(0, chi.size, 7):
        z, rem = divmod(v, nx * ny)
        y, x = divmod(rem, nx)
        for d in range(27):
            dz, dy, dx = d // 9 - 1, (d // 3) % 3 - 1, d % 3 - 1
            zz = z + dz
            if not 0 <= zz < nz:
                assert Lb[v, d] == 0.0
                continue
            u = zz * nx * ny + ((y + dy) % ny) * nx + (x + dx) % nx
            assert abs(Lb[v, d] - M[v, u]) < 1e-12 * np.max(np.abs(M[v]))


# ------------------------------------------------------------ GPU parity
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_01734_gb300 import build, rt3d
    build.build()
    rt3d.load()
    return torch, rt3d


def _dev(torch, x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _dev_bc(torch, bc):
    return {k: (_dev(torch, v) if isinstance(v, np.ndarray) else v) for k, v in bc.items()}


def _relerr(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.mark.gpu
def test_gpu_line_step_parity():
    torch, rt3d = _gpu()
    n = (13, 11, 9)
    chi, eps, B, bc = _box(n, 1e-3, 7)
    scale, wphi = inputs.line_profile(5, xmax=2.5, strength=3.0)
    J0 = np.full(chi.shape, 0.5)
    Jo, relo, _ = oracle.line_ali_step(chi, scale, wphi, eps, B, J0, 4, 8, True, bc)
    g = rt3d.Grid(n, 4, 8, rt3d.PARABOLIC, rt3d.FP64)
    J = _dev(torch, J0)
    st = g.line_solve(_dev(torch, chi), scale, wphi, _dev(torch, eps), _dev(torch, B),
                      _dev_bc(torch, bc), J, tol=1e-9, max_iter=1, raise_on_nonconv=False)
    assert st["status"] == rt3d.ENOTCONVERGED
    assert st["iterations"] == 1 and st["fs_lambda"] == 5 and st["jacobi_sweeps"] > 0
    assert _relerr(J.cpu().numpy(), Jo) < 1e-11
    assert abs(st["rel_change"] - relo) < 1e-9 * relo


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gpu_line_solve_matches_oracle(precision):
    torch, rt3d = _gpu()
    n = (13, 11, 9)
    chi, eps, B, bc = _box(n, 1e-2, 8)
    scale, wphi = inputs.line_profile(5, xmax=2.5, strength=3.0)
    Jo, it = oracle.line_ali_solve(chi, scale, wphi, eps, B, 4, 8, True, bc, tol=1e-13,
                                   max_iter=3000)
    assert it > 0
    prec = rt3d.FP64 if precision == "fp64" else rt3d.FP32_FS_FP64_ALI
    g = rt3d.Grid(n, 4, 8, rt3d.PARABOLIC, prec)
    J = torch.zeros(chi.shape, dtype=torch.float64, device="cuda")
    st = g.line_solve(_dev(torch, chi), scale, wphi, _dev(torch, eps), _dev(torch, B),
                      _dev_bc(torch, bc), J, tol=1e-9, max_iter=3000)
    assert _relerr(J.cpu().numpy(), Jo) < 1e-8, st
    assert 0 <= st["est_error"] <= 1e-9
    if precision == "mixed":
        # FP32 formal solutions, then FP64 residuals (one per wavelength each),
        # the last certifying the result
        n64 = st["fs_lambda"] - st["fs_lambda32"]
        assert 0 < st["fs_lambda32"] and n64 >= 2 * 5 and n64 % 5 == 0, st
        assert 0 < st["residual64"] < 1e-7, st
    else:
        assert st["fs_lambda"] == 5 * st["iterations"]
        assert st["fs_lambda32"] == 0


@pytest.mark.gpu
def test_gpu_line_with_equal_opacities_is_the_continuum_solve():
    torch, rt3d = _gpu()
    n = (12, 10, 8)
    chi, eps, B, bc = _box(n, 1e-2, 9)
    Jo, it, _, _ = oracle.ali_solve(chi, eps, B, 4, 8, False, bc, tol=1e-13, max_iter=3000)
    assert it > 0
    g = rt3d.Grid(n, 4, 8, rt3d.LINEAR, rt3d.FP64)
    J = torch.zeros(chi.shape, dtype=torch.float64, device="cuda")
    g.line_solve(_dev(torch, chi), [1.0, 1.0, 1.0], [0.2, 0.5, 0.3], _dev(torch, eps),
                 _dev(torch, B), _dev_bc(torch, bc), J, tol=1e-9, max_iter=3000)
    assert _relerr(J.cpu().numpy(), Jo) < 1e-8
    # the grid's continuum solve afterwards rebuilds its own Lambda*
    J2 = torch.zeros(chi.shape, dtype=torch.float64, device="cuda")
    g.solve(_dev(torch, chi), _dev(torch, eps), _dev(torch, B), _dev_bc(torch, bc), J2,
            tol=1e-9, max_iter=3000)
    assert _relerr(J2.cpu().numpy(), Jo) < 1e-8


@pytest.mark.gpu
@pytest.mark.parametrize("scale,wphi", [([1.0, 0.0], [0.5, 0.5]), ([1.0, -1.0], [0.5, 0.5]),
                                        ([1.0, 1.0], [0.5, -0.1]), ([1.0, 1.0], [0.0, 0.0]),
                                        ([1.0, float("nan")], [0.5, 0.5])])
def test_gpu_line_bad_profile_is_einval(scale, wphi):
    torch, rt3d = _gpu()
    n = (6, 6, 4)
    chi, eps, B, bc = _box(n, 1e-2, 1)
    g = rt3d.Grid(n, 2, 4, rt3d.LINEAR, rt3d.FP64)
    J = torch.zeros(chi.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(rt3d.RT3DError) as ei:
        g.line_solve(_dev(torch, chi), scale, wphi, _dev(torch, eps), _dev(torch, B), None, J,
                     tol=1e-8, max_iter=10)
    assert ei.value.status == rt3d.EINVAL
