"""The LTE diffusion inner boundary of the paper's test cases (Sec. 3.1, 3.2)
on the GPU against the FP64 CPU oracle: the face arrays built by the library
(bit-exact), the formal solution entering upward characteristics (on the
spherical grid, those leaving the core) with I = I_bottom + mu dB/dtau in
every kernel (1e-12 relative in FP64, 2e-5 in FP32), and converged solves of
the grey atmosphere (1e-8), single and batched, Cartesian and spherical."""
import numpy as np
import pytest

import oracle
from paper_2102_01734_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


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


def relerr(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def _grey(n, seed, scale=1.0):
    """Grey atmosphere of n = (nx, ny, nz) with the lognormal field; chi scaled
    so that the innermost voxels have optical depths near 1 (the diffusion
    gradient then reaches the interior)."""
    chi, eps, B, bc = inputs.grey_config(n, 1e-2, seed=seed)
    chi = chi * scale
    B = 0.75 * (inputs.grey_tau(chi) + 2.0 / 3.0)
    return chi, eps, B


def _bc(chi, B):
    I_face, grad = oracle.diffusion_bc(chi, B)
    return {"I_top": 0.0, "I_bottom": I_face, "I_bottom_grad": grad}


def _dev_bc(bc):
    return {k: (dev(v) if isinstance(v, np.ndarray) else v) for k, v in bc.items()}


@pytest.mark.parametrize("n,nl", [((11, 9, 7), 1), ((12, 10, 5), 3), ((5, 4, 1), 2)])
def test_face_arrays_bit_exact(rt3d, n, nl):
    """rt3d_diffusion_bc against the oracle on stacked grids (one layer:
    gradient 0)."""
    rng = np.random.default_rng(3)
    shape = (nl, n[2], n[1], n[0])
    chi = 10 ** rng.uniform(-2, 2, shape)
    B = rng.uniform(0.5, 3.0, shape)
    g = rt3d.Grid(n, 2, 4)
    I_face, grad = g.diffusion_bc(dev(chi), dev(B))
    torch.cuda.synchronize()
    for l in range(nl):
        If_o, g_o = oracle.diffusion_bc(chi[l], B[l])
        assert np.array_equal(I_face[l].cpu().numpy(), If_o)
        assert np.array_equal(grad[l].cpu().numpy(), g_o)


@pytest.mark.parametrize("n,nth,nph,seed", [((11, 9, 7), 4, 8, 1), ((17, 13, 11), 6, 10, 2)])
def test_formal_solution_with_diffusion_boundary(rt3d, n, nth, nph, seed):
    """FP64 formal solution (with Lambda*) and the FP32 one in every ray-bundle
    shape (one, two and four characteristics per thread: each reads the
    gradient face for its own rows), and float-float, with the diffusion
    boundary, against the oracle."""
    chi, eps, B = _grey(n, seed, scale=1e-2)
    bc = _bc(chi, B)
    S = B * rng_factor(chi.shape, seed)
    for parabolic in (False, True):
        Jo, Lo = oracle.fs_cart(chi, S, nth, nph, parabolic, bc, lstar=True)
        # the gradient term is visible: without it J differs well above the bar
        Jp = oracle.fs_cart(chi, S, nth, nph, parabolic, {"I_top": 0.0, "I_bottom": bc["I_bottom"]})
        assert relerr(Jp, Jo) > 1e3 * TOL32
        g = rt3d.Grid(n, nth, nph, int(parabolic), rt3d.FP64)
        J, L = g.formal_solution(dev(chi), dev(S), _dev_bc(bc), lstar=True)
        assert relerr(J.cpu().numpy(), Jo) < TOL64
        J = g.formal_solution(dev(chi), dev(S), _dev_bc(bc))
        assert relerr(J.cpu().numpy(), Jo) < TOL64
        g = rt3d.Grid(n, nth, nph, int(parabolic), rt3d.FP32_FS_FP64_ALI)
        J, L = g.formal_solution(dev(chi), dev(S), _dev_bc(bc), lstar=True)
        assert relerr(J.cpu().numpy(), Jo) < TOL32
        for shape in [(128, 1, 0, 0), (256, 1, 1, 1), (128, 2, 1, 1), (256, 4, 1, 1),
                      (128, 4, 0, 1)]:
            g.set_fs_shape(shape)
            J = g.formal_solution(dev(chi), dev(S), _dev_bc(bc))
            assert relerr(J.cpu().numpy(), Jo) < TOL32, (parabolic, shape)
        J = g.formal_solution_ff(dev(chi), dev(S), _dev_bc(bc))
        assert relerr(J.cpu().numpy(), Jo) < 1e-11
        # host face arrays are staged the same way
        J = g.formal_solution(dev(chi), dev(S), bc)
        assert relerr(J.cpu().numpy(), Jo) < TOL32


def rng_factor(shape, seed):
    return np.random.default_rng(100 + seed).uniform(0.8, 1.2, shape)


@pytest.mark.parametrize("accel", ["ali", "krylov"])
def test_grey_atmosphere_converges_to_the_oracle(rt3d, accel):
    """Converged J of the grey scattering atmosphere with the diffusion inner
    boundary (face arrays from the library), every precision, against the
    oracle's dense direct solve with the same boundary."""
    n = (9, 8, 10)
    chi, eps, B = _grey(n, 4, scale=1e-2)
    bc = _bc(chi, B)
    Jo = oracle.direct_solve(chi, eps, B, 4, 8, True, bc)
    acc = rt3d.ACCEL_NONE if accel == "ali" else rt3d.ACCEL_KRYLOV
    for prec in (rt3d.FP64, rt3d.FP32_FS_FP64_ALI, rt3d.FP32_FS_FF_REFINE):
        g = rt3d.Grid(n, 4, 8, rt3d.PARABOLIC, prec, accel=acc)
        I_face, grad = g.diffusion_bc(dev(chi), dev(B))
        J = dev(B).clone()
        st = g.solve(dev(chi), dev(eps), dev(B),
                     {"I_top": 0.0, "I_bottom": I_face, "I_bottom_grad": grad}, J,
                     tol=1e-9, max_iter=20000)
        err = relerr(J.cpu().numpy(), Jo)
        assert err < 1e-8, (prec, err, st["iterations"])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batched_grey_wavelengths(rt3d, precision):
    """Wavelengths with their own opacity scale, hence their own diffusion
    gradient: per-wavelength face arrays from one library call on the stacked
    grids, every wavelength against the oracle's direct solve."""
    n = (12, 10, 9)
    chi, eps, B = _grey(n, 2, scale=1e-2)
    scales = np.array([0.3, 1.0, 4.0])
    eps_l = np.array([1e-2, 1e-4, 1e-1])
    nl = len(scales)
    chis = np.stack([s * chi for s in scales])
    Bs = np.stack([B] * nl)
    epss = np.stack([np.full(chi.shape, e) for e in eps_l])
    prec = rt3d.FP64 if precision == "fp64" else rt3d.FP32_FS_FP64_ALI
    g = rt3d.Grid(n, 4, 8, rt3d.PARABOLIC, prec)
    I_face, grad = g.diffusion_bc(dev(chis), dev(Bs))
    J = dev(Bs).clone()
    st = g.solve_batched(dev(chis), dev(epss), dev(Bs),
                         {"I_top": 0.0, "I_bottom": I_face, "I_bottom_grad": grad}, J,
                         tol=1e-9, max_iter=3000)
    assert st["converged"] == nl
    Jg = J.cpu().numpy()
    for l in range(nl):
        Jo = oracle.direct_solve(chis[l], epss[l], Bs[l], 4, 8, True, _bc(chis[l], Bs[l]))
        assert relerr(Jg[l], Jo) < 1e-8, l


# ---- the spherical grid: the diffusion condition on the core sphere

def _sph_atmosphere(n, seed, scale=1.0):
    """Grey shell: chi ~ r^-12 with a mild random factor, B = 3/4 (tau + 2/3)
    of the radial optical depth (np, nt, nr)."""
    nr, nt, np_ = n
    re = 1.3 ** (np.arange(nr + 1) / nr)
    rc = np.sqrt(re[:-1] * re[1:])
    rng = np.random.default_rng(seed)
    chi = np.broadcast_to(scale * 12 * rc ** -12.0, (np_, nt, nr)).copy()
    chi *= np.exp(0.2 * rng.standard_normal(chi.shape))
    tau = scale * (rc ** -11.0 - 1.3 ** -11.0)
    B = np.broadcast_to(0.75 * (tau + 2.0 / 3.0), (np_, nt, nr)).copy()
    B *= rng.uniform(0.95, 1.05, B.shape)
    return chi, B


@pytest.mark.parametrize("n,nl", [((9, 7, 12), 1), ((6, 5, 8), 2), ((1, 4, 6), 1)])
def test_sph_face_arrays_bit_exact(rt3d, n, nl):
    """rt3d_diffusion_bc on a spherical grid: the core faces against the
    oracle, bit for bit (one shell: gradient 0)."""
    chi, B = _sph_atmosphere(n, 3)
    chis = np.stack([chi * (1.0 + 0.5 * l) for l in range(nl)])
    Bs = np.stack([B] * nl)
    g = rt3d.Grid(n, 2, 4, geometry=rt3d.SPHERICAL)
    I_face, grad = g.diffusion_bc(dev(chis if nl > 1 else chis[0]), dev(Bs if nl > 1 else Bs[0]))
    torch.cuda.synchronize()
    I_face, grad = I_face.cpu().numpy().reshape(nl, n[2], n[1]), grad.cpu().numpy().reshape(nl, n[2], n[1])
    for l in range(nl):
        If_o, g_o = oracle.diffusion_bc_sph(chis[l], Bs[l])
        assert np.array_equal(I_face[l], If_o)
        assert np.array_equal(grad[l], g_o)


@pytest.mark.parametrize("parabolic", [False, True])
def test_sph_formal_solution_with_diffusion_boundary(rt3d, parabolic):
    """Every spherical kernel (FP64 and FP32, with and without Lambda*) with
    the core's diffusion condition, on the device cache and on two host
    residencies (chunked launches: the per-ray entry intensities are read
    through the chunk's rays), against the oracle."""
    n = (9, 7, 12)
    nth, nph = 3, 6
    chi, B = _sph_atmosphere(n, 1, scale=0.3)
    S = B * np.random.default_rng(7).uniform(0.8, 1.2, B.shape)
    I_face, grad = oracle.diffusion_bc_sph(chi, B)
    Jo, Lo = oracle.fs_sph(chi, S, B, nth, nph, parabolic, I_out=0.0, I_irr=10.0, lstar=True,
                           core_face=I_face, core_grad=grad)
    Jp = oracle.fs_sph(chi, S, B, nth, nph, parabolic, I_out=0.0, I_irr=10.0,
                       core_face=I_face)
    assert relerr(Jp, Jo) > 1e3 * TOL32  # the gradient term is visible
    bc = {"I_top": 0.0, "I_irr": 10.0, "I_bottom": dev(I_face), "I_bottom_grad": dev(grad)}
    seg = None
    for cache in (rt3d.CACHE_DEVICE, rt3d.CACHE_HOST_STREAMED, rt3d.CACHE_HOST_CHORDS):
        for prec, tol in ((rt3d.FP64, TOL64), (rt3d.FP32_FS_FP64_ALI, TOL32)):
            sb = 0
            if cache != rt3d.CACHE_DEVICE:
                sb = (24 if cache == rt3d.CACHE_HOST_STREAMED else 8) * seg // 5
            g = rt3d.Grid(n, nth, nph, int(parabolic), prec, geometry=rt3d.SPHERICAL,
                          cache=cache, stream_bytes=sb)
            seg = g.info()["segments"]
            J, L = g.formal_solution(dev(chi), dev(S), bc, lstar=True)
            assert relerr(J.cpu().numpy(), Jo) < tol, (cache, prec)
            Lg = L.cpu().numpy().T
            lerr = np.max(np.abs(Lg - Lo) / np.max(np.abs(Lo), axis=1, keepdims=True))
            assert lerr < tol, (cache, prec, lerr)
            J = g.formal_solution(dev(chi), dev(S), bc)
            assert relerr(J.cpu().numpy(), Jo) < tol, (cache, prec)
            # host face arrays are staged the same way
            hbc = {"I_top": 0.0, "I_irr": 10.0, "I_bottom": I_face, "I_bottom_grad": grad}
            J = g.formal_solution(dev(chi), dev(S), hbc)
            assert relerr(J.cpu().numpy(), Jo) < tol, (cache, prec)
            J = g.formal_solution_ff(dev(chi), dev(S), bc)
            assert relerr(J.cpu().numpy(), Jo) < 1e-11, (cache, prec)
            g.close()


def test_sph_grey_solve_matches_direct_solution(rt3d):
    """Converged J of a grey scattering shell with the core's diffusion
    condition (faces from the library), FP64 and mixed precision, plain ALI
    and Krylov, against the dense solve of (1 - Lambda(1-eps)) J =
    Lambda(eps B) + J_bc built column by column from the oracle."""
    n = (6, 5, 8)
    nth, nph = 2, 6
    chi, B = _sph_atmosphere(n, 3, scale=0.3)
    eps = np.full(chi.shape, 1e-2)
    I_face, grad = oracle.diffusion_bc_sph(chi, B)
    N = chi.size
    zero = np.zeros(chi.shape)
    M = np.zeros((N, N))
    e = np.zeros(chi.shape)
    for u in range(N):
        e.reshape(-1)[:] = 0.0
        e.reshape(-1)[u] = 1.0
        M[:, u] = oracle.fs_sph(chi, e, zero, nth, nph, True, 0.0, 0.0,
                                core_face=np.zeros_like(I_face)).reshape(-1)
    Jbc = oracle.fs_sph(chi, zero, B, nth, nph, True, 0.0, 10.0, core_face=I_face,
                        core_grad=grad).reshape(-1)
    ef = eps.reshape(-1)
    Jd = np.linalg.solve(np.eye(N) - M * (1 - ef)[None, :],
                         M @ (ef * B.reshape(-1)) + Jbc).reshape(chi.shape)
    for prec in (rt3d.FP64, rt3d.FP32_FS_FP64_ALI):
        for accel in (rt3d.ACCEL_NONE, rt3d.ACCEL_KRYLOV):
            g = rt3d.Grid(n, nth, nph, rt3d.PARABOLIC, prec, accel=accel,
                          geometry=rt3d.SPHERICAL)
            If_d, g_d = g.diffusion_bc(dev(chi), dev(B))
            J = dev(B).clone()
            g.solve(dev(chi), dev(eps), dev(B), {"I_top": 0.0, "I_bottom": If_d,
                                                 "I_bottom_grad": g_d, "I_irr": 10.0},
                    J, tol=1e-10, max_iter=4000)
            err = relerr(J.cpu().numpy(), Jd)
            assert err < 1e-8, (prec, accel, err)
