"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: traced voxel indices and chords bit-exact; J and Lambda* within 1e-12
relative in the FP64 mode and 2e-5 relative in the FP32 formal-solution mode;
converged J within 1e-8 of the oracle's converged J.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2102_01734_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5
HERE = os.path.dirname(os.path.abspath(__file__))


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


def dev_bc(bc):
    return {k: (dev(v) if isinstance(v, np.ndarray) else v) for k, v in bc.items()}


def relerr(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def lstar_err(Lg, Lo):
    """Lambda* (27,N) from the GPU vs (N,27) from the oracle, relative to the
    largest entry of each row."""
    Lg = Lg.T
    scale = np.max(np.abs(Lo), axis=1, keepdims=True)
    return float(np.max(np.abs(Lg - Lo) / scale))


# ------------------------------------------------------------------- tracer
@pytest.mark.parametrize("n,nth,nph", [((13, 11, 9), 6, 10), ((4, 4, 1), 2, 4),
                                       ((40, 37, 23), 8, 16)])
def test_template_bit_exact(rt3d, n, nth, nph):
    g = rt3d.Grid(n, nth, nph)
    mu, phi, d, w = oracle.directions(nth, nph)
    shape = (n[2], n[1], n[0])
    for o in range(nth * nph):
        vox, ln = g.template(o)
        ov, ol = oracle.trace_cart(shape, d[o], 0, 0)
        assert np.array_equal(vox, ov), o
        assert np.array_equal(ln.view(np.int64), ol.view(np.int64)), o
    info = g.info()
    assert info["nangles"] == nth * nph


def test_template_bit_exact_box129(rt3d):
    g = rt3d.Grid(129, 32, 64, rt3d.PARABOLIC, rt3d.FP32_FS_FP64_ALI)
    mu, phi, d, w = oracle.directions(32, 64)
    for o in range(0, 2048, 7):
        vox, ln = g.template(o)
        ov, ol = oracle.trace_cart((129, 129, 129), d[o], 0, 0)
        assert np.array_equal(vox, ov), o
        assert np.array_equal(ln.view(np.int64), ol.view(np.int64)), o
    assert g.info()["segments"] > 2.5e10


# ---------------------------------------------------------- formal solution
CASES = [
    # (n, ntheta, nphi, seed) -- ragged tails: nx*ny not a multiple of 128
    ((17, 13, 11), 4, 8, 1),
    ((9, 9, 4), 2, 5, 2),
    ((4, 5, 1), 2, 6, 3),
    ((33, 20, 7), 6, 6, 4),
]


def _case(n, seed):
    chi, eps, B, bc = inputs.cartesian_config(n, 1e-2, seed=seed)
    rng = np.random.default_rng(seed)
    S = rng.uniform(0.2, 2.0, chi.shape)
    bc = {"I_top": rng.uniform(0, 0.3, chi.shape[1:]), "I_bottom": bc["I_bottom"]}
    return chi, S, bc


@pytest.mark.parametrize("parabolic", [False, True])
@pytest.mark.parametrize("n,nth,nph,seed", CASES)
def test_fs_fp64_parity(rt3d, n, nth, nph, seed, parabolic):
    chi, S, bc = _case(n, seed)
    g = rt3d.Grid(n, nth, nph, int(parabolic), rt3d.FP64)
    J, L = g.formal_solution(dev(chi), dev(S), dev_bc(bc), lstar=True)
    Jo, Lo = oracle.fs_cart(chi, S, nth, nph, parabolic, bc, lstar=True)
    assert relerr(J.cpu().numpy(), Jo) < TOL64
    assert lstar_err(L.cpu().numpy(), Lo) < TOL64
    # the formal solution without Lambda* runs a separate kernel
    J2 = g.formal_solution(dev(chi), dev(S), dev_bc(bc))
    assert relerr(J2.cpu().numpy(), Jo) < TOL64


@pytest.mark.parametrize("parabolic", [False, True])
@pytest.mark.parametrize("n,nth,nph,seed", CASES)
def test_fs_fp32_parity(rt3d, n, nth, nph, seed, parabolic):
    chi, S, bc = _case(n, seed)
    g = rt3d.Grid(n, nth, nph, int(parabolic), rt3d.FP32_FS_FP64_ALI)
    J, L = g.formal_solution(dev(chi), dev(S), dev_bc(bc), lstar=True)
    Jo, Lo = oracle.fs_cart(chi, S, nth, nph, parabolic, bc, lstar=True)
    assert relerr(J.cpu().numpy(), Jo) < TOL32
    assert lstar_err(L.cpu().numpy(), Lo) < TOL32
    # the formal solution without Lambda* runs a separate kernel
    J2 = g.formal_solution(dev(chi), dev(S), dev_bc(bc))
    assert relerr(J2.cpu().numpy(), Jo) < TOL32


SHAPES = [(b, r, w, bl) for b in (64, 128, 256) for r in (1, 2, 4) for w in (0, 1, 2) for bl in (0, 1)]


@pytest.mark.parametrize("n,nth,nph,seed", [((17, 13, 11), 12, 16, 5), ((4, 5, 3), 2, 6, 6),
                                          ((37, 14, 9), 8, 16, 7)])
def test_fs_fast_every_shape(rt3d, n, nth, nph, seed):
    """The FP32 formal solution without Lambda* in every ray-bundle shape,
    widening and branch form (ragged bundles; odd and even point counts
    through the two-point loop), and the autotuner's choice."""
    chi, S, bc = _case(n, seed)
    for parabolic in (False, True):
        Jo = oracle.fs_cart(chi, S, nth, nph, parabolic, bc)
        g = rt3d.Grid(n, nth, nph, int(parabolic), rt3d.FP32_FS_FP64_ALI)
        for shape in SHAPES:
            g.set_fs_shape(shape)
            for _ in range(2):  # the fold leaves the accumulators zeroed
                J = g.formal_solution(dev(chi), dev(S), dev_bc(bc))
                assert relerr(J.cpu().numpy(), Jo) < TOL32, (parabolic, shape)
        g.set_fs_shape(None)
        J = g.formal_solution(dev(chi), dev(S), dev_bc(bc))
        assert relerr(J.cpu().numpy(), Jo) < TOL32
        info = g.info()
        assert info["fs_shape"] in [rt3d.fs_tune_shape(i) for i in range(rt3d.FS_TUNE_SHAPES)]
        assert all(t > 0 for t in info["fs_tune_ms"])
    with pytest.raises(rt3d.RT3DError):
        g.set_fs_shape((96, 1, 0, 0))
    with pytest.raises(rt3d.RT3DError):
        g.set_fs_shape((128, 1, 3, 0))


# Float-float formal solution: per-step coefficient errors measured on a CPU
# emulation of its arithmetic against mpmath are <= 2e-12 relative for d (the
# closed form just above u = 1/2), 2e-13 for a and 6e-14 for e0; J, a weighted
# mean of intensities built from them, is held to 1e-11.
TOLFF = 1e-11


@pytest.mark.parametrize("parabolic", [False, True])
@pytest.mark.parametrize("n,nth,nph,seed", CASES)
def test_fs_ff_parity(rt3d, n, nth, nph, seed, parabolic):
    """Float-float formal solution against the FP64 oracle (grids of both
    mixed precisions)."""
    chi, S, bc = _case(n, seed)
    Jo = oracle.fs_cart(chi, S, nth, nph, parabolic, bc)
    for prec in (rt3d.FP32_FS_FP64_ALI, rt3d.FP32_FS_FF_REFINE):
        g = rt3d.Grid(n, nth, nph, int(parabolic), prec)
        for _ in range(2):
            J = g.formal_solution_ff(dev(chi), dev(S), dev_bc(bc))
            assert relerr(J.cpu().numpy(), Jo) < TOLFF, (prec, relerr(J.cpu().numpy(), Jo))


def test_fs_ff_extremes(rt3d):
    """dtau from 1e-7 to 3e3 and zero (series branch, Tang exp branch, e^-u
    below FP32 range), S and chi over many decades."""
    rng = np.random.default_rng(11)
    n = (16, 12, 10)
    shape = (10, 12, 16)
    chi = 10 ** rng.uniform(-7, 3.5, shape)
    chi[2:4, 3:6, 4:9] = 0.0
    S = 10 ** rng.uniform(-3, 3, shape)
    bc = {"I_top": 0.5, "I_bottom": 1.5}
    for parabolic in (False, True):
        Jo = oracle.fs_cart(chi, S, 4, 8, parabolic, bc)
        g = rt3d.Grid(n, 4, 8, int(parabolic), rt3d.FP32_FS_FF_REFINE)
        J = g.formal_solution_ff(dev(chi), dev(S), bc)
        assert relerr(J.cpu().numpy(), Jo) < TOLFF, (parabolic, relerr(J.cpu().numpy(), Jo))


def test_fs_ff_box129_sampled(rt3d):
    """Full-size box (129^3, 32 x 64 angles, parabolic): sampled voxels of the
    float-float formal solution against the oracle's per-voxel route."""
    cfg = inputs.CONFIGS["box129_field"]
    chi, eps, B, bc = inputs.cartesian_config(129, cfg["eps"], seed=cfg["seed"])
    S = B.copy()
    g = rt3d.Grid(129, 32, 64, rt3d.PARABOLIC, rt3d.FP32_FS_FF_REFINE)
    J = g.formal_solution_ff(dev(chi), dev(S), dev_bc(bc)).cpu().numpy().reshape(-1)
    rng = np.random.default_rng(1)
    vs = [0, 129 * 129 * 100 + 7, chi.size - 1] + list(rng.integers(0, chi.size, 2))
    for v in vs:
        Jv = oracle.fs_cart_voxel(chi, S, 32, 64, int(v), True, bc)
        assert abs(J[v] - Jv) / abs(Jv) < TOLFF, (v, abs(J[v] - Jv) / abs(Jv))


def test_fs_thick_thin_extremes(rt3d):
    """Per-voxel dtau from 1e-7 to 3e3 and zero (both series and closed-form
    branches, vacuum and opaque voxels next to each other), every FP32
    ray-bundle shape."""
    rng = np.random.default_rng(9)
    n = (16, 12, 10)
    shape = (10, 12, 16)
    chi = 10 ** rng.uniform(-7, 3.5, shape)
    chi[2:4, 3:6, 4:9] = 0.0  # a vacuum patch: zero-length optical intervals
    S = rng.uniform(0.1, 3.0, shape)
    bc = {"I_top": 0.5, "I_bottom": 1.5}
    for parabolic in (False, True):
        Jo = oracle.fs_cart(chi, S, 4, 8, parabolic, bc)
        for prec, tol in ((rt3d.FP64, TOL64), (rt3d.FP32_FS_FP64_ALI, TOL32)):
            g = rt3d.Grid(n, 4, 8, int(parabolic), prec)
            J = g.formal_solution(dev(chi), dev(S), bc)
            assert relerr(J.cpu().numpy(), Jo) < tol, (parabolic, prec)
            if prec == rt3d.FP32_FS_FP64_ALI:
                for shape in SHAPES:
                    g.set_fs_shape(shape)
                    J = g.formal_solution(dev(chi), dev(S), bc)
                    assert relerr(J.cpu().numpy(), Jo) < tol, (parabolic, shape)


def test_fs_host_pointers_match_device(rt3d):
    chi, S, bc = _case((17, 13, 11), 1)
    g = rt3d.Grid((17, 13, 11), 4, 8, rt3d.PARABOLIC, rt3d.FP64)
    Jd = g.formal_solution(dev(chi), dev(S), dev_bc(bc)).cpu().numpy()
    Jh = g.formal_solution(chi, S, bc)
    assert isinstance(Jh, np.ndarray)
    assert np.max(np.abs(Jh - Jd) / Jd) < 1e-14


def test_fs_box129_sampled(rt3d):
    """Full-size box (129^3, 32 x 64 angles, parabolic, k^-3 lognormal field),
    FP32 formal solution as timed by the benchmark; sampled voxels against
    the oracle's per-voxel route."""
    cfg = inputs.CONFIGS["box129_field"]
    chi, eps, B, bc = inputs.cartesian_config(129, cfg["eps"], seed=cfg["seed"])
    S = B.copy()
    g = rt3d.Grid(129, 32, 64, rt3d.PARABOLIC, rt3d.FP32_FS_FP64_ALI)
    J = g.formal_solution(dev(chi), dev(S), dev_bc(bc)).cpu().numpy().reshape(-1)
    rng = np.random.default_rng(0)
    vs = [0, 129 * 129 * 64 + 65 * 129 + 3, chi.size - 1] + list(rng.integers(0, chi.size, 2))
    for v in vs:
        Jv = oracle.fs_cart_voxel(chi, S, 32, 64, int(v), True, bc)
        assert abs(J[v] - Jv) / abs(Jv) < TOL32, v


# ----------------------------------------------------------------- OS solve
def test_os_solve_parity(rt3d):
    rng = np.random.default_rng(2)
    n = (11, 9, 7)
    shape = (7, 9, 11)
    chi = 10 ** rng.uniform(-1, 1.5, shape)
    _, Lo = oracle.fs_cart(chi, np.ones(shape), 4, 6, False, lstar=True)
    eps = 10 ** rng.uniform(-4, -1, shape)
    r = rng.standard_normal(shape)
    dJo, mo = oracle.os_jacobi(Lo, eps, r, max_sweeps=50, tol=1e-6)
    g = rt3d.Grid(n, 4, 6, rt3d.LINEAR, rt3d.FP64)
    dJ, m = g.os_solve(dev(np.ascontiguousarray(Lo.T)), dev(eps), dev(r), max_sweeps=50, tol=1e-6)
    assert m == mo
    assert np.max(np.abs(dJ.cpu().numpy() - dJo)) < 1e-12 * np.max(np.abs(dJo))


def test_os_solve_mixed_fixed_sweeps(rt3d):
    """Mixed mode: FP32 coefficients times the FP32 copy of the sweep, FP64
    state; a fixed number of sweeps against the oracle's FP64 Jacobi (ragged
    voxel count: 693 is not a multiple of the 32-voxel coefficient block)."""
    rng = np.random.default_rng(3)
    n = (11, 9, 7)
    shape = (7, 9, 11)
    chi = 10 ** rng.uniform(-1, 1.5, shape)
    _, Lo = oracle.fs_cart(chi, np.ones(shape), 4, 6, False, lstar=True)
    eps = 10 ** rng.uniform(-4, -1, shape)
    r = rng.standard_normal(shape)
    dJo, mo = oracle.os_jacobi(Lo, eps, r, max_sweeps=12, tol=0.0)
    g = rt3d.Grid(n, 4, 6, rt3d.LINEAR, rt3d.FP32_FS_FP64_ALI)
    dJ, m = g.os_solve(dev(np.ascontiguousarray(Lo.T)), dev(eps), dev(r), max_sweeps=12, tol=0.0)
    assert m == mo == 12
    assert np.max(np.abs(dJ.cpu().numpy() - dJo)) < 2e-6 * np.max(np.abs(dJo))


def test_ali_step_parity(rt3d):
    chi, eps, B, bc = inputs.cartesian_config((13, 11, 9), 1e-3, seed=7)
    J0 = np.full(chi.shape, 0.5)
    # oracle: one iteration of Eq. alo
    S = (1 - eps) * J0 + eps * B
    Jfs, Lo = oracle.fs_cart(chi, S, 4, 8, True, bc, lstar=True)
    dJo, _ = oracle.os_jacobi(Lo, eps, Jfs - J0, 50, 1e-3)
    Jo = J0 + dJo
    g = rt3d.Grid((13, 11, 9), 4, 8, rt3d.PARABOLIC, rt3d.FP64)
    J = dev(J0)
    rel = g.ali_step(dev(chi), dev(eps), dev(B), dev_bc(bc), J)
    assert relerr(J.cpu().numpy(), Jo) < 1e-11
    assert abs(rel - np.max(np.abs(dJo) / np.abs(Jo))) < 1e-9 * rel


# ---------------------------------------------------------- converged solve
def _golden33():
    vals = [float(l) for l in open(os.path.join(HERE, "golden", "box33_fp64_J.txt"))
            if not l.startswith("#")]
    return np.array(vals)


@pytest.mark.parametrize("accel", ["ali", "krylov"])
@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_ff"])
def test_solve_box33_matches_golden(rt3d, precision, accel):
    chi, eps, B, bc = inputs.cartesian_config(33, 1e-2)
    prec = {"fp64": rt3d.FP64, "mixed": rt3d.FP32_FS_FP64_ALI,
            "mixed_ff": rt3d.FP32_FS_FF_REFINE}[precision]
    acc = rt3d.ACCEL_NONE if accel == "ali" else rt3d.ACCEL_KRYLOV
    g = rt3d.Grid(33, 8, 16, rt3d.LINEAR, prec, accel=acc)
    J = torch.zeros(chi.shape, dtype=torch.float64, device="cuda")
    st = g.solve(dev(chi), dev(eps), dev(B), dev_bc(bc), J, tol=1e-9, max_iter=3000)
    ref = _golden33()[:, None, None]
    err = np.max(np.abs(J.cpu().numpy() - ref) / ref)
    assert err < 1e-8, (err, st)
    assert st["residual64"] < 1e-8
    assert st["jacobi_sweeps"] > 0


@pytest.mark.parametrize("accel", ["ali", "krylov"])
@pytest.mark.parametrize("parabolic", [False, True])
def test_solve_field_matches_oracle(rt3d, parabolic, accel):
    n = (14, 12, 11)
    chi, eps, B, bc = inputs.cartesian_config(n, 1e-4, seed=3)
    Jo, it, _, _ = oracle.ali_solve(chi, eps, B, 4, 8, parabolic, bc, tol=1e-13, max_iter=3000)
    assert it > 0
    acc = rt3d.ACCEL_NONE if accel == "ali" else rt3d.ACCEL_KRYLOV
    for prec in (rt3d.FP64, rt3d.FP32_FS_FP64_ALI, rt3d.FP32_FS_FF_REFINE):
        g = rt3d.Grid(n, 4, 8, int(parabolic), prec, accel=acc)
        J = torch.zeros(chi.shape, dtype=torch.float64, device="cuda")
        st = g.solve(dev(chi), dev(eps), dev(B), dev_bc(bc), J, tol=1e-9, max_iter=3000)
        err = relerr(J.cpu().numpy(), Jo)
        assert err < 1e-8, (prec, err, st)


@pytest.mark.parametrize("accel", ["ali", "krylov"])
def test_solve_bench_regime_matches_direct_solve(rt3d, accel):
    """Converged J in the regime of the 129^3 workload (eps = 1e-6, parabolic,
    opacity profile times a lognormal k^-3 field, B = 1 + 0.2 g) on a box the
    oracle's dense direct solve handles: every precision within 1e-8."""
    n = (7, 7, 9)
    chi, eps, B, bc = inputs.cartesian_config(n, 1e-6, seed=5)
    Jo = oracle.direct_solve(chi, eps, B, 4, 8, True, bc)
    acc = rt3d.ACCEL_NONE if accel == "ali" else rt3d.ACCEL_KRYLOV
    for prec in (rt3d.FP64, rt3d.FP32_FS_FP64_ALI, rt3d.FP32_FS_FF_REFINE):
        g = rt3d.Grid(n, 4, 8, rt3d.PARABOLIC, prec, accel=acc)
        J = torch.from_numpy(B.copy()).to("cuda")
        st = g.solve(dev(chi), dev(eps), dev(B), dev_bc(bc), J, tol=1e-9, max_iter=20000)
        err = relerr(J.cpu().numpy(), Jo)
        assert err < 1e-8, (prec, accel, err, st["iterations"])


# ----------------------------------------------------------- error paths
def test_iteration_cap_is_enotconverged(rt3d):
    chi, eps, B, bc = inputs.cartesian_config(8, 1e-4)
    g = rt3d.Grid(8, 2, 4, rt3d.LINEAR, rt3d.FP64)
    J = torch.zeros(chi.shape, dtype=torch.float64, device="cuda")
    st = g.solve(dev(chi), dev(eps), dev(B), dev_bc(bc), J, tol=1e-12, max_iter=2,
                 raise_on_nonconv=False)
    assert st["status"] == rt3d.ENOTCONVERGED
    assert st["iterations"] == 2
    assert torch.isfinite(J).all()


def test_nan_input_is_enumeric(rt3d):
    chi, eps, B, bc = inputs.cartesian_config(8, 1e-2)
    B = B.copy()
    B[3, 2, 1] = np.nan
    g = rt3d.Grid(8, 2, 4, rt3d.LINEAR, rt3d.FP64)
    J = torch.zeros(chi.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(rt3d.RT3DError) as ei:
        g.solve(dev(chi), dev(eps), dev(B), dev_bc(bc), J, tol=1e-8, max_iter=20)
    assert ei.value.status == rt3d.ENUMERIC
