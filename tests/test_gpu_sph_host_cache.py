"""Host-resident spherical geometry cache (the SmallGPU mode of Sec. 4.3: the
tracking cache kept in host memory and moved to the GPU solid angle by solid
angle), streamed through two device buffers, read in place, or split by
precision (FP32 records on the device, FP64 chords streamed): the records
against the device-resident cache (bit-exact) and the oracle's tracer, the
formal solutions (with and without Lambda*, FP64 and FP32) against the
oracle, and converged solves against the dense direct solution."""
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


def atmosphere(n, seed, tau_core=20.0):
    """chi = C r^-12 (times a mild random factor), shape (nphi, ntheta, nr)."""
    nr, nt, np_ = n
    rng = np.random.default_rng(seed)
    re = 1.3 ** (np.arange(nr + 1) / nr)
    rc = np.sqrt(re[:-1] * re[1:])
    chi = np.broadcast_to(tau_core * 12 * rc ** -12.0, (np_, nt, nr)).copy()
    chi *= np.exp(0.3 * rng.standard_normal(chi.shape))
    B = 1.0 + 0.2 * rng.uniform(-1, 1, chi.shape)
    return chi, B


def modes(rt3d):
    """(name, mode, bytes per segment held on the host and streamed)."""
    return [("streamed", rt3d.CACHE_HOST_STREAMED, 24), ("mapped", rt3d.CACHE_HOST_MAPPED, 24),
            ("chords", rt3d.CACHE_HOST_CHORDS, 8)]


def segments(rt3d, n, nth, nph):
    g = rt3d.Grid(n, nth, nph, geometry=rt3d.SPHERICAL)
    seg = g.info()["segments"]
    g.close()
    return seg


@pytest.mark.parametrize("parts", [1, 5, 10 ** 9])
def test_host_records_equal_the_device_cache(rt3d, parts):
    """Every ray of every angle: cells, FP64 chords, launch voxel and kind
    bit-exact against the device cache (one chunk; about five; one angle per
    chunk when the chunk budget is below one angle), and against the oracle's
    tracer for the first angles."""
    nth, nph = 2, 6
    seg = segments(rt3d, N3, nth, nph)
    gd = rt3d.Grid(N3, nth, nph, geometry=rt3d.SPHERICAL)
    mu, phi, d, w = oracle.directions(nth, nph)
    for name, mode, per in modes(rt3d):
        sb = max(per * seg // parts, 1)
        g = rt3d.Grid(N3, nth, nph, geometry=rt3d.SPHERICAL, cache=mode, stream_bytes=sb)
        info = g.info()
        assert info["cache"] == mode and info["segments"] == seg
        assert info["host_bytes"] == per * seg
        want = {1: 1, 10 ** 9: nth * nph}.get(parts)
        if want is not None:
            assert info["cache_chunks"] == want, (name, info["cache_chunks"])
        else:
            assert 3 <= info["cache_chunks"] <= 8, (name, info["cache_chunks"])
        for o in range(nth * nph):
            i = 0
            while True:
                r, rd = g.sph_ray(o, i), gd.sph_ray(o, i)
                if rd is None:
                    assert r is None
                    break
                vox, ln, lv, kind = r
                vd, lnd, lvd, kd = rd
                assert np.array_equal(vox, vd) and (lv, kind) == (lvd, kd), (name, o, i)
                assert np.array_equal(ln.view(np.int64), lnd.view(np.int64)), (name, o, i)
                if o < 2:
                    ovox, oln, core, pin = oracle.sph_trace(N3, d[o], int(lv))
                    assert np.array_equal(vox, ovox) and np.array_equal(ln, oln)
                i += 1
        g.close()
    # the device mode holds no host memory and one chunk
    info = gd.info()
    assert info["host_bytes"] == 0 and info["cache_chunks"] == 1


@pytest.mark.parametrize("parabolic", [False, True])
def test_host_cache_formal_solutions(rt3d, parabolic):
    """FP64 (with and without Lambda*) and FP32 (with Lambda*; without it the
    record kernel) formal solutions on the host cache, cut into about seven
    chunks: J and Lambda* against the oracle (1e-12 / 2e-5), and J against the
    device cache's (the same per-ray arithmetic; only the order of the FP64
    reductions differs)."""
    nth, nph = 3, 6
    chi, B = atmosphere(N3, 1)
    rng = np.random.default_rng(2)
    S = rng.uniform(0.5, 1.5, chi.shape)
    core = B[:, :, 0].copy()
    Jo, Lo = oracle.fs_sph(chi, S, B, nth, nph, parabolic, I_out=0.3, I_irr=10.0, lstar=True)
    seg = segments(rt3d, N3, nth, nph)
    for prec, tol in ((rt3d.FP64, 1e-12), (rt3d.FP32_FS_FP64_ALI, 2e-5)):
        dbc = {"I_top": 0.3, "I_bottom": dev(core), "I_irr": 10.0}
        gd = rt3d.Grid(N3, nth, nph, int(parabolic), prec, geometry=rt3d.SPHERICAL)
        Jd, Ld = gd.formal_solution(dev(chi), dev(S), dbc, lstar=True)
        Jd2 = gd.formal_solution(dev(chi), dev(S), dbc)
        Jd, Ld, Jd2 = Jd.cpu().numpy(), Ld.cpu().numpy(), Jd2.cpu().numpy()
        for name, mode, per in modes(rt3d):
            g = rt3d.Grid(N3, nth, nph, int(parabolic), prec, geometry=rt3d.SPHERICAL,
                          cache=mode, stream_bytes=per * seg // 7)
            assert g.info()["cache_chunks"] >= 4
            J, L = g.formal_solution(dev(chi), dev(S), dbc, lstar=True)
            J, L = J.cpu().numpy(), L.cpu().numpy()
            err = np.max(np.abs(J - Jo) / np.abs(Jo))
            assert err < tol, (name, prec, err)
            lerr = np.max(np.abs(L.T - Lo) / np.max(np.abs(Lo), axis=1, keepdims=True))
            assert lerr < tol, (name, prec, lerr)
            assert np.max(np.abs(J - Jd) / np.abs(Jd)) < 1e-12, (name, prec)
            assert np.max(np.abs(L - Ld)) <= 1e-12 * np.max(np.abs(Ld)), (name, prec)
            for _ in range(3):  # the slots are reused across formal solutions
                J2 = g.formal_solution(dev(chi), dev(S), dbc).cpu().numpy()
                assert np.max(np.abs(J2 - Jo) / np.abs(Jo)) < tol, (name, prec)
                assert np.max(np.abs(J2 - Jd2) / np.abs(Jd2)) < 1e-12, (name, prec)
            # float-float: streams or reads the FP64 chords like the FP64 kernel
            Jf = g.formal_solution_ff(dev(chi), dev(S), dbc).cpu().numpy()
            assert np.max(np.abs(Jf - Jo) / np.abs(Jo)) < 1e-11, (name, prec)
            g.close()


def test_host_cache_solve_matches_direct_solution(rt3d):
    """Converged J of every host mode, FP64 and mixed precision, plain ALI and
    Krylov, against the dense solve of (1 - Lambda(1-eps)) J = Lambda(eps B)
    + J_bc built column by column from the oracle."""
    n = (6, 5, 8)
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
    seg = segments(rt3d, n, nth, nph)
    for name, mode, per in modes(rt3d):
        for prec in (rt3d.FP64, rt3d.FP32_FS_FP64_ALI, rt3d.FP32_FS_FF_REFINE):
            for accel in (rt3d.ACCEL_NONE, rt3d.ACCEL_KRYLOV):
                g = rt3d.Grid(n, nth, nph, rt3d.PARABOLIC, prec, accel=accel,
                              geometry=rt3d.SPHERICAL, cache=mode, stream_bytes=per * seg // 4)
                J = dev(B).clone()
                g.solve(dev(chi), dev(eps), dev(B), {"I_top": 0.0, "I_bottom": dev(core),
                                                     "I_irr": 10.0}, J, tol=1e-10, max_iter=4000)
                err = np.max(np.abs(J.cpu().numpy() - Jd) / np.abs(Jd))
                assert err < 1e-8, (name, prec, accel, err)
                g.close()
