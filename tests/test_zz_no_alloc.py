"""The allocation-free OS solve (rt3d_os_solve_noalloc) against the grid
entry point rt3d_os_solve and the FP64 CPU oracle's Jacobi solve.

The allocation-free variant exists for callers that cannot allocate device
memory (for example an application that pre-reserves all device memory in its
own pool, or a time-critical loop that must not call cudaMalloc/cudaFree).
Its scratch lives in a fixed device array shared by all calls, so two calls in
a row must each give the grid entry point's answer: nothing may leak from the
first call into the second.
"""
import numpy as np
import pytest

import oracle

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


def _problem(n, seed):
    nx, ny, nz = n
    shape = (nz, ny, nx)
    rng = np.random.default_rng(seed)
    chi = 10 ** rng.uniform(-1, 1.5, shape)
    _, L = oracle.fs_cart(chi, np.ones(shape), 4, 6, seed % 2 == 0, lstar=True)
    eps = 10 ** rng.uniform(-4, -1, shape)
    r = rng.standard_normal(shape)
    return L, eps, r


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def test_noalloc_matches_grid_os_solve_and_oracle_twice(rt3d):
    # second problem larger than the first, first one repeated last: stale
    # scratch from an earlier call would show up as a mismatch
    for n, seed in (((11, 9, 7), 1), ((24, 20, 16), 2), ((11, 9, 7), 3)):
        L, eps, r = _problem(n, seed)
        Ld = _dev(L.T)  # the library's layout: [27][N]
        g = rt3d.Grid(n, 4, 6, rt3d.LINEAR, rt3d.FP64)
        ref, m_ref = g.os_solve(Ld, _dev(eps), _dev(r), max_sweeps=50, tol=1e-6)
        g.close()
        dJo, mo = oracle.os_jacobi(L, eps, r, max_sweeps=50, tol=1e-6)
        out = torch.full(r.shape, np.nan, dtype=torch.float64, device="cuda")
        m = rt3d.os_solve_noalloc(n, Ld, _dev(eps), _dev(r), out, max_sweeps=50, tol=1e-6)
        torch.cuda.synchronize()
        assert m == m_ref == mo
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b)), n
        assert np.max(np.abs(a - dJo)) <= 1e-12 * np.max(np.abs(dJo)), n


def test_noalloc_at_its_limits(rt3d):
    """N = RT3D_NOALLOC_MAX_VOXELS voxels and max_sweeps = 256 (tol 0: every
    sweep runs), against the FP64 oracle, on two calls in a row. The band is
    synthetic: positive entries whose sum stays below 1 (a convergent Jacobi
    iteration), which the solve accepts like a traced Lambda*."""
    n = (64, 64, 16)
    N = n[0] * n[1] * n[2]
    assert N == 65536
    rng = np.random.default_rng(11)
    for seed in (1, 2):
        L = rng.uniform(0.0, 0.9 / 27, (N, 27))
        eps = 10 ** rng.uniform(-6, -1, (n[2], n[1], n[0]))
        r = rng.standard_normal((n[2], n[1], n[0]))
        dJo, mo = oracle.os_jacobi(L, eps, r, max_sweeps=256, tol=0.0)
        out = torch.full(r.shape, np.nan, dtype=torch.float64, device="cuda")
        m = rt3d.os_solve_noalloc(n, _dev(L.T), _dev(eps), _dev(r), out, max_sweeps=256, tol=0.0)
        torch.cuda.synchronize()
        assert m == mo == 256
        a = out.cpu().numpy()
        assert np.max(np.abs(a - dJo)) <= 1e-12 * np.max(np.abs(dJo)), seed


def test_noalloc_rejects_oversize_and_host_arrays(rt3d):
    n = (64, 64, 17)  # 69632 voxels > 65536
    x = torch.zeros(n[0] * n[1] * n[2], dtype=torch.float64, device="cuda")
    L = torch.zeros(27 * x.numel(), dtype=torch.float64, device="cuda")
    with pytest.raises(rt3d.RT3DError) as ei:
        rt3d.os_solve_noalloc(n, L, x, x, x)
    assert ei.value.status == rt3d.EINVAL and "limit" in rt3d.last_error()
    h = np.zeros(8 * 8 * 4)
    with pytest.raises(rt3d.RT3DError) as ei:
        rt3d.os_solve_noalloc((8, 8, 4), np.zeros(27 * h.size), h, h, h)
    assert ei.value.status == rt3d.EINVAL
