"""Parity at the largest extents a grid accepts along one axis: nx = 2047
(the widest box: 11-bit x offsets in the cached step code) and nz = 1023 (the
tallest: 10-bit layer index), against the FP64 CPU oracle. Bars as in
test_gpu_parity.py: templates bit-exact, J and Lambda* within 1e-12 (FP64)
and 2e-5 (FP32 formal solution)."""
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


def lstar_err(Lg, Lo):
    scale = np.max(np.abs(Lo), axis=1, keepdims=True)
    return float(np.max(np.abs(Lg.T - Lo) / scale))


def _case(n, seed):
    chi, _, B, bc = inputs.cartesian_config(n, 1e-2, seed=seed)
    rng = np.random.default_rng(seed)
    S = rng.uniform(0.2, 2.0, chi.shape)
    return chi, S, {"I_top": 0.1, "I_bottom": bc["I_bottom"]}


@pytest.mark.parametrize("n,fp32", [((2047, 4, 2), True), ((4, 4, 1023), False)])
def test_widest_and_tallest_boxes(rt3d, n, fp32):
    nth, nph = 2, 4
    chi, S, bc = _case(n, 21)
    shape = chi.shape
    tbc = {"I_top": bc["I_top"], "I_bottom": dev(bc["I_bottom"])}
    Jo, Lo = oracle.fs_cart(chi, S, nth, nph, True, bc, lstar=True)
    mu, phi, d, w = oracle.directions(nth, nph)
    g = rt3d.Grid(n, nth, nph, rt3d.PARABOLIC, rt3d.FP64)
    for o in range(nth * nph):
        vox, ln = g.template(o)
        ov, ol = oracle.trace_cart(shape, d[o], 0, 0)
        assert np.array_equal(vox, ov), o
        assert np.array_equal(ln.view(np.int64), ol.view(np.int64)), o
    J, L = g.formal_solution(dev(chi), dev(S), tbc, lstar=True)
    assert relerr(J.cpu().numpy(), Jo) < TOL64
    assert lstar_err(L.cpu().numpy(), Lo) < TOL64
    J2 = g.formal_solution(dev(chi), dev(S), tbc)
    assert relerr(J2.cpu().numpy(), Jo) < TOL64
    if fp32:
        g32 = rt3d.Grid(n, nth, nph, rt3d.PARABOLIC, rt3d.FP32_FS_FP64_ALI)
        J3, L3 = g32.formal_solution(dev(chi), dev(S), tbc, lstar=True)
        assert relerr(J3.cpu().numpy(), Jo) < TOL32
        assert lstar_err(L3.cpu().numpy(), Lo) < TOL32
        J4 = g32.formal_solution(dev(chi), dev(S), tbc)
        assert relerr(J4.cpu().numpy(), Jo) < TOL32
