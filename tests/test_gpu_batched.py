"""Batched wavelengths (one geometry, many independent problems) against
the FP64 CPU oracle's converged solution of every wavelength."""
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


def _batch(n, nl, seed):
    """nl wavelengths drawn as the batched workload draws them (eps log-uniform
    in [1e-8, 1e-1], opacity scale 10^U(-3, 3)), the last two replaced by the
    corners of that range: eps = 1e-8 with scales 1e-3 and 1e3."""
    chi, _, B, bc = inputs.cartesian_config(n, 1e-2, seed=seed)
    eps_l, scale_l = inputs.batched_wavelengths(nl, seed=3)
    eps_l, scale_l = np.array(eps_l, dtype=float), np.array(scale_l, dtype=float)
    eps_l[-2:] = 1e-8
    scale_l[-2:] = (1e-3, 1e3)
    chis = np.stack([s * chi for s in scale_l])
    epss = np.stack([np.full(chi.shape, e) for e in eps_l])
    Bs = np.stack([B] * nl)
    bots = np.stack([B[0]] * nl)
    return chis, epss, Bs, bots


@pytest.mark.parametrize("precision", ["mixed", "mixed_ff", "fp64"])
def test_batched_matches_oracle_per_wavelength(rt3d, precision):
    n = (12, 10, 9)
    nl = 5
    chis, epss, Bs, bots = _batch(n, nl, 2)
    prec = {"fp64": rt3d.FP64, "mixed": rt3d.FP32_FS_FP64_ALI,
            "mixed_ff": rt3d.FP32_FS_FF_REFINE}[precision]
    g = rt3d.Grid(n, 4, 8, rt3d.PARABOLIC, prec)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
    J = d(Bs).clone()
    st = g.solve_batched(d(chis), d(epss), d(Bs), {"I_top": 0.0, "I_bottom": d(bots)}, J,
                         tol=1e-9, max_iter=3000)
    assert st["converged"] == nl
    assert np.all(st["per_lambda"] == 0)
    Jg = J.cpu().numpy()
    for l in range(nl):
        # reference: dense direct solve of (1 - Lambda(1-eps)) J = Lambda(eps B) + J_bc
        bc = {"I_top": 0.0, "I_bottom": bots[l]}
        Jo = oracle.direct_solve(chis[l], epss[l], Bs[l], 4, 8, True, bc)
        err = np.max(np.abs(Jg[l] - Jo) / np.abs(Jo))
        assert err < 1e-8, (l, err)


def test_batched_equals_unbatched(rt3d):
    """Each wavelength of a batch gives the unbatched rt3d_solve result."""
    n = (16, 14, 12)
    nl = 4
    chis, epss, Bs, bots = _batch(n, nl, 4)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
    g = rt3d.Grid(n, 4, 8, rt3d.PARABOLIC, rt3d.FP32_FS_FP64_ALI)
    J = d(Bs).clone()
    st = g.solve_batched(d(chis), d(epss), d(Bs), {"I_top": 0.0, "I_bottom": d(bots)}, J,
                         tol=1e-9, max_iter=3000)
    assert st["graph_replays"] > 0 and st["fs_lambda64"] >= 2 * nl
    # the batched autotuner timed every one-characteristic-per-thread shape
    cands = [rt3d.fs_tune_shape(i) for i in range(rt3d.FS_TUNE_SHAPES)]
    assert st["fs_shape"] in [c for c in cands if c[1] == 1]
    assert all((t > 0) == (c[1] == 1) for t, c in zip(st["fs_tune_ms"], cands))
    for l in range(nl):
        Jl = d(Bs[l]).clone()
        g.solve(d(chis[l]), d(epss[l]), d(Bs[l]), {"I_top": 0.0, "I_bottom": d(bots[l])}, Jl,
                tol=1e-9, max_iter=3000)
        a, b = J[l].cpu().numpy(), Jl.cpu().numpy()
        assert np.max(np.abs(a - b) / np.abs(b)) < 2e-9, l
