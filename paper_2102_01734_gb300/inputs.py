"""Seeded synthetic atmospheres shaped like the paper's test cases.

Input generation only: nothing here computes any step of the formal solution
or of the ALI iteration. Both the CUDA path and the CPU oracle are fed from
these arrays.

Workloads (they stand in for the paper's PBC test atmosphere, Sec. 3.1; no
dataset is involved):

* ``vertical_chi(nz)``: chi(z) = 10^(-4 + 6 (nz-1-z)/(nz-1)) per unit length,
  z = 0 the inner (bottom) layer, so the outer layer has chi = 1e-4 and the
  inner one 1e2 (per-voxel vertical optical depth 1e-4 .. 1e2).
* ``powerlaw_field(shape, seed)``: Gaussian random field with power spectrum
  P(k) ~ k^-3: seeded white noise, FFT, amplitude times |k|^-3/2, k = 0 mode
  removed, inverse FFT, scaled to unit standard deviation and clipped to
  +-4.5 so that B = 1 + 0.2 g stays positive.
* ``cartesian_config(...)``: chi = vertical_chi * exp(0.5 g) (sigma_ln = 0.5),
  B = 1 + 0.2 g, uniform eps; boundary: no incoming intensity at the top,
  I = B of the entered bottom voxel at the bottom.

* ``grey_config(...)``: the paper's PBC test atmosphere with its grey
  temperature structure (Sec. 3.1, items 3 and 4): chi as in
  ``cartesian_config``, the vertical optical depth of each column at the
  voxel centres tau(nz-1) = chi(nz-1)/2, tau(z) = tau(z+1) + (chi(z) +
  chi(z+1))/2 (unit spacing, tau growing inward), and B = 3/4 (tau + 2/3),
  the grey (Eddington) structure T^4 = 3/4 Teff^4 (tau + 2/3) in units of
  sigma Teff^4 / pi; boundary: no incoming intensity at the top, and the
  LTE diffusion condition at the bottom (its face arrays are derived from
  chi and B by the library, not here).

* ``spherical_config(...)``: the paper's second test geometry (a spherical
  shell, Sec. 3.2) on a (r, theta, phi) grid with log-spaced radial edges from
  r_in to r_out: chi = C r^-12 at the cell's geometric-mean radius with C set
  by the radial optical depth tau_core of the shell, B = 1, uniform eps;
  boundary: I = B leaving the core, no incoming intensity at the outer sphere
  except an irradiation I_irr (in units of B) from the side x > 0.

* ``line_profile(nl, ...)``: the wavelengths of one spectral line for the
  line-transfer solve (profile-averaged mean intensity, Sec. 2): nl points
  x_l equally spaced in [-xmax, xmax] Doppler widths, opacity scale
  strength * exp(-x_l^2) (a Doppler profile, 1 at line centre), and
  weights wphi_l = trapezoid weight * exp(-x_l^2) / sqrt(pi), normalised to
  sum 1 (the quadrature of int phi dx = 1 on the sampled band).

Cartesian arrays have shape (nz, ny, nx), x fastest; spherical ones
(nphi, ntheta, nr), r fastest.
"""
from __future__ import annotations

import numpy as np


def vertical_chi(nz: int) -> np.ndarray:
    z = np.arange(nz, dtype=np.float64)
    if nz == 1:
        return np.full(1, 1e-4)
    return 10.0 ** (-4.0 + 6.0 * (nz - 1 - z) / (nz - 1))


def powerlaw_field(shape, seed: int, slope: float = -3.0, clip: float = 4.5) -> np.ndarray:
    rng = np.random.default_rng(seed)
    white = rng.standard_normal(shape)
    f = np.fft.fftn(white)
    ks = np.meshgrid(*[np.fft.fftfreq(n) for n in shape], indexing="ij")
    k = np.sqrt(sum(kk * kk for kk in ks))
    amp = np.zeros_like(k)
    nz = k > 0
    amp[nz] = k[nz] ** (slope / 2.0)
    g = np.real(np.fft.ifftn(f * amp))
    g -= g.mean()
    g /= g.std()
    return np.clip(g, -clip, clip)


def cartesian_config(n, eps: float, seed: int | None = None, sigma_ln: float = 0.5,
                     b_amp: float = 0.2):
    """(chi, eps, B, bc) on a box of n = (nx, ny, nz) voxels (or an int)."""
    if np.isscalar(n):
        n = (int(n),) * 3
    nx, ny, nz = n
    shape = (nz, ny, nx)
    chi = np.broadcast_to(vertical_chi(nz)[:, None, None], shape).copy()
    if seed is None:
        B = np.ones(shape)
    else:
        g = powerlaw_field(shape, seed)
        chi = chi * np.exp(sigma_ln * g)
        B = 1.0 + b_amp * g
    epsa = np.full(shape, float(eps))
    bc = {"I_top": 0.0, "I_bottom": B[0].copy()}
    return chi, epsa, B, bc


def grey_tau(chi: np.ndarray) -> np.ndarray:
    """Vertical optical depth at the voxel centres of each column of chi
    (nz, ny, nx): half a voxel below the top face, then trapezoidal steps."""
    tau = np.empty_like(chi)
    tau[-1] = 0.5 * chi[-1]
    for z in range(chi.shape[0] - 2, -1, -1):
        tau[z] = tau[z + 1] + 0.5 * (chi[z] + chi[z + 1])
    return tau


def grey_config(n, eps: float, seed: int | None = None, sigma_ln: float = 0.5):
    """(chi, eps, B, bc) of the grey atmosphere: B = 3/4 (tau + 2/3); bc holds
    only I_top = 0 (the diffusion faces come from the library)."""
    if np.isscalar(n):
        n = (int(n),) * 3
    nx, ny, nz = n
    shape = (nz, ny, nx)
    chi = np.broadcast_to(vertical_chi(nz)[:, None, None], shape).copy()
    if seed is not None:
        chi = chi * np.exp(sigma_ln * powerlaw_field(shape, seed))
    B = 0.75 * (grey_tau(chi) + 2.0 / 3.0)
    return chi, np.full(shape, float(eps)), B, {"I_top": 0.0}


# Named workloads (sizes of the benchmark configurations).
CONFIGS = {
    # plain method, FP64: 33^3 box, 8 x 16 angles, linear interpolation
    "box33_fp64": dict(n=33, eps=1e-2, seed=None, ntheta=8, nphi=16, parabolic=False),
    # 129^3 box with the k^-3 lognormal field, 32 x 64 angles, parabolic
    "box129_field": dict(n=129, eps=1e-6, seed=1, ntheta=32, nphi=64, parabolic=True),
    # 97^3 box, 16 x 32 angles, batched wavelengths
    "box97_batched": dict(n=97, eps=None, seed=1, ntheta=16, nphi=32, parabolic=True),
}


def spherical_config(n, eps: float, tau_core: float = 100.0, r_in: float = 1.0,
                     r_out: float = 1.3, I_irr: float = 10.0):
    """(chi, eps, B, bc) on an (nr, ntheta, nphi) spherical grid; chi = C r^-12
    with tau(r_in) = integral of chi over [r_in, r_out] = tau_core."""
    nr, nt, np_ = (int(v) for v in n)
    re = r_in * (r_out / r_in) ** (np.arange(nr + 1) / nr)
    rc = np.sqrt(re[:-1] * re[1:])
    C = tau_core * 11.0 / (r_in ** -11 - r_out ** -11)
    chi = np.broadcast_to(C * rc ** -12.0, (np_, nt, nr)).copy()
    B = np.ones_like(chi)
    eps_a = np.full_like(chi, eps)
    bc = {"I_top": 0.0, "I_bottom": np.ones((np_, nt)), "I_irr": float(I_irr)}
    return chi, eps_a, B, bc


def batched_wavelengths(nlambda: int, seed: int = 3):
    """Per-wavelength eps (log-uniform in [1e-8, 1e-1]) and opacity scale
    10^U(-3, 3), seeded."""
    rng = np.random.default_rng(seed)
    eps = 10.0 ** rng.uniform(-8.0, -1.0, nlambda)
    scale = 10.0 ** rng.uniform(-3.0, 3.0, nlambda)
    return eps, scale


def line_profile(nl: int, xmax: float = 3.0, strength: float = 1.0):
    """(scale, wphi) of nl wavelengths across a Doppler line profile."""
    x = np.linspace(-xmax, xmax, nl) if nl > 1 else np.zeros(1)
    phi = np.exp(-x * x) / np.sqrt(np.pi)
    w = np.full(nl, 2.0 * xmax / max(nl - 1, 1))
    if nl > 1:
        w[0] *= 0.5
        w[-1] *= 0.5
    wphi = w * phi
    wphi /= wphi.sum()
    return strength * np.exp(-x * x), wphi
