"""The synthetic workloads match the recipe they stand for: the vertical
opacity profile, the k^-3 Gaussian random field, chi and B built from it, the
batched wavelength draws and the spherical shell's radial optical depth."""
import numpy as np
from scipy import integrate

from paper_2102_01734_gb300 import inputs


def test_vertical_profile_spans_1e_minus_4_to_1e2():
    chi = inputs.vertical_chi(129)
    assert chi[0] == 1e2 and abs(chi[-1] - 1e-4) < 1e-18
    assert np.allclose(np.diff(np.log10(chi)), -6.0 / 128)


def test_field_has_unit_variance_zero_mean_and_a_k_minus_3_spectrum():
    g = inputs.powerlaw_field((64, 64, 64), seed=1)
    assert abs(g.mean()) < 1e-3 and abs(g.std() - 1.0) < 1e-3
    assert g.max() <= 4.5 and g.min() >= -4.5
    # spherically averaged power spectrum: slope -3 over the mid range
    p = np.abs(np.fft.fftn(g)) ** 2
    ks = np.meshgrid(*[np.fft.fftfreq(64)] * 3, indexing="ij")
    k = np.sqrt(sum(kk * kk for kk in ks)).ravel()
    bins = np.geomspace(4 / 64, 24 / 64, 9)  # enough modes per shell
    idx = np.digitize(k, bins)
    kc = [np.exp(np.log(k[idx == i]).mean()) for i in range(1, len(bins))]
    pc = [p.ravel()[idx == i].mean() for i in range(1, len(bins))]
    slope = np.polyfit(np.log(kc), np.log(pc), 1)[0]
    assert abs(slope + 3.0) < 0.15, slope


def test_cartesian_config_builds_chi_and_b_from_the_field():
    chi, eps, B, bc = inputs.cartesian_config((20, 18, 16), 1e-6, seed=5)
    g = inputs.powerlaw_field((16, 18, 20), 5)
    assert np.allclose(chi, inputs.vertical_chi(16)[:, None, None] * np.exp(0.5 * g), rtol=1e-14)
    assert np.allclose(B, 1.0 + 0.2 * g, rtol=1e-14)
    assert np.all(B > 0) and np.all(eps == 1e-6)
    assert bc["I_top"] == 0.0 and np.array_equal(bc["I_bottom"], B[0])


def test_batched_wavelength_draws():
    eps, scale = inputs.batched_wavelengths(256, seed=3)
    assert eps.min() >= 1e-8 and eps.max() <= 1e-1
    assert scale.min() >= 1e-3 and scale.max() <= 1e3
    le = np.log10(eps)
    assert abs(le.mean() + 4.5) < 0.3  # log-uniform over [-8, -1]


def test_spherical_shell_radial_optical_depth():
    n = (65, 33, 65)
    chi, eps, B, bc = inputs.spherical_config(n, 1e-4, tau_core=100.0)
    assert chi.shape == (65, 33, 65)
    # chi = C r^-12 at the geometric-mean radius of every radial cell
    re = 1.3 ** (np.arange(66) / 65)
    rc = np.sqrt(re[:-1] * re[1:])
    C = chi[0, 0, 0] * rc[0] ** 12
    assert np.allclose(chi[3, 7, :], C * rc ** -12.0, rtol=1e-14)
    # the exact integral of C r^-12 over [1, 1.3] is tau_core
    tau, _ = integrate.quad(lambda r: C * r ** -12.0, 1.0, 1.3, epsabs=0, epsrel=1e-12)
    assert abs(tau - 100.0) < 1e-9
    assert np.all(B == 1.0) and bc["I_irr"] == 10.0 and np.all(bc["I_bottom"] == 1.0)
