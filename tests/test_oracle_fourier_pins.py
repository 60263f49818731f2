"""Pins of the Fourier stability oracle (Section 4): the xi_x integrals against the
plasma-dispersion closed form, the photon sphere integrals against quadrature, the CIS
conserved modes at theta -> 0, and the paper's statements about CIS and GSIS for its
cases A, B and C (d_r = 2, d_v = 1, Z_r = 2.67, Z_v = 26.7)."""
import math

import numpy as np
import pytest

from oracle import fourier as FO


@pytest.fixture(scope="module")
def grid():
    return FO.velocity_grid(n_x=1601, L=10.0)


@pytest.mark.parametrize("a", [0.3, 1.0, 3.0])
def test_xi_x_integrals_match_the_faddeeva_form(a):
    x = np.linspace(-12, 12, 40001)
    g = np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)
    for k in range(5):
        dense = np.trapezoid(g * x ** k / (1 + 1j * a * x), x)
        assert abs(dense - FO.xi_x_integral_faddeeva(k, a)) < 1e-10


def test_photon_sphere_integrals():
    mu, wm = np.polynomial.legendre.leggauss(400)
    for b in (0.05, 1.0, 20.0):
        i0, i1 = FO.photon_integrals(b)
        assert abs(i0 - 2 * math.pi * np.sum(wm / (1 + 1j * b * mu))) < 1e-10
        assert abs(i1 - 2 * math.pi * np.sum(wm * mu / (1 + 1j * b * mu))) < 1e-10


def test_the_velocity_grid_integrates_the_equilibrium_moments(grid):
    xi, w = grid
    f = (2 * math.pi) ** -1.5 * np.exp(-0.5 * np.sum(xi * xi, axis=1))
    assert abs(w @ f - 1) < 1e-12
    assert abs(w @ (xi[:, 0] ** 2 * f) - 1) < 1e-12
    assert abs(w @ (np.sum(xi * xi, axis=1) ** 2 * f) - 15) < 1e-10


def test_cis_keeps_conserved_modes_at_long_wavelength(grid):
    p = FO.Params(ratio=0.1, sigma_R=0.01)
    e = FO.spectral_radius_cis(p, 1e-5, grid)
    assert abs(e - 1.0) < 1e-3


KNT = np.logspace(-3, 1, 9)


def test_case_a_cis_converges(grid):
    """(Kn/Kn_p) sigma_R < 0.03: e_max <= 1 at every wavelength."""
    for ratio, sig in ((1.0, 0.01), (0.1, 0.1), (1e-3, 0.1)):
        p = FO.Params(ratio, sig)
        assert max(FO.spectral_radius_cis(p, k, grid) for k in KNT) <= 1.0 + 1e-6


@pytest.mark.parametrize("ratio,sig", [(0.1, 0.5), (10.0, 0.005)])
def test_cases_b_and_c_cis_diverge_at_long_wavelength(grid, ratio, sig):
    p = FO.Params(ratio, sig)
    assert FO.spectral_radius_cis(p, 1e-2, grid) > 1.0


@pytest.mark.parametrize("ratio,sig", [(1.0, 0.01), (0.1, 0.5), (10.0, 0.005)])
def test_gsis_decay_factor_below_one_half(grid, ratio, sig):
    """Near-continuum wavelengths, Kn theta <= 1, where CIS slows down or diverges."""
    p = FO.Params(ratio, sig)
    assert max(FO.spectral_radius_gsis(p, k, grid) for k in np.logspace(-3, 0, 7)) < 0.5
