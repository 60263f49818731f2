"""Oracle (test infrastructure only): gas/photon model coefficients of Section 2.1.

Every function restates one definition of the paper's Section 2.1 in FP64.
"""
from __future__ import annotations

import numpy as np


def mason_monchick_A(d_r, d_v, Z_r, Z_v, Sc):
    """Thermal relaxation-rate matrix A from the asymptotic expansion of the WCU
    equation (Section 2.1, the matrix following the auxiliary heat fluxes)."""
    A = np.zeros((3, 3))
    A[0, 0] = 2.0 / 3.0 + 5.0 / 6.0 * (d_r / ((3 + d_r) * Z_r) + d_v / ((3 + d_v) * Z_v))
    A[0, 1] = -5.0 / (2.0 * (3 + d_r) * Z_r)
    A[0, 2] = -5.0 / (2.0 * (3 + d_v) * Z_v)
    A[1, 0] = -d_r / ((3 + d_r) * Z_r)
    A[1, 1] = Sc + 3.0 / (2.0 * (3 + d_r) * Z_r)
    A[2, 0] = -d_v / ((3 + d_v) * Z_v)
    A[2, 2] = Sc + 3.0 / (2.0 * (3 + d_v) * Z_v)
    return A


def relaxation_matrix(model):
    """A of the model: the user-given 3x3 matrix, else the Mason-Monchick form."""
    if model.A is not None:
        return np.asarray(model.A, np.float64).reshape(3, 3)
    return mason_monchick_A(model.d_r, model.d_v, model.Z_r, model.Z_v, model.Sc)


def aux_heat_flux_matrix(A, Z_r, Z_v):
    """(q_0, q_1, q_2) = Mix @ (q_t, q_r, q_v), Section 2.1, with Z_int = (1/Z_r + 1/Z_v)^-1."""
    Zi = 1.0 / (1.0 / Z_r + 1.0 / Z_v)
    return np.array([
        [(2.0 - 3.0 * A[0, 0]) * Zi + 1.0, -3.0 * A[0, 1] * Zi, -3.0 * A[0, 2] * Zi],
        [-A[1, 0] * Zi, 1.0 - A[1, 1] * Zi, -A[1, 2] * Zi],
        [-A[2, 0] * Zi, -A[2, 1] * Zi, 1.0 - A[2, 2] * Zi],
    ])


def mode_temperatures(T_t, T_r, T_v, d_r, d_v):
    """T_tr, T_tv and total T for constant d_v (Section 2.1)."""
    T_tr = (3.0 * T_t + d_r * T_r) / (3.0 + d_r)
    T_tv = (3.0 * T_t + d_v * T_v) / (3.0 + d_v)
    T = (3.0 * T_t + d_r * T_r + d_v * T_v) / (3.0 + d_r + d_v)
    return T_tr, T_tv, T


def d_v_of_T(T_v, T_v_ref):
    """Vibrational degrees of freedom d_v(T_v) (Section 2.1)."""
    x = T_v_ref / T_v
    return 2.0 * x / np.expm1(x)


def relaxation_time(rho, T_t, Kn, omega):
    """tau = sqrt(2/pi) T_t^(omega-1) Kn / rho (Section 2.1)."""
    return np.sqrt(2.0 / np.pi) * T_t ** (omega - 1.0) * Kn / rho


def absorption(rho, model):
    """k_eff = 1/Kn_photon (Section 2.1); optionally scaled by the local density."""
    k = 1.0 / model.Kn_p
    return k * rho if model.k_eff_density_scaled else k * np.ones_like(rho)


def kappa_gas(p_t, tau, A, d_r, d_v):
    """kappa_gas = (p_t tau / 2) A^-1 diag(5, d_r, d_v) (Eq. NSF_thermal_conductivities).

    Returns an array [..., 3, 3] for array-valued p_t*tau.
    """
    base = np.linalg.inv(A) @ np.diag([5.0, d_r, d_v])
    return 0.5 * np.asarray(p_t * tau)[..., None, None] * base


def sound_speed(T_t):
    """Frozen acoustic speed of the convective system, whose pressure is the
    translational pressure p_t = rho T_t only: c_s = sqrt(5 T_t / 3)."""
    return np.sqrt(5.0 * T_t / 3.0)
