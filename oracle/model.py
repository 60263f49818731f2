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


def relaxation_matrix(model, d_v=None):
    """A of the model: the user-given 3x3 matrix, else the Mason-Monchick form at d_v
    (default: the model's constant d_v; per cell, d_v(T_v) when it depends on T_v)."""
    if model.A is not None:
        return np.asarray(model.A, np.float64).reshape(3, 3)
    return mason_monchick_A(model.d_r, model.d_v if d_v is None else d_v, model.Z_r, model.Z_v, model.Sc)


def aux_heat_flux_matrix(A, Z_r, Z_v):
    """(q_0, q_1, q_2) = Mix @ (q_t, q_r, q_v), Section 2.1, with Z_int = (1/Z_r + 1/Z_v)^-1."""
    Zi = 1.0 / (1.0 / Z_r + 1.0 / Z_v)
    return np.array([
        [(2.0 - 3.0 * A[0, 0]) * Zi + 1.0, -3.0 * A[0, 1] * Zi, -3.0 * A[0, 2] * Zi],
        [-A[1, 0] * Zi, 1.0 - A[1, 1] * Zi, -A[1, 2] * Zi],
        [-A[2, 0] * Zi, -A[2, 1] * Zi, 1.0 - A[2, 2] * Zi],
    ])


def d_v_of_T(T_v, T_v_ref):
    """Vibrational degrees of freedom d_v(T_v) = 2 x / (e^x - 1), x = T_v_ref / T_v (Section 2.1)."""
    x = T_v_ref / T_v
    return 2.0 * x / np.expm1(x)


def vib_energy(T, model):
    """Vibrational energy per unit density, d_v(T) T / 2 (Section 2.1: e_v = d_v(T_v) rho T_v / 2).
    With the temperature-dependent d_v this is T_v_ref / (e^(T_v_ref / T) - 1)."""
    T = np.asarray(T, np.float64)
    if getattr(model, "dv_temperature_dependent", False):
        return model.Tv_ref / np.expm1(model.Tv_ref / T)
    return 0.5 * model.d_v * T


def vib_temperature(eps, model):
    """Inverse of vib_energy: the T with d_v(T) T / 2 = eps; in closed form
    T_v_ref / ln(1 + T_v_ref / eps) for the temperature-dependent d_v."""
    eps = np.asarray(eps, np.float64)
    if getattr(model, "dv_temperature_dependent", False):
        return model.Tv_ref / np.log1p(model.Tv_ref / eps)
    return 2.0 * eps / model.d_v


def vib_heat_capacity(T, model):
    """d(vib_energy)/dT: x^2 e^x / (e^x - 1)^2 with x = T_v_ref / T, or d_v / 2."""
    T = np.asarray(T, np.float64)
    if getattr(model, "dv_temperature_dependent", False):
        x = model.Tv_ref / T
        return x * x * np.exp(x) / np.expm1(x) ** 2
    return 0.5 * model.d_v * np.ones_like(T)


def dv_local(T_v, model):
    """d_v at the vibrational temperature: the constant, or d_v(T_v)."""
    if getattr(model, "dv_temperature_dependent", False):
        return d_v_of_T(np.asarray(T_v, np.float64), model.Tv_ref)
    return model.d_v * np.ones_like(np.asarray(T_v, np.float64))


def _solve_equal_temperature(base, rhs, model):
    """The T with base T + 2 vib_energy(T) = rhs, by Newton from rhs / (base + d_v):
    the left side increases with T, so the root is unique; iterate to |dT| <= 1e-15 T."""
    T = rhs / (base + 2.0 * vib_heat_capacity(np.maximum(rhs / (base + 1.0), 1e-3), model))
    for _ in range(60):
        g = base * T + 2.0 * vib_energy(T, model) - rhs
        dT = g / (base + 2.0 * vib_heat_capacity(T, model))
        T = T - dT
        if np.all(np.abs(dT) <= 1e-15 * np.abs(T)):
            break
    return T


def mode_temperatures(T_t, T_r, T_v, model):
    """T_tr, T_tv and total T (Section 2.1):
        T_tr = (3 T_t + d_r T_r) / (3 + d_r),
        (3 + d_v(T_tv)) T_tv = 3 T_t + d_v(T_v) T_v,
        (3 + d_r + d_v(T)) T = 3 T_t + d_r T_r + d_v(T_v) T_v,
    explicit for constant d_v and solved by Newton for the temperature-dependent one."""
    d_r = model.d_r
    T_tr = (3.0 * T_t + d_r * T_r) / (3.0 + d_r)
    ev = 2.0 * vib_energy(T_v, model)
    if not getattr(model, "dv_temperature_dependent", False):
        d_v = model.d_v
        return T_tr, (3.0 * T_t + d_v * T_v) / (3.0 + d_v), (3.0 * T_t + d_r * T_r + d_v * T_v) / (3.0 + d_r + d_v)
    T_tv = _solve_equal_temperature(3.0, 3.0 * T_t + ev, model)
    T = _solve_equal_temperature(3.0 + d_r, 3.0 * T_t + d_r * T_r + ev, model)
    return T_tr, T_tv, T


def relaxation_time(rho, T_t, Kn, omega):
    """tau = sqrt(2/pi) T_t^(omega-1) Kn / rho (Section 2.1)."""
    return np.sqrt(2.0 / np.pi) * T_t ** (omega - 1.0) * Kn / rho


def absorption(rho, model):
    """k_eff = 1/Kn_photon (Section 2.1); optionally scaled by the local density."""
    k = 1.0 / model.Kn_p
    return k * rho if model.k_eff_density_scaled else k * np.ones_like(rho)


def sound_speed(T_t):
    """Frozen acoustic speed of the convective system, whose pressure is the
    translational pressure p_t = rho T_t only: c_s = sqrt(5 T_t / 3)."""
    return np.sqrt(5.0 * T_t / 3.0)
