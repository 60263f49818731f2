"""Pins of the oracle's temperature-dependent vibrational degrees of freedom
d_v(T_v) = 2 x / (e^x - 1), x = T_v_ref / T_v (Section 2.1).

* the vibrational energy d_v(T) T / 2, its closed-form inverse and its derivative,
  against the paper's definition written out here and central differences;
* T_tv and T satisfy the paper's implicit definitions (3 + d_v(T_tv)) T_tv =
  3 T_t + d_v(T_v) T_v and (3 + d_r + d_v(T)) T = 3 T_t + d_r T_r + d_v(T_v) T_v;
* with those temperatures the reference distributions conserve mass, momentum and energy
  (the d_v(T_tv) denominator is what makes the energy balance hold);
* moments of an equilibrium return its T_v; the exact source Jacobian block equals
  central differences of the source; a uniform equilibrium stays a fixed point of the
  kinetic sweep and of the synthetic residual.
"""
import dataclasses

import numpy as np
import pytest

import gsis_inputs as gi
from gsis_inputs import quadrature as Q
from oracle import kinetic as K
from oracle import macro as MA
from oracle import model as mdl

TREF = 3.0


def _model(**kw):
    return dataclasses.replace(gi.workloads.ModelParams(), dv_temperature_dependent=True, Tv_ref=TREF, **kw)


def _dv(T):
    x = TREF / T
    return 2.0 * x / (np.exp(x) - 1.0)


def test_vibrational_energy_inverse_and_heat_capacity():
    m = _model()
    T = np.linspace(0.3, 8.0, 50)
    e = mdl.vib_energy(T, m)
    assert np.allclose(e, 0.5 * _dv(T) * T, rtol=1e-14)
    assert np.allclose(mdl.vib_temperature(e, m), T, rtol=1e-13)
    h = 1e-6
    fd = (mdl.vib_energy(T + h, m) - mdl.vib_energy(T - h, m)) / (2 * h)
    assert np.allclose(mdl.vib_heat_capacity(T, m), fd, rtol=1e-8)
    assert np.all(_dv(T) < 2.0) and abs(_dv(np.array([1e4]))[0] - 2.0) < 1e-3   # classical limit d_v -> 2
    const = gi.workloads.ModelParams()
    assert np.allclose(mdl.vib_energy(T, const), 0.5 * const.d_v * T)


def test_mode_temperatures_solve_the_implicit_definitions():
    m = _model()
    rng = np.random.default_rng(3)
    Tt, Tr, Tv = (rng.uniform(0.5, 4.0, 40) for _ in range(3))
    T_tr, T_tv, T = mdl.mode_temperatures(Tt, Tr, Tv, m)
    assert np.allclose((3 + _dv(T_tv)) * T_tv, 3 * Tt + _dv(Tv) * Tv, rtol=1e-13)
    assert np.allclose((3 + m.d_r + _dv(T)) * T, 3 * Tt + m.d_r * Tr + _dv(Tv) * Tv, rtol=1e-13)
    assert np.allclose(T_tr, (3 * Tt + m.d_r * Tr) / (3 + m.d_r))
    # equal mode temperatures are their own equilibrium
    _, T_tv, T = mdl.mode_temperatures(Tt, Tt, Tt, m)
    assert np.allclose(T_tv, Tt, rtol=1e-13) and np.allclose(T, Tt, rtol=1e-13)


@pytest.mark.parametrize("dim", [1, 2])
def test_reference_conserves_energy_with_temperature_dependent_dv(dim):
    m = _model()
    xi, w = Q.trapezoid_nd(64, 13.0, dim)
    M = gi.fields.random_macro_fields(5, dim, seed=21, u_scale=0.4, q_scale=0.1)
    F = K.fields_from_record(M, m.sigma_R)
    g = K.reference_planes(F, xi, dim, m)
    rho, u = F["rho"], F["u"]
    assert np.allclose(g[..., 0] @ w, rho, rtol=1e-10)
    for a in range(dim):
        assert np.allclose((g[..., 0] * w) @ xi[:, a], rho * u[:, a], rtol=1e-10, atol=1e-12)
    c2 = np.sum((xi[None, :, :dim] - u[:, None, :dim]) ** 2, axis=-1)
    E = 0.5 * ((c2 * g[..., 0]) @ w + g[..., 1] @ w) + g[..., 2] @ w + g[..., 3] @ w
    E_ref = rho * (1.5 * F["T_t"] + 0.5 * m.d_r * F["T_r"] + 0.5 * _dv(F["T_v"]) * F["T_v"])
    assert np.allclose(E, E_ref, rtol=1e-10)
    # the vibrational energy of g alone relaxes towards d_v(T_tv) T_tv / 2, not the
    # constant-d_v value: the two models differ
    const = gi.workloads.ModelParams(d_v=float(_dv(np.array([1.5]))[0]))
    g_c = K.reference_planes(F, xi, dim, const)
    assert np.abs(g_c[..., 3] @ w - g[..., 3] @ w).max() > 1e-4


def test_moments_of_equilibrium_return_the_vibrational_temperature():
    m = _model()
    xi, w = Q.trapezoid_nd(48, 12.0, 2)
    om, wo = Q.photon_product(4, 4)
    M = gi.fields.random_macro_fields(4, 2, seed=22, u_scale=0.3)
    F = K.fields_from_record(M, m.sigma_R)
    f = K.equilibrium_planes(F, xi, 2, m)
    G = K.moments(f, np.zeros((4, om.shape[0])), xi, w, om, wo, 2, m)
    assert np.allclose(G["T_v"], F["T_v"], rtol=1e-11)
    assert np.allclose(f[..., 3] @ w, F["rho"] * 0.5 * _dv(F["T_v"]) * F["T_v"], rtol=1e-11)


@pytest.mark.parametrize("dependent", [False, True])
def test_source_jacobian_block_matches_central_differences(dependent):
    m = _model() if dependent else gi.workloads.ModelParams()
    dim = 2
    Fr = K.fields_from_record(gi.fields.random_macro_fields(6, dim, seed=24, u_scale=0.3), m.sigma_R)
    W = MA.conservative(Fr, dim, m)
    E, ER = 1 + dim, 4 + dim
    J = MA.source_jacobian_block(MA.primitive(W, dim, m), dim, m)

    def Q_of(Wx):
        # sources in the gas-energy rows (e_gas, e_r, e_v, e_R) with tau and k_eff frozen
        prim = MA.primitive(Wx, dim, m)
        tau = mdl.relaxation_time(prim[0], MA.primitive(W, dim, m)[2], m.Kn, m.omega)
        Tt = prim[2]
        q = MA.source(prim, dim, m)
        # undo the T_t dependence of tau: rescale the relaxation terms to the frozen tau
        tau_x = mdl.relaxation_time(prim[0], Tt, m.Kn, m.omega)
        Qr = q[:, E + 1] * tau_x / tau
        k = mdl.absorption(prim[0], m)
        exch = k * (4 * m.sigma_R * prim[4] ** 4 - prim[5])
        Qv = (q[:, E + 2] + exch) * tau_x / tau - exch
        return np.stack([-exch, Qr, Qv, exch], 1)

    for col, row in enumerate((E, E + 1, E + 2, ER)):
        h = 1e-6 * np.abs(W[:, row]).max()
        dW = np.zeros_like(W)
        dW[:, row] = h
        if row == ER:                    # gas-energy variables: e_R moves, e_gas = e - e_R held
            dW[:, E] = h
        fd = (Q_of(W + dW) - Q_of(W - dW)) / (2 * h)
        assert np.allclose(J[:, :, col], fd, rtol=1e-6, atol=1e-8 * np.abs(J).max()), (col, J[0, :, col], fd[0])


def test_uniform_equilibrium_stays_a_fixed_point_with_dv_of_T():
    wl = gi.workloads.slab(n_cells=8, T_left=1.0, T_right=1.0)
    wl = gi.workloads.with_model(gi.workloads.with_solver(wl, order=2), dv_temperature_dependent=True, Tv_ref=TREF)
    M = gi.fields.uniform_fields(8, rho=1.1, T=1.0)
    F = K.fields_from_record(M, wl.model.sigma_R)
    f = K.equilibrium_planes(F, wl.xi, 1, wl.model)
    I = K.photon_equilibrium(F["T_R"], wl.omega.shape[0], wl.model.sigma_R)
    fn, In = K.kinetic_sweep(f, I, wl)
    assert np.abs(fn - f).max() < 1e-13 * np.abs(f).max()
    faces = MA.Faces(K.Geometry(wl.mesh))
    Fk = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, 1, wl.model)
    hot = MA.high_order_terms(faces, Fk, MA.kinetic_boundary_flux(faces, f, I, wl), wl)
    assert np.abs(MA.residual(MA.conservative(Fk, 1, wl.model), faces, hot, wl)).max() < 1e-12
