"""The normal-shock workload's boundary states: the Rankine-Hugoniot downstream state
conserves the mass, momentum and energy fluxes of the upstream state (Section 'Normal
shock wave'), and the step initial state and far-field patches carry those two states."""
import numpy as np

import gsis_inputs as gi


def _fluxes(rho, u, T, dof_internal):
    p = rho * T
    e = rho * (0.5 * u * u + 0.5 * (3.0 + dof_internal) * T)
    return rho * u, rho * u * u + p, u * (e + p)


def test_rankine_hugoniot_conserves_fluxes():
    for d_r, d_v, Mach in ((2.0, 1.16, 5.0), (2.0, 0.0, 2.0), (0.0, 0.0, 3.0)):
        gamma = (5.0 + d_r + d_v) / (3.0 + d_r + d_v)
        rho_d, u_d, T_d = gi.workloads.rankine_hugoniot(Mach, gamma)
        up = _fluxes(1.0, np.sqrt(gamma) * Mach, 1.0, d_r + d_v)
        down = _fluxes(rho_d, u_d, T_d, d_r + d_v)
        assert np.allclose(up, down, rtol=1e-12)
        assert rho_d > 1.0 and T_d > 1.0 and u_d < np.sqrt(gamma * T_d)   # subsonic downstream


def test_monatomic_strong_shock_limit():
    # gamma = 5/3 as Mach -> infinity: density ratio (gamma + 1) / (gamma - 1) = 4
    rho_d, _, _ = gi.workloads.rankine_hugoniot(1e4, 5.0 / 3.0)
    assert abs(rho_d - 4.0) < 1e-6


def test_shock_workload_states():
    wl = gi.workloads.normal_shock(length=20.0, dx=0.5, n_xi=32, n_theta=8)
    assert wl.mesh.n_cells == 40 and abs(wl.model.Kn - 5.0 * np.pi / 16.0) < 1e-15
    up, down = wl.mesh.patches
    M = gi.fields.shock_fields(wl)
    x = wl.mesh.cell_centroid[:, 0]
    assert np.all(M[x <= 0, 0] == up.rho) and np.all(M[x > 0, 0] == down.rho)
    assert np.all(M[x > 0, 4:8] == down.T_t) and np.all(M[x <= 0, 1] == up.u[0])
    # the photon directions cover the sphere: sum of weights 4 pi, first moment zero
    assert abs(wl.wo.sum() - 4.0 * np.pi) < 1e-12 and abs((wl.wo * wl.omega[:, 0]).sum()) < 1e-12
