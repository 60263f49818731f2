"""Pins of the oracle's synthetic-equation solver and GSIS loop (Sections 2.2, 3, 5, 6).

* a uniform equilibrium at rest between walls at its own temperature is a fixed point of
  the macroscopic residual (exactly with the slab's Gauss-Hermite grid, to the
  quadrature error with the cavity's trapezoid grid);
* pure conduction between two walls with no high-order terms: T^(1+omega) is linear
  and the heat flux is -K_g d(T^(1+omega))/dx / (1 + omega) with
  K_g = sqrt(2/pi) Kn/2 * 1^T A^-1 diag(5, d_r, d_v) 1 (Eqs. NSF_constitutive and
  NSF_thermal_conductivities with mu = p tau);
* GSIS keeps the total mass of a closed domain, reaches in a few dozen iterations a
  residual that CIS does not reach in the same number (Section 6), and in the
  near-continuum, optically thick limit on a coarse mesh converges to the Kirchhoff
  solution of the radiative NSF conduction problem (Section 4), with first-order
  convergence under refinement, where CIS stays far from it.
"""
import numpy as np
import pytest

import gsis_inputs as gi
from oracle import gsis as OG
from oracle import kinetic as K
from oracle import macro as MA
from oracle import model as mdl


def _zero_hot(faces, dim):
    nf, nb = faces.i.shape[0], faces.bf_cell.shape[0]
    return {"sigma": np.zeros((nf, dim, dim)), "q_t": np.zeros((nf, dim)), "q_r": np.zeros((nf, dim)),
            "q_v": np.zeros((nf, dim)), "q_R": np.zeros((nf, dim)), "boundary": np.zeros((nb, dim + 5))}


def _eq_state(wl, T):
    M = gi.fields.uniform_fields(wl.mesh.n_cells, T=T)
    F = K.fields_from_record(M, wl.model.sigma_R)
    f = K.equilibrium_planes(F, wl.xi, wl.dim, wl.model)
    I = K.photon_equilibrium(F["T_R"], wl.omega.shape[0], wl.model.sigma_R)
    return F, f, I


def _K_g(model):
    A = mdl.mason_monchick_A(model.d_r, model.d_v, model.Z_r, model.Z_v, model.Sc)
    return np.sqrt(2.0 / np.pi) * model.Kn / 2.0 * np.ones(3) @ np.linalg.inv(A) @ np.diag(
        [5.0, model.d_r, model.d_v]) @ np.ones(3)


@pytest.mark.parametrize("order", [1, 2])
def test_uniform_equilibrium_is_a_macroscopic_fixed_point(order):
    wl = gi.workloads.with_solver(gi.workloads.slab(n_cells=8, T_left=1.0, T_right=1.0), order=order)
    faces = MA.Faces(K.Geometry(wl.mesh))
    F, f, I = _eq_state(wl, 1.0)
    Fk = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, 1, wl.model)
    hot = MA.high_order_terms(faces, Fk, MA.kinetic_boundary_flux(faces, f, I, wl), wl)
    assert np.abs(MA.residual(MA.conservative(F, 1, wl.model), faces, _zero_hot(faces, 1), wl)).max() < 1e-12
    assert np.abs(MA.residual(MA.conservative(Fk, 1, wl.model), faces, hot, wl)).max() < 1e-12

    wl = gi.workloads.with_solver(gi.workloads.cavity(n_side=6, u_lid=0.0, T_lid=1.0), order=order)
    faces = MA.Faces(K.Geometry(wl.mesh))
    F, f, I = _eq_state(wl, 1.0)
    Fk = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, 2, wl.model)
    qerr = max(np.abs(Fk["T_t"] - 1.0).max(), np.abs(Fk["rho"] - 1.0).max())
    assert 1e-8 < qerr < 1e-4
    hot = MA.high_order_terms(faces, Fk, MA.kinetic_boundary_flux(faces, f, I, wl), wl)
    assert np.abs(MA.residual(MA.conservative(Fk, 2, wl.model), faces, hot, wl)).max() < 20 * qerr


def test_conduction_closed_form():
    TL, TR = 1.0, 1.2
    wl = gi.workloads.with_model(gi.workloads.slab(n_cells=32, Kn=0.01, T_left=TL, T_right=TR), sigma_R=1e-12)
    wl = gi.workloads.with_solver(wl, order=2, max_inner=3000, tol_inner=1e-13, cfl_macro=1000)
    faces = MA.Faces(K.Geometry(wl.mesh))
    F, _, _ = _eq_state(wl, 1.1)
    hot = _zero_hot(faces, 1)
    W = MA.macro_solve(MA.conservative(F, 1, wl.model), faces, hot, wl)
    Fn = MA.fields_from_W(W, 1, wl.model)
    om = wl.model.omega
    x = wl.mesh.cell_centroid[:, 0]
    y = Fn["T_t"] ** (1 + om)
    mid = np.abs(x - 0.5) < 0.3
    slope, icpt = np.polyfit(x[mid], y[mid], 1)
    assert np.abs(y[mid] - (slope * x[mid] + icpt)).max() < 3e-4 * y.max()
    # temperature jumps at the walls are positive and small at Kn = 0.01
    assert 0.0 < Fn["T_t"][0] - TL < 0.02 and 0.0 < TR - Fn["T_t"][-1] < 0.02
    Fv = MA.viscous_flux(faces, MA.primitive(W, 1, wl.model), {k: v for k, v in hot.items() if k != "boundary"},
                         1, wl.model)
    fmid = np.abs(faces.xf[:, 0] - 0.5) < 0.25
    assert np.allclose(Fv[fmid, 2], -_K_g(wl.model) * slope / (1 + om), rtol=2e-3)
    # energy leaves through the hot wall as fast as it enters through the cold one
    bf = MA.macro_boundary_flux(faces, MA.primitive(W, 1, wl.model), wl)
    assert abs(bf[0, 2] + bf[1, 2]) < 1e-6 and np.abs(bf[:, 0]).max() < 1e-14


def _slab_run(n_cells, Kn, Kn_p, sigma_R, mode, iters, T_right=1.5, tol=1e-10, order=2):
    wl = gi.workloads.slab(n_cells=n_cells, Kn=Kn, Kn_p=Kn_p, sigma_R=sigma_R, T_right=T_right)
    wl = gi.workloads.with_solver(wl, order=order, relax_block=16, max_inner=200, n_cis_precond=3)
    F, f, I = _eq_state(wl, 1.25)
    h = []
    f, I, Fo, n = OG.solve(f, I, wl, mode=mode, max_iter=iters, tol=tol, history=h)
    return wl, Fo, h


def test_gsis_accelerates_a_near_continuum_slab_and_keeps_mass():
    wl, Fg, hg = _slab_run(32, 0.01, 1.0, 0.01, "gsis", 40, tol=1e-8)
    assert hg[-1] < 1e-8 and len(hg) <= 35
    _, Fc, hc = _slab_run(32, 0.01, 1.0, 0.01, "cis", 40, tol=1e-8)
    assert min(hc) > 1e-3
    # closed domain: GSIS iterations keep the mass reached after the CIS start
    _, F3, _ = _slab_run(32, 0.01, 1.0, 0.01, "cis", 3)
    vol = wl.mesh.cell_volume
    assert abs(np.sum(Fg["rho"] * vol) - np.sum(F3["rho"] * vol)) < 1e-12


def _kirchhoff(wl, x, TL=1.0, TR=1.5):
    m, om = wl.model, wl.model.omega
    Kg = _K_g(m)
    Phi = lambda T: Kg * T ** (1 + om) / (1 + om) + (4.0 / 3.0) * m.sigma_R * m.Kn_p * T ** 4
    target = Phi(TL) + (Phi(TR) - Phi(TL)) * x
    Tg = np.linspace(0.9 * TL, 1.1 * TR, 40001)
    return np.interp(target, Phi(Tg), Tg)


def test_asymptotic_preserving_slab():
    """Kn = Kn_p = 1e-3 on 16 cells (Delta x = 62 mean free paths): all temperatures
    equal, total temperature within the O(Delta x) error of the first-order wall faces of
    Kirchhoff's solution of q_gas + q_R = const; CIS after as many iterations is far off."""
    wl, Fg, hg = _slab_run(16, 1e-3, 1e-3, 0.01, "gsis", 60, tol=1e-8)
    assert hg[-1] < 1e-8
    x = wl.mesh.cell_centroid[:, 0]
    Tex = _kirchhoff(wl, x)
    err = np.abs(OG.total_temperature(Fg, wl.model) - Tex).max()
    assert err < 0.025
    assert max(np.abs(Fg[k] - Fg["T_t"]).max() for k in ("T_r", "T_v", "T_R")) < 1e-3
    _, Fc, _ = _slab_run(16, 1e-3, 1e-3, 0.01, "cis", 60)
    assert np.abs(OG.total_temperature(Fc, wl.model) - Tex).max() > 0.1


@pytest.mark.slow
def test_asymptotic_preserving_slab_refines_first_order():
    wl16, F16, _ = _slab_run(16, 1e-3, 1e-3, 0.01, "gsis", 60, tol=1e-8)
    wl32, F32, h32 = _slab_run(32, 1e-3, 1e-3, 0.01, "gsis", 60, tol=1e-8)
    e16 = np.abs(OG.total_temperature(F16, wl16.model) - _kirchhoff(wl16, wl16.mesh.cell_centroid[:, 0])).max()
    e32 = np.abs(OG.total_temperature(F32, wl32.model) - _kirchhoff(wl32, wl32.mesh.cell_centroid[:, 0])).max()
    assert e32 < 0.5 * e16


@pytest.mark.slow
def test_gsis_converges_on_the_heated_lid_cavity():
    wl = gi.workloads.with_solver(gi.workloads.cavity(n_side=8, Kn=0.01, Kn_p=10.0, T_lid=3.0, u_lid=0.18),
                                  precision="fp64", order=2, relax_block=16, max_inner=100, n_cis_precond=3)
    F, f, I = _eq_state(wl, 1.0)
    hg = []
    OG.solve(f, I, wl, mode="gsis", max_iter=30, tol=1e-6, history=hg)
    assert hg[-1] < 1e-6
