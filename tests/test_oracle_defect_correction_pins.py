"""Pins of the defect-corrected synthetic residual (an extension of the GSIS step, off by
default): R(W) - R(W^{k+1/2}) + r^{k+1/2}, with r the moments of the kinetic residual
(oracle/gsis.py ``kinetic_residual_rows``, ``gsis_step``)."""
import numpy as np

import gsis_inputs as gi
from oracle import gsis as OG
from oracle import kinetic as K
from oracle import macro as MA


def test_residual_rows_of_equilibrium_planes_are_the_conservative_variables():
    """Fed equilibrium planes and the photon equilibrium in place of a residual, the rows are
    the moments that define the conservative variables: rho, rho u, the total energy (with
    the hidden translational part from H0 and e_R), e_r, e_v, e_R."""
    for wl in (gi.workloads.slab(4), gi.workloads.cavity(n_side=2, n_v=24)):
        n = wl.mesh.n_cells
        M = gi.fields.smooth_random_fields(wl.mesh.cell_centroid, 3, u_scale=0.3)
        F = K.fields_from_record(M, wl.model.sigma_R)
        f = K.equilibrium_planes(F, wl.xi, wl.dim, wl.model)
        I = K.photon_equilibrium(F["T_R"], wl.omega.shape[0], wl.model.sigma_R)
        rows = OG.kinetic_residual_rows(f, I, wl)
        W = MA.conservative(K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, wl.dim, wl.model), wl.dim, wl.model)
        assert rows.shape == (n, MA.nvar(wl.dim))
        assert np.abs(rows - W).max() < 1e-12 * np.abs(W).max()


def _steady_slab(n=16, order=2):
    wl = gi.workloads.with_solver(gi.workloads.slab(n, Kn=0.1), precision="fp64", order=order, relax_block=16,
                                  max_inner=400, tol_inner=1e-12)
    M = gi.fields.uniform_fields(n, T=1.25)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 1, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 0,
                                       noise=0.0)
    geo = K.Geometry(wl.mesh)
    for _ in range(3000):
        f, I, e, F = OG.cis_step(f, I, wl, geo)
        if e < 1e-13:
            break
    assert e < 1e-13
    return wl, geo, f, I, F


def test_kinetic_steady_state_is_a_fixed_point_of_the_corrected_step():
    """From the kinetic steady state (CIS to eps < 1e-13) one GSIS step with the defect
    correction changes the fields by no more than rounding, while the paper's step moves
    them: its synthetic equations are consistent with the kinetic discretisation only to
    the discretisation error."""
    wl, geo, f, I, F = _steady_slab()
    faces = MA.Faces(geo)
    eps = {}
    for dc in (0, 1):
        w2 = gi.workloads.with_solver(wl, defect_correction=dc)
        eps[dc] = OG.gsis_step(f, I, w2, geo, faces, F)[2]
    assert eps[1] < 1e-10, eps
    assert eps[0] > 100 * max(eps[1], 1e-12), eps
