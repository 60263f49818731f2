"""Pins of the oracle's positivity bound on the implicit update (an extension: the
solver's ``positivity`` theta keeps every value at least theta times its previous value).

* it leaves steady states alone: the exact fixed points of the sweep stay exact;
* where it acts, the result is exactly theta times the previous value, and it acts only
  where the unbounded update falls below that;
* theta = 0 is the paper's scheme, value for value.
"""
import numpy as np

import gsis_inputs as gi
from gsis_inputs import quadrature as Q
from oracle import kinetic as K


def _box(theta, order=2):
    m = gi.mesh.box_tetrahedra(2, seed=6, patches=[gi.mesh.Patch(gi.mesh.WALL, T_t=1.0) for _ in range(6)])
    r = Q.gauss_hermite_1d(8)
    xi, w = Q.tensor_grid([r, r, r])
    om, wo = Q.photon_product(2, 4)
    wl = gi.workloads.Workload("box", m, xi, w, om, wo, gi.workloads.ModelParams(Kn=0.3, Kn_p=2.0))
    return gi.workloads.with_solver(wl, order=order, precision="fp64", positivity=theta)


def test_bound_keeps_the_equilibrium_fixed_point():
    wl = _box(0.5)
    F = K.fields_from_record(gi.fields.uniform_fields(wl.mesh.n_cells, rho=0.9, T=1.0), wl.model.sigma_R)
    f = K.equilibrium_planes(F, wl.xi, 3, wl.model)
    I = K.photon_equilibrium(F["T_R"], wl.omega.shape[0], wl.model.sigma_R)
    fn, In = K.kinetic_sweep(f, I, wl, relax_block=8)
    assert np.abs(fn - f).max() < 1e-13 * np.abs(f).max()
    assert np.abs(In - I).max() < 1e-13 * np.abs(I).max()


def test_bound_acts_exactly_where_the_update_falls_below_it():
    wl = gi.workloads.with_solver(gi.workloads.cylinder(n_theta=8, n_radial=4, n_v=16, n_polar=4, n_azim=8),
                                  precision="fp64", order=2, relax_block=16, venkat_K=0.01)
    far = wl.mesh.patches[1]
    F = K.fields_from_record(gi.fields.uniform_fields(wl.mesh.n_cells, rho=far.rho, u=far.u, T=far.T_t),
                             wl.model.sigma_R)
    f = K.equilibrium_planes(F, wl.xi, 2, wl.model)
    I = K.photon_equilibrium(F["T_R"], wl.omega.shape[0], wl.model.sigma_R)
    G = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, 2, wl.model)      # the fields the solver takes
    fu, Iu = K.kinetic_sweep(f, I, wl, relax_block=16, F=G)
    theta = 0.25
    fb, Ib = K.kinetic_sweep(f, I, gi.workloads.with_solver(wl, positivity=theta), relax_block=16, F=G)
    low = fu < theta * f
    assert low.mean() > 0.1                                       # the impulsive start needs it
    assert np.array_equal(fb[low], theta * f[low])
    assert np.array_equal(fb[~low], fu[~low])
    assert np.all(fb >= theta * f) and np.all(Ib >= theta * I)
    assert np.array_equal(K.kinetic_sweep(f, I, gi.workloads.with_solver(wl, positivity=0.0), relax_block=16,
                                          F=G)[0], fu)
