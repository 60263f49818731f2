"""Pins of the oracle's mirror-plane (SYMMETRY) boundary: specular reflection of molecules
and photons.

* the reflection maps every velocity and direction of the symmetric grids onto its mirror
  image;
* the kinetic flux through a mirror face carries no mass and no energy for any
  distribution, and its momentum flux is normal to the face;
* the synthetic equations' mirror flux carries no mass or energy, and at rest only the
  pressure;
* mirror symmetry: a slab between two equal walls, converged, equals on its left half the
  half slab that ends in a mirror plane, converged (first order, where the mirror face's
  upwind flux is exactly the interior face's); GSIS on the half slab converges to the same
  state.
"""
import dataclasses

import numpy as np

import gsis_inputs as gi
from gsis_inputs import mesh as GM
from gsis_inputs import quadrature as Q
from oracle import gsis as OG
from oracle import kinetic as K
from oracle import macro as MA


def test_reflection_maps_the_grids_onto_their_mirror_images():
    for xi in (Q.gauss_hermite_1d(32)[0], Q.trapezoid_nd(28, 6.0, 2)[0]):
        d = xi.shape[1]
        for a in range(d):
            n = np.zeros(d)
            n[a] = 1.0 if a == 0 else -1.0
            idx = K.reflection_index(xi, n)
            img = xi.copy()
            img[:, a] = -img[:, a]
            assert np.allclose(xi[idx], img, atol=1e-12)
            assert np.array_equal(idx[idx], np.arange(xi.shape[0]))        # an involution
    om, _ = Q.photon_product(8, 8)
    for n in (np.array([1.0, 0.0, 0.0]), np.array([0.0, -1.0, 0.0])):
        idx = K.reflection_index(om, n)
        img = om - 2.0 * (om @ n)[:, None] * n[None]
        assert np.allclose(om[idx], img, atol=1e-12)                  # Omega_z is kept


def _half_slab(n=8, T_wall=1.5, **kw):
    wl = gi.workloads.slab(2 * n, T_left=T_wall, T_right=T_wall, **kw)
    m = GM.slab_1d(n, 0.5, patches=[GM.Patch(GM.WALL, T_t=T_wall), GM.Patch(GM.SYMMETRY)])
    return dataclasses.replace(wl, mesh=m, name="halfslab%d" % n)


def test_mirror_face_flux_carries_no_mass_or_energy():
    wl = gi.workloads.with_solver(_half_slab(), order=1)
    rng = np.random.default_rng(4)
    M = gi.fields.random_macro_fields(8, 1, seed=5, u_scale=0.3)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 1, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 6)
    faces = MA.Faces(K.Geometry(wl.mesh))
    kb = MA.kinetic_boundary_flux(faces, f, I, wl)
    b = 1                                             # the mirror face (patch 1)
    assert wl.mesh.patches[faces.bf_patch[b]].kind == K.SYMMETRY
    scale = np.abs(kb).max()
    assert abs(kb[b, 0]) < 1e-14 * scale               # mass
    assert abs(kb[b, 2]) < 1e-14 * scale               # total energy (gas and photons)
    assert abs(kb[b, 3]) < 1e-14 * scale and abs(kb[b, 4]) < 1e-14 * scale and abs(kb[b, 5]) < 1e-14 * scale
    assert kb[b, 1] > 0.1 * scale                      # the normal momentum flux (pressure)
    # synthetic equations: a cell at rest pushes only its pressure through the mirror
    F = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, 1, wl.model)
    F["u"][:] = 0.0
    prim = MA.primitive(MA.conservative(F, 1, wl.model), 1, wl.model)
    mb = MA.macro_boundary_flux(faces, prim, wl)
    c = faces.bf_cell[b]
    assert abs(mb[b, 0]) < 1e-15 and np.abs(mb[b, 2:]).max() < 1e-15
    assert abs(mb[b, 1] - F["rho"][c] * F["T_t"][c]) < 1e-13
    assert rng is not None


def _start(wl):
    M = gi.fields.uniform_fields(wl.mesh.n_cells, T=1.0)
    F = K.fields_from_record(M, wl.model.sigma_R)
    return K.equilibrium_planes(F, wl.xi, 1, wl.model), K.photon_equilibrium(F["T_R"], wl.omega.shape[0],
                                                                             wl.model.sigma_R)


def test_mirror_plane_reproduces_the_symmetric_slab():
    """With Jacobi relaxation (every cell updated from the previous iterate) the iterates of
    the full slab stay mirror-symmetric, and the mirror face of the half slab receives at
    each step exactly what the full slab's middle face receives: the two trajectories agree
    step by step.  (The steady state of a closed domain is fixed only up to its total mass,
    which other orderings reach along different paths.)"""
    kw = dict(Kn=0.3, Kn_p=1.0)
    full = gi.workloads.with_solver(gi.workloads.slab(16, T_left=1.5, T_right=1.5, **kw), order=1, relax_block=1)
    half = gi.workloads.with_solver(_half_slab(8, **kw), order=1, relax_block=1)
    ff, If = _start(full)
    fh, Ih = _start(half)
    gf, gh = K.Geometry(full.mesh), K.Geometry(half.mesh)
    for k in range(20):
        ff, If, ef, _ = OG.cis_step(ff, If, full, gf)
        fh, Ih, eh, _ = OG.cis_step(fh, Ih, half, gh)
        assert np.isfinite(ef) and abs(ef - eh) < 1e-12 * ef
    assert np.abs(ff[8:] - ff[7::-1][:, ::-1]).max() < 1e-12 * np.abs(ff).max()     # the full slab stays symmetric
    assert np.abs(fh - ff[:8]).max() < 1e-12 * np.abs(ff).max()
    assert np.abs(Ih - If[:8]).max() < 1e-12 * np.abs(If).max()


def test_gsis_converges_with_a_mirror_plane():
    half = gi.workloads.with_solver(_half_slab(8, Kn=0.05, Kn_p=1.0), order=2, relax_block=16, n_cis_precond=3,
                                    max_inner=200)
    f, I = _start(half)
    h = []
    f, I, F, n = OG.solve(f, I, half, mode="gsis", max_iter=80, tol=1e-9, history=h)
    assert h[-1] < 1e-9
    # no mass leaves through the wall or the mirror
    assert abs(np.sum(F["rho"] * half.mesh.cell_volume) - 0.5) < 0.05
