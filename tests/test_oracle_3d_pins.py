"""Pins of the oracle on 3-D tetrahedral meshes (the capsule case of Section 6 in three
dimensions: f0, f1, f2 over the full velocity space, no hidden components).

* the tetrahedral box and capsule meshes are closed (sum of S n over every cell's faces
  is zero), their normals are unit and point out of the owner, and the volumes add up
  to the unit cube less the body;
* the least-squares weights differentiate linear fields exactly on tetrahedra;
* ``moments`` of a 3-D Grad-type distribution returns the full stress tensor and heat
  fluxes it was built with, and ``moments`` of the reference distribution follows the
  heat-flux relaxation law q -> q - A q in all three components;
* a uniform equilibrium at the walls' state (symmetric Gauss-Hermite grid, so the wall
  re-emission balances exactly) and a uniform free stream matching the far field are
  fixed points of the 3-D sweep at orders 1 and 2;
* the sweep commutes with a cyclic permutation of the coordinate axes (mesh, velocities,
  flow and wall velocity permuted together): no axis is treated differently.
"""
import numpy as np
import pytest

import gsis_inputs as gi
from gsis_inputs import quadrature as Q
from oracle import kinetic as K
from oracle import model as mdl


def _closure(m):
    acc = np.zeros((m.n_cells, m.dim))
    np.add.at(acc, m.face_owner, m.face_normal * m.face_area[:, None])
    inner = m.face_nbr >= 0
    np.add.at(acc, m.face_nbr[inner], -m.face_normal[inner] * m.face_area[inner, None])
    return np.abs(acc).max()


@pytest.mark.parametrize("mk", [lambda: gi.mesh.box_tetrahedra(5, seed=4), lambda: gi.mesh.capsule_tetrahedra(8)])
def test_tetrahedral_meshes_are_closed_and_oriented(mk):
    m = mk()
    assert _closure(m) < 1e-15
    assert np.allclose(np.linalg.norm(m.face_normal, axis=1), 1.0, atol=1e-14)
    out = np.einsum("fd,fd->f", m.face_normal, m.face_centroid - m.cell_centroid[m.face_owner])
    assert out.min() > 0.0
    inner = m.face_nbr >= 0
    into = np.einsum("fd,fd->f", m.face_normal[inner], m.cell_centroid[m.face_nbr[inner]] - m.face_centroid[inner])
    assert into.min() > 0.0
    # every cell has four faces
    cnt = np.bincount(m.face_owner, minlength=m.n_cells) + np.bincount(m.face_nbr[inner], minlength=m.n_cells)
    assert np.all(cnt == 4)


def test_box_volume_and_capsule_body():
    assert abs(gi.mesh.box_tetrahedra(4, seed=1).cell_volume.sum() - 1.0) < 1e-13
    m = gi.mesh.capsule_tetrahedra(16)
    box = gi.mesh.box_tetrahedra(16, seed=2)
    # the dropped cells are those whose centroids lie in the body; the exposed faces are
    # the body's patch (0) and the cube's sides its far field (1)
    assert box.n_cells - m.n_cells > 0
    assert abs(m.cell_volume.sum() + (box.cell_volume.sum() - m.cell_volume.sum()) - 1.0) < 1e-13
    assert set(np.unique(m.face_nbr[m.face_nbr < 0])) == {-1, -2}
    wall = m.face_nbr == -1
    xc = m.face_centroid[wall]
    r = np.hypot(xc[:, 1] - 0.5, xc[:, 2] - 0.5)
    assert xc[:, 0].min() > 0.25 and xc[:, 0].max() < 0.6 and r.max() < 0.25
    # the body is the sphere-cone: every dropped cell's centroid lies inside its profile
    inside = np.hypot(box.cell_centroid[:, 1] - 0.5, box.cell_centroid[:, 2] - 0.5) <= \
        gi.mesh.sphere_cone_radius(box.cell_centroid[:, 0])
    assert int(inside.sum()) == box.n_cells - m.n_cells
    far = m.face_nbr == -2
    assert np.all(np.min(np.minimum(m.face_centroid[far], 1.0 - m.face_centroid[far]), axis=1) < 1e-12)


def test_lsq_gradient_exact_for_linear_fields_on_tetrahedra():
    m = gi.mesh.box_tetrahedra(3, seed=3)
    geo = K.Geometry(m)
    g = np.array([1.7, -0.9, 0.4])
    q = 0.3 + m.cell_centroid @ g
    n_checked = 0
    for i in range(m.n_cells):
        if len(geo.lsq[i][0]) >= 3:
            grad, _ = K.limited_slope(geo, i, q, 5.0)
            assert np.allclose(grad, g, atol=1e-12)
            n_checked += 1
    assert n_checked == m.n_cells


def test_moments_of_3d_grad_distribution():
    """f0 = rho M [1 + sigma:cc/(2 p T) + (q.c/(p T))(c^2/(5T) - 1)], f1, f2 with their own
    heat fluxes, on a 3-D trapezoid grid: every stress and heat-flux component returns."""
    model = gi.workloads.ModelParams()
    rng = np.random.default_rng(41)
    xi, w = Q.trapezoid_nd(36, 9.0, 3)
    n = 3
    f = np.zeros((n, xi.shape[0], 4))
    want = []
    for k in range(n):
        rho, T, Tr, Tv = rng.uniform(0.7, 1.4), rng.uniform(0.8, 1.3), rng.uniform(0.8, 1.4), rng.uniform(0.8, 1.4)
        u = rng.uniform(-0.3, 0.3, 3)
        p = rho * T
        S = rng.uniform(-0.05, 0.05, (3, 3)) * p
        sig = 0.5 * (S + S.T)
        sig -= np.trace(sig) / 3.0 * np.eye(3)
        q, qr, qv = (rng.uniform(-1, 1, 3) * 0.05 * p * np.sqrt(T) for _ in range(3))
        c = xi - u[None]
        c2 = np.sum(c * c, axis=1)
        M = (2 * np.pi * T) ** -1.5 * np.exp(-c2 / (2 * T))
        f[k, :, 0] = rho * M * (1 + np.einsum("va,ab,vb->v", c, sig, c) / (2 * p * T)
                                + (c @ q) / (p * T) * (c2 / (5 * T) - 1))
        f[k, :, 2] = 0.5 * model.d_r * Tr * rho * M + (c @ qr) / T * M
        f[k, :, 3] = 0.5 * model.d_v * Tv * rho * M + (c @ qv) / T * M
        want.append((rho, u, T, Tr, Tv, sig, q, qr, qv))
    om, wo = Q.photon_product(4, 4)
    G = K.moments(f, np.zeros((n, om.shape[0])), xi, w, om, wo, 3, model)
    for k, (rho, u, T, Tr, Tv, sig, q, qr, qv) in enumerate(want):
        assert abs(G["rho"][k] - rho) < 1e-12
        assert np.allclose(G["u"][k], u, atol=1e-12)
        assert abs(G["T_t"][k] - T) < 1e-12
        assert abs(G["T_r"][k] - Tr) < 1e-12 and abs(G["T_v"][k] - Tv) < 1e-12
        assert np.allclose(G["sigma"][k], sig, atol=1e-12)
        assert np.allclose(G["q_t"][k], q, atol=1e-12)
        assert np.allclose(G["q_r"][k], qr, atol=1e-12)
        assert np.allclose(G["q_v"][k], qv, atol=1e-12)


def test_3d_reference_distribution_follows_the_heat_flux_relaxation_law():
    model = gi.workloads.ModelParams()
    xi, w = Q.trapezoid_nd(56, 14.0, 3)       # truncation and spacing errors below 1e-12
    M = gi.fields.random_macro_fields(3, 3, seed=42, u_scale=0.4, q_scale=0.1)
    F = K.fields_from_record(M, model.sigma_R)
    g = K.reference_planes(F, xi, 3, model)
    assert np.abs(g[..., 1]).max() == 0.0                       # no hidden components
    om, wo = Q.photon_product(4, 4)
    G = K.moments(g, np.zeros((3, om.shape[0])), xi, w, om, wo, 3, model)
    A = mdl.mason_monchick_A(model.d_r, model.d_v, model.Z_r, model.Z_v, model.Sc)
    q = np.stack([F["q_t"], F["q_r"], F["q_v"]], 1)
    expect = q - np.einsum("ij,njd->nid", A, q)
    assert np.allclose(G["rho"], F["rho"], rtol=1e-11) and np.allclose(G["u"], F["u"], atol=1e-11)
    for m, key in enumerate(("q_t", "q_r", "q_v")):
        assert np.abs(expect[:, m, 2]).max() > 1e-3              # the z components are exercised
        assert np.allclose(G[key], expect[:, m], rtol=1e-9, atol=1e-11)


def _box_workload(order, patches, n_gh=8):
    m = gi.mesh.box_tetrahedra(2, seed=6, patches=patches)
    r = Q.gauss_hermite_1d(n_gh)
    xi, w = Q.tensor_grid([r, r, r])
    om, wo = Q.photon_product(2, 4)
    wl = gi.workloads.Workload("box", m, xi, w, om, wo, gi.workloads.ModelParams(Kn=0.3, Kn_p=2.0))
    return gi.workloads.with_solver(wl, order=order, precision="fp64")


@pytest.mark.parametrize("order", [1, 2])
def test_uniform_wall_equilibrium_is_a_fixed_point_in_3d(order):
    T = 1.0        # the Gauss-Hermite weight itself: the moments are exact
    wl = _box_workload(order, [gi.mesh.Patch(gi.mesh.WALL, T_t=T) for _ in range(6)])
    Mf = gi.fields.uniform_fields(wl.mesh.n_cells, rho=0.9, T=T)
    F = K.fields_from_record(Mf, wl.model.sigma_R)
    f = K.equilibrium_planes(F, wl.xi, 3, wl.model)
    I = K.photon_equilibrium(F["T_R"], wl.omega.shape[0], wl.model.sigma_R)
    fn, In = K.kinetic_sweep(f, I, wl, relax_block=8)
    assert np.abs(fn - f).max() < 1e-13 * np.abs(f).max()
    assert np.abs(In - I).max() < 1e-13 * np.abs(I).max()


@pytest.mark.parametrize("order", [1, 2])
def test_uniform_free_stream_is_a_fixed_point_in_3d(order):
    u = (0.7, -0.4, 0.5)
    far = gi.mesh.Patch(gi.mesh.FARFIELD, rho=1.3, u=u, T_t=1.1, T_r=1.1, T_v=1.1, T_R=1.1)
    # collisionless: what is left is transport, exact whatever the quadrature
    wl = gi.workloads.with_model(_box_workload(order, [far] * 6), Kn=1e12, Kn_p=1e12)
    Mf = gi.fields.uniform_fields(wl.mesh.n_cells, rho=1.3, u=u, T=1.1)
    F = K.fields_from_record(Mf, wl.model.sigma_R)
    f = K.equilibrium_planes(F, wl.xi, 3, wl.model)
    I = K.photon_equilibrium(F["T_R"], wl.omega.shape[0], wl.model.sigma_R)
    G = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, 3, wl.model)
    fn, In = K.kinetic_sweep(f, I, wl, relax_block=8, F=G)
    assert np.abs(fn - f).max() < 1e-13 * np.abs(f).max()
    assert np.abs(In - I).max() < 1e-13 * np.abs(I).max()


def test_sweep_commutes_with_a_cyclic_permutation_of_the_axes():
    perm = [1, 2, 0]                                           # new axis a is old axis perm[a]
    lid = gi.mesh.Patch(gi.mesh.WALL, u=(0.3, -0.2, 0.25), T_t=1.6)
    pats = [gi.mesh.Patch(gi.mesh.WALL, T_t=1.0) for _ in range(5)] + [lid]
    wl = _box_workload(2, pats, n_gh=6)
    Mf = gi.fields.random_macro_fields(wl.mesh.n_cells, 3, seed=43, u_scale=0.3, q_scale=0.05)
    f, I = gi.fields.noisy_equilibrium(Mf, wl.xi, wl.omega, 3, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 44)
    fn, In = K.kinetic_sweep(f, I, wl, relax_block=8)

    m = wl.mesh
    mp = gi.mesh.Mesh(dim=3, n_cells=m.n_cells, face_owner=m.face_owner, face_nbr=m.face_nbr,
                      face_normal=m.face_normal[:, perm], face_area=m.face_area,
                      face_centroid=m.face_centroid[:, perm], cell_volume=m.cell_volume,
                      cell_centroid=m.cell_centroid[:, perm],
                      patches=[gi.mesh.Patch(p.kind, rho=p.rho, u=tuple(np.asarray(p.u)[perm]), T_t=p.T_t,
                                             T_r=p.T_r, T_v=p.T_v, T_R=p.T_R) for p in m.patches])
    wlp = gi.workloads.Workload("box_p", mp, wl.xi[:, perm], wl.w, wl.omega[:, perm], wl.wo, wl.model, wl.solver)
    fp, Ip = K.kinetic_sweep(f, I, wlp, relax_block=8)
    assert np.abs(fp - fn).max() < 1e-12 * np.abs(fn).max()
    assert np.abs(Ip - In).max() < 1e-12 * np.abs(In).max()
    F = K.moments(fn, In, wl.xi, wl.w, wl.omega, wl.wo, 3, wl.model)
    Fp = K.moments(fp, Ip, wlp.xi, wlp.w, wlp.omega, wlp.wo, 3, wl.model)
    assert np.allclose(Fp["u"], F["u"][:, perm], atol=1e-12)
    assert np.allclose(Fp["q_t"], F["q_t"][:, perm], atol=1e-12)
    assert np.allclose(Fp["sigma"], F["sigma"][:, perm][:, :, perm], atol=1e-12)
