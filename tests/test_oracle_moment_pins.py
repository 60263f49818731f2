"""Pins of the oracle's moments of non-equilibrium distributions, of the far-field branch
of the macroscopic boundary flux and of the convergence measure.

* ``moments`` on a Grad-type distribution (a Maxwellian times the textbook 13-moment
  polynomial in the peculiar velocity) must return the stress and heat fluxes the
  polynomial was built with.  The reduced planes (F0, H0, f1, f2) are formed here by
  summing a full 3-D evaluation over the hidden velocity components, so the hidden-
  direction stress carried by H0 and the H0 term of q_t are both exercised.
* ``moments`` of the reference distribution g of a state with heat fluxes q must return
  q - A q: the heat-flux relaxation law that defines A (Section 2.1).
* the far-field branch of ``macro_boundary_flux`` at the free-stream state equals the
  exact Euler flux of that state, and its dissipative parts push in the physical
  direction (mass out of a denser cell, heat out of a hotter one, shear against the slip).
* ``epsilon`` (Section 6) on two cells with numbers worked out by hand.
"""
import numpy as np
import pytest

import gsis_inputs as gi
from gsis_inputs import quadrature as Q
from oracle import gsis as OG
from oracle import kinetic as K
from oracle import macro as MA
from oracle import model as mdl


def _grad13_planes(dim, n, L, states, d_r, d_v):
    """Reduced planes of f0 = rho M [1 + sigma:cc/(2 p T) + (q.c/(p T))(c^2/(5T) - 1)],
    f1 = (d_r/2) T_r rho M + (q_r.c/T) M, f2 likewise, M the unit Maxwellian at (u, T):
    evaluated on a 3-D trapezoid grid and summed over the 3 - dim hidden components."""
    xi3, w3 = Q.trapezoid_nd(n, L, 3)
    x1, w1 = Q.trapezoid_weights(n, L)
    out = []
    for (rho, u, T, Tr, Tv, sig, q, qr, qv) in states:
        c = xi3 - np.asarray(u)[None, :]
        c2 = np.sum(c * c, axis=1)
        M = (2 * np.pi * T) ** -1.5 * np.exp(-c2 / (2 * T))
        p = rho * T
        scc = np.einsum("va,ab,vb->v", c, sig, c)
        qc, qrc, qvc = c @ q, c @ qr, c @ qv
        f0 = rho * M * (1 + scc / (2 * p * T) + qc / (p * T) * (c2 / (5 * T) - 1))
        f1 = 0.5 * d_r * Tr * rho * M + qrc / T * M
        f2 = 0.5 * d_v * Tv * rho * M + qvc / T * M
        hid2 = np.sum(c[:, dim:] ** 2, axis=1)       # hidden components carry no flow velocity
        shape = (n ** dim, n ** (3 - dim))
        wh = np.ones(1)
        for _ in range(3 - dim):
            wh = np.outer(wh, w1).ravel()
        red = lambda a: a.reshape(shape) @ wh
        out.append(np.stack([red(f0), red(hid2 * f0), red(f1), red(f2)], axis=-1))
    xi, w = Q.trapezoid_nd(n, L, dim)
    return np.stack(out), xi, w


@pytest.mark.parametrize("dim", [1, 2])
def test_moments_of_grad_distribution_return_its_stress_and_heat_fluxes(dim):
    model = gi.workloads.ModelParams()
    rng = np.random.default_rng(31)
    states = []
    for _ in range(3):
        rho, T = rng.uniform(0.7, 1.4), rng.uniform(0.8, 1.4)
        u = np.zeros(3)
        u[:dim] = rng.uniform(-0.3, 0.3, dim)
        p = rho * T
        sig = np.zeros((3, 3))
        if dim == 2:
            sxx, syy, sxy = rng.uniform(-0.05, 0.05, 3) * p
            sig[0, 0], sig[1, 1], sig[0, 1] = sxx, syy, sxy
            sig[1, 0] = sxy
            sig[2, 2] = -(sxx + syy)                  # traceless, hidden zz carried by H0
        else:
            sxx = rng.uniform(-0.05, 0.05) * p
            sig[0, 0], sig[1, 1], sig[2, 2] = sxx, -sxx / 2, -sxx / 2
        q, qr, qv = (np.zeros(3) for _ in range(3))
        amp = 0.05 * p * np.sqrt(T)
        q[:dim], qr[:dim], qv[:dim] = (rng.uniform(-1, 1, dim) * amp for _ in range(3))
        states.append((rho, u, T, rng.uniform(0.8, 1.4), rng.uniform(0.8, 1.4), sig, q, qr, qv))
    f, xi, w = _grad13_planes(dim, 40, 10.0, states, model.d_r, model.d_v)
    om, wo = Q.photon_product(4, 4)
    G = K.moments(f, np.zeros((len(states), om.shape[0])), xi, w, om, wo, dim, model)
    for k, (rho, u, T, Tr, Tv, sig, q, qr, qv) in enumerate(states):
        assert abs(G["rho"][k] - rho) < 1e-12
        assert np.allclose(G["u"][k], u, atol=1e-12)
        assert abs(G["T_t"][k] - T) < 1e-12
        assert abs(G["T_r"][k] - Tr) < 1e-12 and abs(G["T_v"][k] - Tv) < 1e-12
        assert np.allclose(G["sigma"][k], sig, atol=1e-12)
        assert np.allclose(G["q_t"][k], q, atol=1e-12)
        assert np.allclose(G["q_r"][k], qr, atol=1e-12)
        assert np.allclose(G["q_v"][k], qv, atol=1e-12)


@pytest.mark.parametrize("dim", [1, 2])
def test_moments_of_reference_distribution_follow_the_heat_flux_relaxation_law(dim):
    """int c (c^2/2) g0 (with H0) = q_t - (A q)_t etc.: dq/dt = -(p/mu) A q (Section 2.1),
    computed through ``moments`` itself."""
    model = gi.workloads.ModelParams()
    xi, w = Q.trapezoid_nd(64, 13.0, dim)
    M = gi.fields.random_macro_fields(4, dim, seed=32, u_scale=0.4, q_scale=0.1)
    F = K.fields_from_record(M, model.sigma_R)
    g = K.reference_planes(F, xi, dim, model)
    om, wo = Q.photon_product(4, 4)
    G = K.moments(g, np.zeros((4, om.shape[0])), xi, w, om, wo, dim, model)
    A = mdl.mason_monchick_A(model.d_r, model.d_v, model.Z_r, model.Z_v, model.Sc)
    q = np.stack([F["q_t"], F["q_r"], F["q_v"]], 1)
    expect = q - np.einsum("ij,njd->nid", A, q)
    assert np.allclose(G["u"], F["u"], atol=1e-11)
    for m, key in enumerate(("q_t", "q_r", "q_v")):
        assert np.abs(expect[:, m, :dim]).max() > 1e-3                 # not trivially zero
        assert np.allclose(G[key][:, :dim], expect[:, m, :dim], rtol=1e-9, atol=1e-11)


def _cyl():
    wl = gi.workloads.cylinder(n_theta=24, n_radial=3, n_v=16, n_polar=4, n_azim=4)
    faces = MA.Faces(K.Geometry(wl.mesh))
    far = [p for p in wl.mesh.patches if p.kind == K.FARFIELD][0]
    isfar = np.array([wl.mesh.patches[p].kind == K.FARFIELD for p in faces.bf_patch])
    return wl, faces, far, isfar


def _state(wl, far, rho=None, u=None, T=None):
    nc = wl.mesh.n_cells
    rho = np.full(nc, far.rho if rho is None else rho)
    uu = np.tile(np.asarray(far.u, float)[:2] if u is None else np.asarray(u, float), (nc, 1))
    T = far.T_t if T is None else T
    Tt, Tr, Tv = (np.full(nc, x) for x in (T, T, T))
    eR = np.full(nc, 4.0 * wl.model.sigma_R * far.T_R ** 4)
    return (rho, uu, Tt, Tr, Tv, eR)


def test_far_field_flux_at_the_free_stream_is_the_euler_flux():
    wl, faces, far, isfar = _cyl()
    out = MA.macro_boundary_flux(faces, _state(wl, far), wl)
    m = wl.model
    u = np.asarray(far.u, float)[:2]
    rho, T = far.rho, far.T_t
    p = rho * T
    E_gas = rho * (1.5 * T + 0.5 * u @ u + 0.5 * m.d_r * T + 0.5 * m.d_v * T)
    for b in np.nonzero(isfar)[0]:
        n = faces.bf_n[b]
        un = u @ n
        euler = np.concatenate([[rho * un], rho * u * un + p * n,
                                [un * (E_gas + p), un * 0.5 * m.d_r * rho * T, un * 0.5 * m.d_v * rho * T, 0.0]])
        assert np.allclose(out[b], euler, rtol=1e-13, atol=1e-13)


def test_far_field_flux_dissipation_points_the_physical_way():
    wl, faces, far, isfar = _cyl()
    base = MA.macro_boundary_flux(faces, _state(wl, far), wl)
    dense = MA.macro_boundary_flux(faces, _state(wl, far, rho=1.2 * far.rho), wl)
    hot = MA.macro_boundary_flux(faces, _state(wl, far, T=1.3 * far.T_t), wl)
    E = 3
    uf = np.asarray(far.u, float)[:2]
    cs = np.sqrt(5.0 * far.T_t / 3.0)
    sub = [b for b in np.nonzero(isfar)[0] if abs(uf @ faces.bf_n[b]) < cs]
    assert len(sub) >= 2
    for b in np.nonzero(isfar)[0]:
        # the cell moves with the free stream: a denser cell pushes more mass out, on
        # inflow faces too (the dissipation outweighs the convective change)
        assert dense[b, 0] > base[b, 0] + 1e-3
    for b in sub:
        # where the normal flow is subsonic, a hotter cell loses energy and internal
        # energy (convective, dissipative and conductive parts); on supersonic inflow
        # faces the convective inflow of the hotter state outweighs the dissipation
        assert hot[b, E] > base[b, E] + 1e-3 and hot[b, E + 1] > base[b, E + 1] and hot[b, E + 2] > base[b, E + 2]
    # tangential slip: the cell moves faster along the face than the free stream, so the
    # viscous stress carries that momentum out (the mass flux is the same for both)
    for b in np.nonzero(isfar)[0][:4]:
        n = faces.bf_n[b]
        t = np.array([-n[1], n[0]])
        slip = MA.macro_boundary_flux(faces, _state(wl, far, u=uf + 0.2 * t), wl)[b]
        ref = MA.macro_boundary_flux(faces, _state(wl, far, u=uf), wl)[b]
        # remove the convective change: Rusanov of the slipping state against the far field
        conv = MA.rusanov(tuple(x[:1] for x in _state(wl, far, u=uf + 0.2 * t)),
                          tuple(x[:1] for x in _state(wl, far, u=uf)), n[None], 2, wl.model)[0]
        conv0 = MA.rusanov(tuple(x[:1] for x in _state(wl, far, u=uf)),
                           tuple(x[:1] for x in _state(wl, far, u=uf)), n[None], 2, wl.model)[0]
        visc = (slip - conv) - (ref - conv0)
        assert visc[1:3] @ t > 1e-3


def test_epsilon_on_two_cells_by_hand():
    model = gi.workloads.ModelParams()          # d_r = 2, d_v = 1.16
    vol = np.array([1.0, 3.0])

    def F(rho, ux, Tt, Tr, Tv):
        G = K.empty_fields(2)
        G["rho"], G["T_t"], G["T_r"], G["T_v"] = (np.array(x, float) for x in (rho, Tt, Tr, Tv))
        G["u"][:, 0] = ux
        return G

    old = F([1.0, 2.0], [0.1, 0.2], [1.0, 1.0], [1.0, 1.0], [1.0, 1.0])
    # velocity term dominates: |du| = (0, 0.1) -> sqrt(0.01 * 3) = 0.1732051;
    # ||u_old|| = sqrt(0.01 * 1 + 0.04 * 3) = 0.3605551; ratio 0.4803845
    new = F([1.1, 2.0], [0.1, 0.3], [1.0, 1.0], [1.0, 1.0], [1.0, 1.0])
    assert abs(OG.epsilon(new, old, vol, model, 1) - 0.17320508075688773 / 0.36055512754639896) < 1e-14
    # temperature term: the total T of cell 1 becomes (3 * 1 + 2 * 1.5 + 1.16 * 1) / 6.16
    # = 7.16 / 6.16; ||dT|| = sqrt(3) (1/6.16... ) -> sqrt(3) * 1.0 / 6.16; ||T_old|| = 2
    new = F([1.0, 2.0], [0.1, 0.2], [1.0, 1.0], [1.0, 1.5], [1.0, 1.0])
    assert abs(OG.epsilon(new, old, vol, model, 1) - np.sqrt(3.0) / 6.16 / 2.0) < 1e-14
    # density term: ||drho|| = 0.1; ||rho_old|| = sqrt(1 + 4 * 3) = sqrt(13)
    new = F([1.1, 2.0], [0.1, 0.2], [1.0, 1.0], [1.0, 1.0], [1.0, 1.0])
    assert abs(OG.epsilon(new, old, vol, model, 1) - 0.1 / np.sqrt(13.0)) < 1e-14
    # no mean flow: the velocity denominator is floored at 0.01 ||sqrt(T_old)|| = 0.01 * 2
    rest = F([1.0, 2.0], [0.0, 0.0], [1.0, 1.0], [1.0, 1.0], [1.0, 1.0])
    moved = F([1.0, 2.0], [0.001, 0.0], [1.0, 1.0], [1.0, 1.0], [1.0, 1.0])
    assert abs(OG.epsilon(moved, rest, vol, model, 1) - 0.001 / 0.02) < 1e-14
    # only the in-plane components count: a change of u_y in a 1-D problem is ignored
    side = F([1.0, 2.0], [0.1, 0.2], [1.0, 1.0], [1.0, 1.0], [1.0, 1.0])
    side["u"][:, 1] = 5.0
    assert OG.epsilon(side, old, vol, model, 1) == 0.0
