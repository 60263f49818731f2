"""Oracle (test infrastructure only): the macroscopic synthetic equations in FP64.

Restates
  * Eq. (macroscopic_equation) with the energy components of Section 2.2;
  * the NSF constitutive relations, Eqs. (NSF_constitutive) and
    (NSF_thermal_conductivities), and the split into NSF part and high-order
    terms, Eqs. (split_constitutive), (getHoTs);
  * the implicit incremental form, Eq. (delta_macro), with the flux increment
    1/2 [dF_j + Gamma_ij (dW_i - dW_j)] and Gamma_ij = |u_n| + c_s + 2 mu/(rho |n.(x_j - x_i)|)
    (Section 5), the diagonal source Jacobian of Appendix A, and point relaxation.

Readings (the paper leaves these open):
  * numerical flux: Rusanov, 1/2 (F(W_L) + F(W_R)) - 1/2 lambda (W_R - W_L) with
    lambda = max(|u_n| + c_s); the dissipation acts on rho, rho u, the gas part of the
    total energy, e_r and e_v, not on e_R, which has no convective flux;
  * face states: limited linear reconstruction of (rho, u, T_t, T_r, T_v, e_R) with the
    least-squares stencil and limiter of the kinetic sweep;
  * face gradients: the average of the two cells' least-squares gradients, with its
    component along x_j - x_i replaced by the difference quotient;
  * high-order terms live on faces: HoT_f = average of the two cells' kinetic stress and
    heat fluxes minus the NSF flux of the kinetic-step state with the same face gradient,
    so the macroscopic viscous flux NSF_f(M) + HoT_f equals the kinetic one at a fixed
    point with the identical discrete operator (the asymptotic-preserving requirement of
    Section 4);
  * boundary faces: a macroscopic boundary flux that responds to the adjacent cell plus a
    boundary high-order term, the kinetic boundary flux of the kinetic step minus that
    macroscopic flux at the kinetic-step state, fixed during the inner iterations.  Walls:
    the flux of an equilibrium at the cell state leaving against the diffuse (black) wall,
    on the same discrete velocity and direction sets, so that the boundary term only
    carries the non-equilibrium part of the kinetic flux and stays small before
    convergence as well; far field: Rusanov and NSF against the far-field state;
  * the implicit operator takes the exact local Jacobian of the sources in the energy rows
    (e_gas, e_r, e_v, e_R; tau and k_eff frozen) as a 4x4 block instead of the diagonal of
    Appendix A: the gas-photon exchange couples e_v and e_R with rate k_eff, far too stiff
    for a diagonal treatment when k_eff = 1/Kn_photon is large;
  * the point relaxation updates the gas energy e_gas = e - e_R in place of the total
    energy (the total-energy equation minus the e_R equation), so that photon diffusion
    only enters the e_R row, whose Gamma adds 2 kappa_R / |n.(x_j - x_i)|; dW_e =
    dW_egas + dW_eR afterwards;
  * D_i = 1/dt + (1/V_i) sum_faces Gamma S - diag(dQ/dW) and the off-diagonal sum
    (1/(2 V_i)) sum_j (dF_j - Gamma dW_j) S, both as printed in Section 5: the full
    Gamma on the diagonal makes the cell-parallel point relaxation diagonally dominant;
  * inner convergence: ||R||_2 below tol_inner times its value at the first inner step.

Pins: tests/test_oracle_macro_pins.py (uniform fixed point, conduction closed form,
GSIS acceleration and mass, asymptotic-preserving slab against Kirchhoff's solution).
"""
from __future__ import annotations

import numpy as np

from . import kinetic as K
from . import model as mdl


# ----------------------------------------------------------------- state conversion
def nvar(dim):
    return dim + 5                         # rho, rho u (dim), e, e_r, e_v, e_R


def conservative(F, dim, model):
    rho, u = F["rho"], F["u"][:, :dim]
    e_r = 0.5 * model.d_r * rho * F["T_r"]
    e_v = rho * mdl.vib_energy(F["T_v"], model)
    e_R = 4.0 * model.sigma_R * F["T_R"] ** 4
    e = 1.5 * rho * F["T_t"] + 0.5 * rho * np.sum(u * u, axis=1) + e_r + e_v + e_R
    return np.column_stack([rho, rho[:, None] * u, e, e_r, e_v, e_R])


def primitive(W, dim, model):
    """(rho, u [n, dim], T_t, T_r, T_v, e_R)."""
    rho = W[:, 0]
    u = W[:, 1:1 + dim] / rho[:, None]
    e, e_r, e_v, e_R = W[:, 1 + dim], W[:, 2 + dim], W[:, 3 + dim], W[:, 4 + dim]
    T_t = (e - e_R - e_r - e_v - 0.5 * rho * np.sum(u * u, axis=1)) / (1.5 * rho)
    return rho, u, T_t, 2.0 * e_r / (model.d_r * rho), mdl.vib_temperature(e_v / rho, model), e_R


def fields_from_W(W, dim, model, template=None):
    rho, u, T_t, T_r, T_v, e_R = primitive(W, dim, model)
    F = K.empty_fields(W.shape[0]) if template is None else {k: v.copy() for k, v in template.items()}
    F["rho"], F["T_t"], F["T_r"], F["T_v"], F["e_R"] = rho, T_t, T_r, T_v, e_R
    F["u"] = np.zeros((W.shape[0], 3))
    F["u"][:, :dim] = u
    F["T_R"] = (np.maximum(e_R, 0.0) / (4.0 * model.sigma_R)) ** 0.25
    return F


# ----------------------------------------------------------------- face topology
class Faces:
    """Interior faces (owner i, neighbour j, unit normal i->j, area, centroid) and
    boundary faces of a mesh, with cell-centre least-squares gradients."""

    def __init__(self, geo):
        m = geo.mesh
        self.geo = geo
        dim = m.dim
        inner = m.face_nbr >= 0
        self.i = m.face_owner[inner].astype(np.int64)
        self.j = m.face_nbr[inner].astype(np.int64)
        self.n = m.face_normal[inner, :dim]
        self.S = m.face_area[inner]
        self.xf = m.face_centroid[inner, :dim]
        self.bf_cell = m.face_owner[~inner].astype(np.int64)
        self.bf_n = m.face_normal[~inner, :dim]
        self.bf_S = m.face_area[~inner]
        self.bf_patch = (-1 - m.face_nbr[~inner]).astype(np.int64)
        d = geo.delta(geo.xc[self.j] - geo.xc[self.i])
        self.dist = np.linalg.norm(d, axis=1)
        self.t = d / self.dist[:, None]
        self.dn = np.abs(np.sum(self.n * d, axis=1))          # |n . (x_j - x_i)|

    def gradient(self, q):
        """Least-squares gradients [nc, dim, k] of cell values q [nc, k] (stencil of the
        kinetic sweep)."""
        geo = self.geo
        g = np.zeros((geo.nc, geo.dim, q.shape[1]))
        for c in range(geo.nc):
            st, C = geo.lsq[c]
            for k, s in enumerate(st):
                g[c] += np.outer(C[k], q[s] - q[c])
        return g

    def face_gradient(self, q, g):
        """avg(grad) with its component along t replaced by (q_j - q_i)/|x_j - x_i|."""
        avg = 0.5 * (g[self.i] + g[self.j])                          # [nf, dim, k]
        along = np.einsum("fd,fdk->fk", self.t, avg)
        jump = (q[self.j] - q[self.i]) / self.dist[:, None]
        return avg + self.t[:, :, None] * (jump - along)[:, None, :]


def limited_values(faces, q, g, K_venkat):
    """Venkatakrishnan-limited reconstruction of cell values q [nc, k] to both sides of
    every interior face: (q_L at owner side, q_R at neighbour side)."""
    geo = faces.geo
    phi = np.ones_like(q)
    for c in range(geo.nc):
        nbrs = geo.face_nbrs[c]
        if not nbrs:
            continue
        dq = q[nbrs] - q[c]
        dmax = np.maximum(dq.max(axis=0), 0.0)
        dmin = np.minimum(dq.min(axis=0), 0.0)
        eps2 = (K_venkat * geo.dx[c]) ** 3
        for nb, _, _, xf in geo.cell_faces[c]:
            if nb < 0:
                continue
            d2 = g[c].T @ geo.delta(xf - geo.xc[c])
            d1 = np.where(d2 > 0.0, dmax, dmin)
            with np.errstate(invalid="ignore", divide="ignore"):
                pf = np.where(d2 != 0.0, K.venkatakrishnan(d1, d2, eps2), 1.0)
            phi[c] = np.minimum(phi[c], pf)
    dL = np.einsum("fdk,fd->fk", g[faces.i], geo.delta(faces.xf - geo.xc[faces.i]))
    dR = np.einsum("fdk,fd->fk", g[faces.j], geo.delta(faces.xf - geo.xc[faces.j]))
    return q[faces.i] + phi[faces.i] * dL, q[faces.j] + phi[faces.j] * dR


# ----------------------------------------------------------------- physics
def sound_speed(T_t):
    return mdl.sound_speed(T_t)


def convective_flux(prim, n, dim, model):
    """F_c . n of Eq. (macroscopic_equation) for states prim = (rho, u, T_t, T_r, T_v, e_R)."""
    rho, u, T_t, T_r, T_v, e_R = prim
    un = np.sum(u * n, axis=1)
    p = rho * T_t
    e_r = 0.5 * model.d_r * rho * T_r
    e_v = rho * mdl.vib_energy(T_v, model)
    e_gas = 1.5 * rho * T_t + 0.5 * rho * np.sum(u * u, axis=1) + e_r + e_v
    F = np.zeros((rho.shape[0], nvar(dim)))
    F[:, 0] = rho * un
    F[:, 1:1 + dim] = rho[:, None] * u * un[:, None] + p[:, None] * n
    F[:, 1 + dim] = un * (e_gas + p)
    F[:, 2 + dim] = un * e_r
    F[:, 3 + dim] = un * e_v
    return F


def prim_to_W(prim, dim, model):
    rho, u, T_t, T_r, T_v, e_R = prim
    e_r = 0.5 * model.d_r * rho * T_r
    e_v = rho * mdl.vib_energy(T_v, model)
    e = 1.5 * rho * T_t + 0.5 * rho * np.sum(u * u, axis=1) + e_r + e_v + e_R
    return np.column_stack([rho, rho[:, None] * u, e, e_r, e_v, e_R])


def rusanov(primL, primR, n, dim, model):
    """Rusanov (local Lax-Friedrichs) flux of F_c . n: the average of the two sides'
    fluxes minus half the largest |u_n| + c_s times the jump of the convected variables
    (e_R is not convected).  Chosen over contact-resolving solvers because its dissipation
    also damps the odd-even density/pressure mode that point relaxation leaves near walls
    in conduction-dominated slabs."""
    FL, FR = convective_flux(primL, n, dim, model), convective_flux(primR, n, dim, model)
    lam = np.maximum(np.abs(np.sum(primL[1] * n, axis=1)) + sound_speed(primL[2]),
                     np.abs(np.sum(primR[1] * n, axis=1)) + sound_speed(primR[2]))
    WL, WR = prim_to_W(primL, dim, model), prim_to_W(primR, dim, model)
    dW = WR - WL
    dW[:, 1 + dim] -= WR[:, 4 + dim] - WL[:, 4 + dim]        # gas part of the total energy
    dW[:, 4 + dim] = 0.0                                        # e_R is not convected
    return 0.5 * (FL + FR) - 0.5 * lam[:, None] * dW


def viscosity(T_t, model):
    """mu = p_t tau = sqrt(2/pi) Kn T_t^omega (Section 2.1)."""
    return np.sqrt(2.0 / np.pi) * model.Kn * T_t ** model.omega


def conductivity_base(T_v, model):
    """A^-1 diag(5, d_r, d_v) of Eq. (NSF_thermal_conductivities) per state [n, 3, 3]: the
    constant matrix, or with A and d_v taken at d_v(T_v) for the temperature-dependent d_v."""
    T_v = np.atleast_1d(np.asarray(T_v, np.float64))
    if not getattr(model, "dv_temperature_dependent", False):
        base = np.linalg.inv(mdl.relaxation_matrix(model)) @ np.diag([5.0, model.d_r, model.d_v])
        return np.broadcast_to(base, (T_v.shape[0], 3, 3))
    return np.stack([np.linalg.inv(mdl.relaxation_matrix(model, dv)) @ np.diag([5.0, model.d_r, dv])
                     for dv in mdl.dv_local(T_v, model)])


def nsf_face(faces, prim_face, grads, dim, model):
    """NSF stress (in-plane, [nf, dim, dim]) and heat fluxes (q_t, q_r, q_v, q_R [nf, dim])
    from face states and face gradients of (u, T_t, T_r, T_v, e_R): Eqs. (NSF_constitutive),
    (NSF_thermal_conductivities)."""
    rho, T_t = prim_face[0], prim_face[2]
    gu = grads["u"]                                             # [nf, dim(grad), dim(comp)]
    mu = viscosity(T_t, model)
    S = np.transpose(gu, (0, 2, 1)) + gu                        # du_a/dx_b + du_b/dx_a
    div = np.einsum("fdd->f", gu)
    sig = -mu[:, None, None] * (S - (2.0 / 3.0) * div[:, None, None] * np.eye(dim)[None])
    kap = 0.5 * mu[:, None, None] * conductivity_base(prim_face[4], model)
    gT = np.stack([grads["T_t"], grads["T_r"], grads["T_v"]], axis=1)     # [nf, 3, dim]
    q = -np.einsum("fij,fjd->fid", kap, gT)
    keff = mdl.absorption(rho, model)
    qR = -(1.0 / (3.0 * keff))[:, None] * grads["e_R"]
    return sig, q[:, 0], q[:, 1], q[:, 2], qR


def _cell_grad_dict(faces, prim, dim):
    rho, u, T_t, T_r, T_v, e_R = prim
    q = np.column_stack([u, T_t, T_r, T_v, e_R])
    g = faces.gradient(q)
    fg = faces.face_gradient(q, g)
    return {"u": fg[:, :, :dim], "T_t": fg[:, :, dim], "T_r": fg[:, :, dim + 1],
            "T_v": fg[:, :, dim + 2], "e_R": fg[:, :, dim + 3]}


def _face_avg_prim(faces, prim):
    return tuple(0.5 * (x[faces.i] + x[faces.j]) for x in prim)


def high_order_terms(faces, F_kin, kin_bflux, wl):
    """Face high-order terms of Eq. (getHoTs): the average of the two cells' kinetic
    stress and heat fluxes minus the NSF values of the kinetic state on the face; on
    boundary faces, the kinetic boundary flux minus the macroscopic one."""
    dim, model = wl.dim, wl.model
    W = conservative(F_kin, dim, model)
    prim = primitive(W, dim, model)
    grads = _cell_grad_dict(faces, prim, dim)
    sig, qt, qr, qv, qR = nsf_face(faces, _face_avg_prim(faces, prim), grads, dim, model)
    avg = lambda x: 0.5 * (x[faces.i] + x[faces.j])
    return {"sigma": avg(F_kin["sigma"][:, :dim, :dim]) - sig,
            "q_t": avg(F_kin["q_t"][:, :dim]) - qt, "q_r": avg(F_kin["q_r"][:, :dim]) - qr,
            "q_v": avg(F_kin["q_v"][:, :dim]) - qv, "q_R": avg(F_kin["q_R"][:, :dim]) - qR,
            "boundary": kin_bflux - macro_boundary_flux(faces, prim, wl)}


def viscous_flux(faces, prim, hot, dim, model):
    """F_v . n with the NSF part at the current state and the fixed high-order terms."""
    grads = _cell_grad_dict(faces, prim, dim)
    pf = _face_avg_prim(faces, prim)
    sig, qt, qr, qv, qR = nsf_face(faces, pf, grads, dim, model)
    sig = sig + hot["sigma"]
    qt, qr, qv, qR = qt + hot["q_t"], qr + hot["q_r"], qv + hot["q_v"], qR + hot["q_R"]
    n = faces.n
    u = pf[1]
    Fv = np.zeros((n.shape[0], nvar(dim)))
    sn = np.einsum("fab,fb->fa", sig, n)
    Fv[:, 1:1 + dim] = sn
    qtot = qt + qr + qv + qR
    Fv[:, 1 + dim] = np.sum(sn * u, axis=1) + np.sum(qtot * n, axis=1)
    Fv[:, 2 + dim] = np.sum(qr * n, axis=1)
    Fv[:, 3 + dim] = np.sum(qv * n, axis=1)
    Fv[:, 4 + dim] = np.sum(qR * n, axis=1)
    return Fv


def macro_boundary_flux(faces, prim, wl):
    """Macroscopic flux [nbf, nvar] out of each boundary face for cell states prim.

    Walls: the flux of an equilibrium leaving at the cell state against the diffuse wall
    (wall_equilibrium_flux).  Its difference from the kinetic wall flux is the boundary
    high-order term, which is small whenever the distribution near the wall is close to
    equilibrium, also before convergence; an NSF wall flux (conduction over the half
    cell) would instead leave the whole free-molecular flux of a non-converged state in
    that term.  Far field: Rusanov flux against the free stream plus NSF terms."""
    dim, model, geo = wl.dim, wl.model, faces.geo
    c, n = faces.bf_cell, faces.bf_n
    nb = c.shape[0]
    out = np.zeros((nb, nvar(dim)))
    rho, u, T_t, T_r, T_v, e_R = (x[c] for x in prim)
    xf = geo.mesh.face_centroid[geo.mesh.face_nbr < 0, :dim]
    dn = np.abs(np.sum(n * geo.delta(xf - geo.xc[c]), axis=1))
    for b in range(nb):
        patch = geo.mesh.patches[faces.bf_patch[b]]
        uw = np.asarray(patch.u, float)[:dim]
        if patch.kind == K.WALL:
            out[b] = wall_equilibrium_flux(faces, tuple(x[c[b]:c[b] + 1] for x in prim), wl, b)
            continue
        if patch.kind == K.SYMMETRY:
            # mirror state: the cell state with its normal velocity reversed; Rusanov between
            # the two carries no mass or energy and the pressure plus the damped normal
            # momentum; no viscous stress, conduction or radiative flux crosses a mirror
            inside = tuple(x[b:b + 1] for x in (rho, u, T_t, T_r, T_v, e_R))
            um = u[b:b + 1] - 2.0 * np.sum(u[b] * n[b]) * n[b:b + 1]
            mirror = (rho[b:b + 1], um, T_t[b:b + 1], T_r[b:b + 1], T_v[b:b + 1], e_R[b:b + 1])
            out[b] = rusanov(inside, mirror, n[b:b + 1], dim, model)[0]
            continue
        inside = (rho[b:b + 1], u[b:b + 1], T_t[b:b + 1], T_r[b:b + 1], T_v[b:b + 1], e_R[b:b + 1])
        far = (np.array([patch.rho]), uw[None], np.array([patch.T_t]), np.array([patch.T_r]),
               np.array([patch.T_v]), np.array([4.0 * model.sigma_R * patch.T_R ** 4]))
        Fc = rusanov(inside, far, n[b:b + 1], dim, model)[0]
        mu = viscosity(0.5 * (T_t[b] + patch.T_t), model)
        du = uw - u[b]
        sn = -mu / dn[b] * (du + (np.dot(n[b], du) / 3.0) * n[b])
        kap = 0.5 * mu * conductivity_base(0.5 * (T_v[b] + patch.T_v), model)[0]
        q = -(kap @ (np.array([patch.T_t, patch.T_r, patch.T_v]) - np.array([T_t[b], T_r[b], T_v[b]]))) / dn[b]
        keff = mdl.absorption(rho[b:b + 1], model)[0]
        qR = -(far[5][0] - e_R[b]) / (3.0 * keff * dn[b])
        out[b] = Fc
        out[b, 1:1 + dim] += sn
        out[b, 1 + dim] += np.dot(sn, 0.5 * (uw + u[b])) + q.sum() + qR
        out[b, 2 + dim] += q[1]
        out[b, 3 + dim] += q[2]
        out[b, 4 + dim] += qR
    return out


def wall_equilibrium_flux(faces, state, wl, b):
    """Flux out of wall face b when the molecules leaving the domain are in equilibrium at
    the cell state and the wall re-emits them diffusely (density from zero net mass flux),
    photons leave isotropically (e_R / 4 pi) and the wall emits black-body; evaluated with
    the discrete velocity and direction quadratures.  Rows as kinetic_boundary_flux."""
    dim, model = wl.dim, wl.model
    xi, w, om, wo = wl.xi, wl.w, wl.omega, wl.wo
    n = faces.bf_n[b]
    patch = faces.geo.mesh.patches[faces.bf_patch[b]]
    rho, u, T_t, T_r, T_v, e_R = state
    Fc = {"rho": rho, "u": np.pad(u, ((0, 0), (0, 3 - dim))), "T_t": T_t, "T_r": T_r, "T_v": T_v}
    fe = K.equilibrium_planes(Fc, xi, dim, model)[0]
    xn = xi[:, :dim] @ n
    rw = K.wall_density(None, fe[:, 0], xi, w, dim, patch, n)
    face = np.where((xn > 0)[:, None], fe, K.incoming_gas(patch, rw, xi, dim, model))
    wf = w * xn
    out = np.zeros(nvar(dim))
    xi2 = np.sum(xi[:, :dim] ** 2, axis=1)
    out[0] = wf @ face[:, 0]
    out[1:1 + dim] = (wf * face[:, 0]) @ xi[:, :dim]
    e_gas = wf @ (0.5 * xi2 * face[:, 0] + 0.5 * face[:, 1] + face[:, 2] + face[:, 3])
    out[2 + dim] = wf @ face[:, 2]
    out[3 + dim] = wf @ face[:, 3]
    on = om[:, :dim] @ n
    Iface = np.where(on > 0, e_R[0] / (4.0 * np.pi), K.incoming_photon(patch, model, om.shape[0]))
    out[4 + dim] = (wo * on) @ Iface
    out[1 + dim] = e_gas + out[4 + dim]
    return out


def source(prim, dim, model):
    """Q of Section 5: relaxation of e_r, e_v and the gas-photon exchange."""
    rho, u, T_t, T_r, T_v, e_R = prim
    T_tr, T_tv, _ = mdl.mode_temperatures(T_t, T_r, T_v, model)
    tau = mdl.relaxation_time(rho, T_t, model.Kn, model.omega)
    k = mdl.absorption(rho, model)
    e_vR = 4.0 * model.sigma_R * T_v ** 4
    Q = np.zeros((rho.shape[0], nvar(dim)))
    Q[:, 2 + dim] = 0.5 * model.d_r * rho * (T_tr - T_r) / (model.Z_r * tau)
    Q[:, 3 + dim] = rho * (mdl.vib_energy(T_tv, model) - mdl.vib_energy(T_v, model)) / (model.Z_v * tau) \
        - k * (e_vR - e_R)                                      # (e_tv - e_v) / (Z_v tau) - k (e_vR - e_R)
    Q[:, 4 + dim] = k * (e_vR - e_R)
    return Q


# ----------------------------------------------------------------- kinetic boundary fluxes
def kinetic_boundary_flux(faces, f, I, wl):
    """Moments of the kinetic flux through every boundary face: outgoing molecules carry
    the cell's distribution, incoming ones the wall (density from zero net mass flux)
    or far-field distribution; photons likewise.  Rows: [nbf, nvar]."""
    mesh, model, dim = wl.mesh, wl.model, wl.dim
    xi, w, om, wo = wl.xi, wl.w, wl.omega, wl.wo
    out = np.zeros((faces.bf_cell.shape[0], nvar(dim)))
    xi2 = np.sum(xi[:, :dim] ** 2, axis=1)
    for b, (c, n, p) in enumerate(zip(faces.bf_cell, faces.bf_n, faces.bf_patch)):
        patch = mesh.patches[p]
        xn = xi[:, :dim] @ n
        if patch.kind == K.SYMMETRY:
            inc = f[c][K.reflection_index(xi[:, :dim], n)]
        else:
            rw = K.wall_density(None, f[c, :, 0], xi, w, dim, patch, n) if patch.kind == K.WALL else 1.0
            inc = K.incoming_gas(patch, rw, xi, dim, model)
        face = np.where((xn > 0)[:, None], f[c], inc)
        wf = w * xn
        out[b, 0] = wf @ face[:, 0]
        out[b, 1:1 + dim] = (wf * face[:, 0]) @ xi[:, :dim]
        e_gas = wf @ (0.5 * xi2 * face[:, 0] + 0.5 * face[:, 1] + face[:, 2] + face[:, 3])
        out[b, 2 + dim] = wf @ face[:, 2]
        out[b, 3 + dim] = wf @ face[:, 3]
        on = om[:, :dim] @ n
        if patch.kind == K.SYMMETRY:
            Iinc = I[c][K.reflection_index(om, np.pad(n, (0, 3 - dim)))]
        else:
            Iinc = K.incoming_photon(patch, model, om.shape[0])
        Iface = np.where(on > 0, I[c], Iinc)
        qR = (wo * on) @ Iface
        out[b, 4 + dim] = qR
        out[b, 1 + dim] = e_gas + qR
    return out


# ----------------------------------------------------------------- residual and solve
def residual(W, faces, hot, wl, offset=None):
    """R_i = -(1/V_i) sum_faces S (F_c + F_v).n + Q_i  (Eq. delta_macro, right-hand side),
    plus a fixed per-cell ``offset`` [nc, nvar] when given (the defect correction of
    gsis.gsis_step)."""
    dim, model, geo = wl.dim, wl.model, faces.geo
    prim = primitive(W, dim, model)
    q = np.column_stack([prim[0], prim[1], prim[2], prim[3], prim[4], prim[5]])
    if wl.solver.order == 2:
        g = faces.gradient(q)
        qL, qR = limited_values(faces, q, g, wl.solver.venkat_K)
    else:
        qL, qR = q[faces.i], q[faces.j]
    split = lambda a: (a[:, 0], a[:, 1:1 + dim], a[:, 1 + dim], a[:, 2 + dim], a[:, 3 + dim], a[:, 4 + dim])
    Fc = rusanov(split(qL), split(qR), faces.n, dim, model)
    Fv = viscous_flux(faces, prim, hot, dim, model)
    flux = (Fc + Fv) * faces.S[:, None]
    R = np.zeros_like(W)
    np.add.at(R, faces.i, -flux)
    np.add.at(R, faces.j, flux)
    bflux = macro_boundary_flux(faces, prim, wl) + hot["boundary"]
    np.add.at(R, faces.bf_cell, -bflux * faces.bf_S[:, None])
    R /= geo.vol[:, None]
    R = R + source(prim, dim, model)
    return R if offset is None else R + offset


def gamma_face(faces, prim, wl):
    """Per-row Gamma_ij [nf, nvar] at the face-average state: |u_n| + c_s +
    2 mu / (rho |n . (x_j - x_i)|) in every row, plus 2 kappa_R / |n . (x_j - x_i)| in the
    total-energy and e_R rows (kappa_R = 1/(3 k_eff), the photon diffusion of
    Eq. NSF_constitutive, which the viscous term alone does not bound)."""
    dim = wl.dim
    rho, u, T_t = (0.5 * (x[faces.i] + x[faces.j]) for x in prim[:3])
    un = np.abs(np.sum(u * faces.n, axis=1))
    base = un + sound_speed(T_t) + 2.0 * viscosity(T_t, wl.model) / (rho * faces.dn)
    G = np.repeat(base[:, None], nvar(dim), axis=1)
    kR = 1.0 / (3.0 * mdl.absorption(rho, wl.model))
    G[:, 4 + dim] += 2.0 * kR / faces.dn
    return G


def boundary_gamma(faces, prim, wl):
    """Gamma of boundary faces [nbf, nvar]: |u_n| + c_s + 2 mu/(rho d_b) with d_b the
    distance from the cell centre to the face along n, plus 2 kappa_R/d_b in the e_R row
    (the boundary flux depends on the cell state through pressure, viscous stress and
    conduction over d_b)."""
    dim, geo = wl.dim, faces.geo
    c, n = faces.bf_cell, faces.bf_n
    rho, u, T_t = prim[0][c], prim[1][c], prim[2][c]
    xf = geo.mesh.face_centroid[geo.mesh.face_nbr < 0, :dim]
    db = np.abs(np.sum(n * geo.delta(xf - geo.xc[c]), axis=1))
    base = np.abs(np.sum(u * n, axis=1)) + sound_speed(T_t) + 2.0 * viscosity(T_t, wl.model) / (rho * db)
    G = np.repeat(base[:, None], nvar(dim), axis=1)
    kR = 1.0 / (3.0 * mdl.absorption(rho, wl.model))
    G[:, 4 + dim] += 2.0 * kR / db
    sym = np.array([geo.mesh.patches[p].kind == K.SYMMETRY for p in faces.bf_patch], bool)
    if sym.any():
        # a mirror face: the Rusanov part only, and no e_R flux
        G[sym] = (np.abs(np.sum(u * n, axis=1)) + sound_speed(T_t))[sym, None]
        G[sym, 4 + dim] = 0.0
    return G


def source_jacobian_block(prim, dim, model):
    """Exact d(Q_egas, Q_r, Q_v, Q_R)/d(e_gas, e_r, e_v, e_R) per cell [n, 4, 4] with rho, rho u,
    tau and k_eff held fixed; e_gas = e - e_R, T_t = (e_gas - e_r - e_v - rho u^2/2)/(1.5 rho).

    Q_v = rho (eps(T_tv) - eps_v) / (Z_v tau) - k (e_vR - e_R) with eps(T) = d_v(T) T / 2,
    eps_v = e_v / rho and T_tv defined by 3 T_tv + 2 eps(T_tv) = 3 T_t + 2 eps_v, so
    dT_tv = (3 dT_t + 2 d eps_v) / (3 + 2 eps'(T_tv)) and, with dT_t = a (de_gas - de_r - de_v),
    a = 2 / (3 rho):
        d(rho eps(T_tv)) = b (3a de_gas - 3a de_r + (2/rho - 3a) de_v),  b = rho eps'(T_tv) / (3 + 2 eps'(T_tv)),
    where 2/rho - 3a = 0; e_vR = 4 sigma_R T_v^4 gives d e_vR / d e_v = 16 sigma_R T_v^3 / (rho eps'(T_v)).
    For constant d_v, eps' = d_v / 2 and these reduce to the constant-coefficient forms
    (Appendix A's diagonal entries are the e_r, e_v and e_R diagonal of this block)."""
    rho, u, T_t, T_r, T_v, e_R = prim
    tau = mdl.relaxation_time(rho, T_t, model.Kn, model.omega)
    k = mdl.absorption(rho, model)
    dr = model.d_r
    T_tv = mdl.mode_temperatures(T_t, T_r, T_v, model)[1]
    cr = rho * 1.5 * dr / (3.0 + dr) / (model.Z_r * tau)          # Q_r = cr (T_t - T_r)
    ctv = mdl.vib_heat_capacity(T_tv, model)
    b = rho * ctv / (3.0 + 2.0 * ctv)
    beta = 16.0 * model.sigma_R * T_v ** 3 / (rho * mdl.vib_heat_capacity(T_v, model))   # d e_vR / d e_v
    a = 1.0 / (1.5 * rho)                                         # d T_t / d e_gas
    zv = 1.0 / (model.Z_v * tau)
    J = np.zeros((rho.shape[0], 4, 4))
    J[:, 0, 2], J[:, 0, 3] = -k * beta, k
    J[:, 1, 0], J[:, 1, 1], J[:, 1, 2] = cr * a, -cr * (a + 2.0 / (dr * rho)), -cr * a
    J[:, 2, 0], J[:, 2, 1] = 3.0 * a * b * zv, -3.0 * a * b * zv
    J[:, 2, 2], J[:, 2, 3] = -zv - k * beta, k
    J[:, 3, 2], J[:, 3, 3] = k * beta, -k
    return J


def macro_solve(W0, faces, hot, wl, history=None, offset=None):
    """Pseudo-time iterations of Eq. (delta_macro) until ||R|| <= tol_inner ||R_0|| or
    max_inner.  Each iteration solves
        D_i dW_i + (1/(2 V_i)) sum_j (dF_j . n_ij - Gamma_ij dW_j) S_ij = R_i,
        D_i = 1/dt + (1/V_i) sum_j Gamma_ij S_ij - dQ/dW (energy-row block),
        dF_j = F_c(W_j + dW_j) - F_c(W_j),
    with macro_sweeps point-relaxation sweeps in which every cell uses its neighbours'
    increments from the previous sweep (Jacobi), then W += dW."""
    dim, model, geo, s = wl.dim, wl.model, faces.geo, wl.solver
    W = W0.copy()
    r0 = None
    for it in range(s.max_inner):
        prim = primitive(W, dim, model)
        R = residual(W, faces, hot, wl, offset)
        rn = np.sqrt(np.sum(R * R))
        if history is not None:
            history.append(rn)
        if r0 is None:
            r0 = rn
        if not np.isfinite(rn) or rn <= s.tol_inner * r0:
            break
        Gam = gamma_face(faces, prim, wl)
        umag = np.sqrt(np.sum(prim[1] ** 2, axis=1))
        inv_dt = (umag + sound_speed(prim[2])) / (s.cfl_macro * geo.dx)
        gsum = np.zeros_like(W)
        np.add.at(gsum, faces.i, Gam * faces.S[:, None])
        np.add.at(gsum, faces.j, Gam * faces.S[:, None])
        np.add.at(gsum, faces.bf_cell, boundary_gamma(faces, prim, wl) * faces.bf_S[:, None])
        E, ER = 1 + dim, 4 + dim
        diag = inv_dt[:, None] + gsum / geo.vol[:, None]
        D = np.zeros((geo.nc, W.shape[1], W.shape[1]))
        idx = np.arange(W.shape[1])
        D[:, idx, idx] = diag
        D[:, E:ER + 1, E:ER + 1] -= source_jacobian_block(prim, dim, model)
        Dinv = np.linalg.inv(D)
        Rg = R.copy()
        Rg[:, E] -= R[:, ER]                                     # gas-energy row
        Wi, Wj = W[faces.i], W[faces.j]
        Fi = convective_flux(primitive(Wi, dim, model), faces.n, dim, model)    # flux of W_i on n_ij
        Fj = convective_flux(primitive(Wj, dim, model), faces.n, dim, model)
        dG = np.zeros_like(W)                                    # increments with e_gas in row E
        for _ in range(s.macro_sweeps):
            dW = dG.copy()
            dW[:, E] += dG[:, ER]                                # total-energy increment
            # owner i sees neighbour j through n_ij; neighbour j sees owner i through -n_ij
            dFj = convective_flux(primitive(Wj + dW[faces.j], dim, model), faces.n, dim, model) - Fj
            dFi = convective_flux(primitive(Wi + dW[faces.i], dim, model), faces.n, dim, model) - Fi
            off = np.zeros_like(W)
            np.add.at(off, faces.i, (dFj - Gam * dG[faces.j]) * faces.S[:, None])
            np.add.at(off, faces.j, (-dFi - Gam * dG[faces.i]) * faces.S[:, None])
            dG = np.einsum("nij,nj->ni", Dinv, Rg - off / (2.0 * geo.vol[:, None]))
        dW = dG.copy()
        dW[:, E] += dG[:, ER]
        W = W + dW
    return W
