"""Oracle (test infrastructure only): the kinetic half of GSIS in plain FP64 NumPy.

Restates
  * the reduced distributions and kinetic model, Eqs. (reduced_distribution),
    (kinetic_equation), with the reference distributions of Eq.
    (reference_distribution) and the Maxwellian of Eq. (equilibrium_distribution);
  * the velocity moments of Eq. (getmoment);
  * the implicit incremental finite-volume step of Eq. (dis_micro) with the
    first-order upwind flux increment, the limited linear reconstruction of Eq.
    (deltaflux_micro) and point relaxation (Section 5).

Reduced velocity spaces (the paper reduces its 1-D/2-D cases to fewer velocity
dimensions without spelling the reduction out): with ``dim`` in-plane velocity
components and ``m = 3 - dim`` hidden ones, f0 is carried as two planes,
F0 = int f0 dxi_hidden and H0 = int |xi_hidden|^2 f0 dxi_hidden; f1 and f2 are
integrated over the hidden components.  Plane order: [F0, H0, f1, f2].
"""
from __future__ import annotations

import numpy as np

from . import model as mdl

WALL, FARFIELD, SYMMETRY = 0, 1, 2


# --------------------------------------------------------------------------- fields
def empty_fields(n):
    z = np.zeros
    return dict(rho=z(n), u=z((n, 3)), T_t=z(n), T_r=z(n), T_v=z(n), T_R=z(n),
                q_t=z((n, 3)), q_r=z((n, 3)), q_v=z((n, 3)), q_R=z((n, 3)), sigma=z((n, 3, 3)),
                e_R=z(n))


def fields_from_record(M, sigma_R):
    """Library per-cell record (26 doubles) -> dict of arrays."""
    n = M.shape[0]
    F = empty_fields(n)
    F["rho"], F["u"] = M[:, 0].copy(), M[:, 1:4].copy()
    F["T_t"], F["T_r"], F["T_v"], F["T_R"] = (M[:, k].copy() for k in (4, 5, 6, 7))
    F["q_t"], F["q_r"], F["q_v"], F["q_R"] = (M[:, k:k + 3].copy() for k in (8, 11, 14, 17))
    s = M[:, 20:26]
    F["sigma"] = np.stack([np.stack([s[:, 0], s[:, 3], s[:, 4]], 1),
                           np.stack([s[:, 3], s[:, 1], s[:, 5]], 1),
                           np.stack([s[:, 4], s[:, 5], s[:, 2]], 1)], 1)
    F["e_R"] = 4.0 * sigma_R * F["T_R"] ** 4
    return F


def fields_to_record(F):
    n = F["rho"].shape[0]
    M = np.zeros((n, 26))
    M[:, 0], M[:, 1:4] = F["rho"], F["u"]
    M[:, 4], M[:, 5], M[:, 6], M[:, 7] = F["T_t"], F["T_r"], F["T_v"], F["T_R"]
    M[:, 8:11], M[:, 11:14], M[:, 14:17], M[:, 17:20] = F["q_t"], F["q_r"], F["q_v"], F["q_R"]
    s = F["sigma"]
    M[:, 20:26] = np.stack([s[:, 0, 0], s[:, 1, 1], s[:, 2, 2], s[:, 0, 1], s[:, 0, 2], s[:, 1, 2]], 1)
    return M


# --------------------------------------------------------------------------- moments
def moments(f, I, xi, w, omega, wo, dim, model):
    """Macroscopic fields of Eq. (getmoment) from f [n, V, 4] and I [n, n_omega].

    Works with any subset of cells.  All moments are taken about the cell's own
    flow velocity (c = xi - u), exactly as written in the paper.
    """
    n = f.shape[0]
    F = empty_fields(n)
    m_hid = 3 - dim
    f0, h0, f1, f2 = f[..., 0], f[..., 1], f[..., 2], f[..., 3]
    rho = f0 @ w
    u = np.zeros((n, 3))
    u[:, :dim] = (f0 * w) @ xi[:, :dim] / rho[:, None]
    c = xi[None, :, :dim] - u[:, None, :dim]                      # [n, V, dim]
    c2 = np.sum(c * c, axis=-1)
    int_c2 = (c2 * f0) @ w + h0 @ w                               # int c^2 f0 over all of xi
    F["rho"], F["u"] = rho, u
    F["T_t"] = int_c2 / (3.0 * rho)
    F["T_r"] = 2.0 * (f1 @ w) / (model.d_r * rho)
    F["T_v"] = mdl.vib_temperature((f2 @ w) / rho, model)     # int f2 = d_v(T_v) rho T_v / 2
    sig = np.zeros((n, 3, 3))
    for a in range(dim):
        for b in range(dim):
            sig[:, a, b] = (c[..., a] * c[..., b] * f0) @ w
    for a in range(dim, 3):                                       # hidden directions share H0
        sig[:, a, a] = (h0 @ w) / m_hid
    sig -= (int_c2 / 3.0)[:, None, None] * np.eye(3)[None]
    F["sigma"] = sig
    for a in range(dim):
        F["q_t"][:, a] = 0.5 * (c[..., a] * (c2 * f0 + h0)) @ w
        F["q_r"][:, a] = (c[..., a] * f1) @ w
        F["q_v"][:, a] = (c[..., a] * f2) @ w
        F["q_R"][:, a] = I @ (wo * omega[:, a])
    F["e_R"] = I @ wo
    F["T_R"] = (np.maximum(F["e_R"], 0.0) / (4.0 * model.sigma_R)) ** 0.25 if model.sigma_R > 0 else 0.0 * rho
    return F


# --------------------------------------------------------------------------- distributions
def unit_maxwellian(xi, u, T, dim):
    """(2 pi T)^(-dim/2) exp(-|xi - u|^2 / 2T) over the in-plane components (Eq.
    equilibrium_distribution, integrated over hidden components).  u, T per cell."""
    c = xi[None, :, :dim] - u[:, None, :dim]
    c2 = np.sum(c * c, axis=-1)
    return (2.0 * np.pi * T[:, None]) ** (-0.5 * dim) * np.exp(-c2 / (2.0 * T[:, None])), c, c2


def reference_planes(F, xi, dim, model):
    """Combined reference distribution g of every plane, Eqs. (kinetic_equation) and
    (reference_distribution): g = (1 - 1/Z_r - 1/Z_v) g_t + g_r/Z_r + g_v/Z_v.

    Returns [n, V, 4].  The q.c(...) Shakhov factors use the in-plane heat fluxes.
    """
    m = 3 - dim
    d_r = model.d_r
    rho, T_t, T_r, T_v = F["rho"], F["T_t"], F["T_r"], F["T_v"]
    # (q0, q1, q2) = Mix (q_t, q_r, q_v); with the temperature-dependent d_v, A and Mix are
    # taken at each cell's d_v(T_v)
    if getattr(model, "dv_temperature_dependent", False):
        dvl = mdl.dv_local(T_v, model)
        Mix = np.stack([mdl.aux_heat_flux_matrix(mdl.relaxation_matrix(model, dv), model.Z_r, model.Z_v)
                        for dv in dvl])
    else:
        Mix = np.broadcast_to(mdl.aux_heat_flux_matrix(mdl.relaxation_matrix(model), model.Z_r, model.Z_v),
                              (rho.shape[0], 3, 3))
    qs = np.stack([F["q_t"], F["q_r"], F["q_v"]], 1)              # [n, mode, component]
    q0, q1, q2 = (np.einsum("nj,nja->na", Mix[:, r], qs) for r in range(3))
    qt, qr, qv = F["q_t"], F["q_r"], F["q_v"]
    T_tr, T_tv, _ = mdl.mode_temperatures(T_t, T_r, T_v, model)
    e_v, e_tv = mdl.vib_energy(T_v, model), mdl.vib_energy(T_tv, model)   # d_v(T) T / 2
    comps = (
        # weight, T_a, q in g0a, multiplier of g0a in g1a, in g2a, q in g1a, q in g2a
        (1.0 - 1.0 / model.Z_r - 1.0 / model.Z_v, T_t, qt, 0.5 * d_r * T_r, e_v, qr, qv),
        (1.0 / model.Z_r, T_tr, q0, 0.5 * d_r * T_tr, e_v, q1, q2),
        (1.0 / model.Z_v, T_tv, q0, 0.5 * d_r * T_r, e_tv, q1, q2),
    )
    n, V = rho.shape[0], xi.shape[0]
    g = np.zeros((n, V, 4))
    for alpha, Ta, qa, k1, k2, qa1, qa2 in comps:
        feq, c, c2 = unit_maxwellian(xi, F["u"], Ta, dim)
        Ta_ = Ta[:, None]
        qc = np.einsum("nvd,nd->nv", c, qa[:, :dim])
        s = 2.0 / (15.0 * Ta_ * rho[:, None] * Ta_)               # 2 / (15 T_a p_a)
        g0a = rho[:, None] * feq * (1.0 + s * qc * ((c2 + m * Ta_) / (2.0 * Ta_) - 2.5))
        h0a = rho[:, None] * feq * (m * Ta_ + s * qc * m * Ta_ * ((c2 + (m + 2) * Ta_) / (2.0 * Ta_) - 2.5))
        g1a = k1[:, None] * g0a + np.einsum("nvd,nd->nv", c, qa1[:, :dim]) / Ta_ * feq
        g2a = k2[:, None] * g0a + np.einsum("nvd,nd->nv", c, qa2[:, :dim]) / Ta_ * feq
        g[..., 0] += alpha * g0a
        g[..., 1] += alpha * h0a
        g[..., 2] += alpha * g1a
        g[..., 3] += alpha * g2a
    return g


def equilibrium_planes(F, xi, dim, model):
    """Multi-temperature local equilibrium: F0 = rho f_eq(T_t), H0 = m T_t F0,
    f1 = (d_r/2) T_r F0, f2 = (d_v(T_v)/2) T_v F0 (the moments of Eq. getmoment)."""
    m = 3 - dim
    feq, _, _ = unit_maxwellian(xi, F["u"], F["T_t"], dim)
    F0 = F["rho"][:, None] * feq
    return np.stack([F0, m * F["T_t"][:, None] * F0, 0.5 * model.d_r * F["T_r"][:, None] * F0,
                     mdl.vib_energy(F["T_v"], model)[:, None] * F0], axis=-1)


def photon_equilibrium(T, n_omega, sigma_R):
    """B_R(T) = sigma_R T^4 / pi in every direction."""
    return np.repeat((sigma_R * T ** 4 / np.pi)[:, None], n_omega, axis=1)


# --------------------------------------------------------------------------- geometry
class Geometry:
    """Cell -> face connectivity and least-squares gradient weights of a face-list mesh."""

    def __init__(self, mesh):
        self.mesh = mesh
        self.dim, self.nc = mesh.dim, mesh.n_cells
        dim = self.dim
        self.cell_faces = [[] for _ in range(self.nc)]  # (nbr or -1-patch, outward n, S, x_face)
        for f in range(mesh.n_faces):
            o, nb = int(mesh.face_owner[f]), int(mesh.face_nbr[f])
            n, S, xf = mesh.face_normal[f, :dim], float(mesh.face_area[f]), mesh.face_centroid[f, :dim]
            self.cell_faces[o].append((nb, n.copy(), S, xf.copy()))
            if nb >= 0:
                self.cell_faces[nb].append((o, -n, S, xf.copy()))
        self.vol = mesh.cell_volume.astype(np.float64)
        self.xc = mesh.cell_centroid[:, :dim].astype(np.float64)
        self.period = float(getattr(mesh, "period", 0.0))
        self.dx = self.vol ** (1.0 / dim)
        # Least squares: grad_i = sum_j C_ij (phi_j - phi_i) over the stencil of cell i,
        # C_ij = (sum_k d_k d_k^T)^-1 d_j, d_j = x_j - x_i.  The stencil is the face
        # neighbours and their face neighbours: with face neighbours alone, the
        # second-order upwind residual on triangles is not contracted by a first-order
        # implicit operator (some eigenvalues of A1^-1 A2 have negative real part).
        # A zero gradient is used where the normal matrix is singular.
        self.face_nbrs = [[fc[0] for fc in self.cell_faces[i] if fc[0] >= 0] for i in range(self.nc)]
        self.lsq = []
        for i in range(self.nc):
            st = set(self.face_nbrs[i])
            for j in self.face_nbrs[i]:
                st.update(self.face_nbrs[j])
            st.discard(i)
            st = sorted(st)
            if len(st) < dim:
                self.lsq.append((st, np.zeros((len(st), dim))))
                continue
            D = self.delta(self.xc[st] - self.xc[i])
            G = D.T @ D
            scale = np.trace(G) / dim
            if np.linalg.det(G) <= 1e-10 * scale ** dim:
                self.lsq.append((st, np.zeros((len(st), dim))))
                continue
            self.lsq.append((st, D @ np.linalg.inv(G).T))

    def delta(self, d):
        """Difference vectors d [..., dim] between two positions of the mesh: as given, or on
        a domain periodic in x (mesh.period > 0) the minimal image of their x component."""
        if self.period > 0.0:
            d = np.array(d, np.float64, copy=True)
            d[..., 0] -= self.period * np.round(d[..., 0] / self.period)
        return d

    def interior_neighbours(self, i):
        return self.face_nbrs[i]


def venkatakrishnan(d1, d2, eps2):
    """Venkatakrishnan's smooth limiter function phi(Delta_1, Delta_2)."""
    return (d1 * d1 + eps2 + 2.0 * d1 * d2) / (d1 * d1 + 2.0 * d2 * d2 + d1 * d2 + eps2)


def limited_slope(geo, i, q, K):
    """Venkatakrishnan-limited least-squares gradient of the cell values q[i] ([..]-shaped
    per cell).  The bounds Delta_max, Delta_min come from the face neighbours.
    Returns (grad [dim, ...], phi [...])."""
    stencil, C = geo.lsq[i]
    qi = q[i]
    grad = np.zeros((geo.dim,) + qi.shape)
    for k, j in enumerate(stencil):
        dq = q[j] - qi
        for a in range(geo.dim):
            grad[a] = grad[a] + C[k, a] * dq
    nbrs = geo.face_nbrs[i]
    if len(nbrs) == 0:
        return grad, np.ones(qi.shape)
    dq = np.stack([q[j] - qi for j in nbrs])                      # [k, ...]
    dmax = np.maximum(dq.max(axis=0), 0.0)
    dmin = np.minimum(dq.min(axis=0), 0.0)
    eps2 = (K * geo.dx[i]) ** 3
    phi = np.ones(qi.shape)
    for nb, _, _, xf in geo.cell_faces[i]:
        if nb < 0:
            continue
        d2 = np.zeros(qi.shape)
        dx = geo.delta(xf - geo.xc[i])
        for a in range(geo.dim):
            d2 = d2 + grad[a] * dx[a]
        d1 = np.where(d2 > 0.0, dmax, dmin)
        with np.errstate(invalid="ignore", divide="ignore"):
            pf = np.where(d2 != 0.0, venkatakrishnan(d1, d2, eps2), 1.0)
        phi = np.minimum(phi, pf)
    return grad, phi


# --------------------------------------------------------------------------- boundaries
def wall_density(geo, f0_cell, xi, w, dim, patch, n):
    """Density of the diffusely re-emitted Maxwellian that makes the net mass flux
    through a wall face zero: rho_w = -sum_{xi.n>0} w xi.n f0 / sum_{xi.n<0} w xi.n F_w."""
    xn = xi[:, :dim] @ n
    Fw, _, _ = unit_maxwellian(xi, np.asarray(patch.u, np.float64)[None], np.array([patch.T_t]), dim)
    out = np.sum(np.where(xn > 0, w * xn * f0_cell, 0.0))
    inc = np.sum(np.where(xn < 0, w * xn * Fw[0], 0.0))
    return -out / inc


def reflection_index(points, n):
    """For each point p of a velocity (or direction) set, the index of its mirror image
    p - 2 (p.n) n under specular reflection at a plane of unit normal n (reading: the sets
    must be symmetric under that reflection; the images are matched to 1e-9 of the set's
    scale).  Photon directions are matched with all three components: reflection at an
    in-plane normal keeps Omega_z."""
    d = points.shape[1]
    img = points - 2.0 * (points @ n[:d])[:, None] * n[None, :d]
    scale = max(np.abs(points).max(), 1.0)
    dist = np.abs(img[:, None, :] - points[None, :, :]).max(axis=-1)
    idx = np.argmin(dist, axis=1)
    if np.any(dist[np.arange(points.shape[0]), idx] > 1e-9 * scale):
        raise ValueError("the set is not symmetric under reflection at this normal")
    return idx


def incoming_gas(patch, rho_w, xi, dim, model):
    """Planes entering the domain through a boundary face ([V, 4])."""
    m = 3 - dim
    if patch.kind == WALL:
        rho, T, Tr, Tv = rho_w, patch.T_t, patch.T_t, patch.T_t
    else:
        rho, T, Tr, Tv = patch.rho, patch.T_t, patch.T_r, patch.T_v
    Fw, _, _ = unit_maxwellian(xi, np.asarray(patch.u, np.float64)[None], np.array([T]), dim)
    F0 = rho * Fw[0]
    return np.stack([F0, m * T * F0, 0.5 * model.d_r * Tr * F0, float(mdl.vib_energy(Tv, model)) * F0], axis=-1)


def incoming_photon(patch, model, n_omega):
    T = patch.T_t if patch.kind == WALL else patch.T_R
    return np.full(n_omega, model.sigma_R * T ** 4 / np.pi)


# --------------------------------------------------------------------------- sources
def relaxation_source(Fc, f, I, wl):
    """Right-hand sides of Eq. (kinetic_equation) without transport, per cell:
    gas (g - f)/tau plus, in the f2 equation, -(f0/rho) k_eff (4 sigma_R T_v^4 - int I);
    photons k_eff (sigma_R T_v^4/pi - I).  Also returns the implicit rates 1/tau, k_eff."""
    model, dim = wl.model, wl.mesh.dim
    g = reference_planes(Fc, wl.xi, dim, model)
    rho, T_v = Fc["rho"], Fc["T_v"]
    tau = mdl.relaxation_time(rho, Fc["T_t"], model.Kn, model.omega)
    keff = mdl.absorption(rho, model)
    src = (g - f) / tau[:, None, None]
    sink = -keff * (4.0 * model.sigma_R * T_v ** 4 - Fc["e_R"]) / rho
    src[..., 3] += sink[:, None] * f[..., 0]
    srcR = keff[:, None] * (model.sigma_R * T_v[:, None] ** 4 / np.pi - I)
    return src, srcR, 1.0 / tau, keff


# --------------------------------------------------------------------------- sweep
def kinetic_residual(f, I, wl, geo, cells, F=None):
    """The right-hand side of Eq. dis_micro at f, I for ``cells``: per cell and discrete
    velocity (photon direction)
      r_i = (g_i - f_i)/tau_i + s_i - (1/V_i) sum_faces S (xi_n^+ f_L + xi_n^- f_R),
      d_i = 1/dt_i + 1/tau_i + (1/V_i) sum_faces S xi_n^+,
    with the coefficients of the reference distributions from the fields F (default: the
    moments of f, I).  Returns (res [n, V, 4], dg [n, V], resR [n, n_omega],
    dR [n, n_omega], offdiag), offdiag[k] listing (neighbour, S xi_n^- / V, S Omega_n^- / V)
    for every interior face of cells[k]."""
    mesh, model, solver = wl.mesh, wl.model, wl.solver
    dim, xi, w, om, wo = mesh.dim, wl.xi, wl.w, wl.omega, wl.wo
    order, K = solver.order, solver.venkat_K

    # cells whose moments are needed: targets and their neighbours (the neighbours'
    # values enter only through f, so their moments are not needed)
    Fc = F if F is not None else moments(f[cells], I[cells], xi, w, om, wo, dim, model)
    src, srcR, rate, rateR = relaxation_source(Fc, f[cells], I[cells], wl)
    umag = np.sqrt(np.sum(Fc["u"] ** 2, axis=1))
    inv_dt = (umag + mdl.sound_speed(Fc["T_t"])) / (solver.cfl_meso * geo.dx[cells])

    slopes, pslopes = {}, {}

    def face_value(j, xf, which):
        """Reconstructed value of cell j at face point xf (order 2), else the cell value."""
        q = f if which == "gas" else I
        if order == 1:
            return q[j]
        cache = slopes if which == "gas" else pslopes
        if j not in cache:
            cache[j] = limited_slope(geo, j, q, K)
        grad, phi = cache[j]
        d = np.zeros(q[j].shape)
        dx = geo.delta(xf - geo.xc[j])
        for a in range(dim):
            d = d + grad[a] * dx[a]
        return q[j] + phi * d

    V = xi.shape[0]
    res = np.zeros((len(cells), V, 4))
    dg = np.zeros((len(cells), V))
    resR = np.zeros((len(cells), om.shape[0]))
    dR = np.zeros((len(cells), om.shape[0]))
    offdiag = []
    for k, i in enumerate(cells):
        r = src[k].copy()
        rR = srcR[k].copy()
        d = np.full(V, inv_dt[k] + rate[k])
        dr_ = np.full(om.shape[0], inv_dt[k] + rateR[k])
        od = []
        for nb, n, S, xf in geo.cell_faces[i]:
            xn = xi[:, :dim] @ n
            on = om[:, :dim] @ n
            xp, xm = np.maximum(xn, 0.0), np.minimum(xn, 0.0)
            op, omn = np.maximum(on, 0.0), np.minimum(on, 0.0)
            if nb >= 0:
                fL, fR = face_value(i, xf, "gas"), face_value(nb, xf, "gas")
                IL, IR = face_value(i, xf, "ph"), face_value(nb, xf, "ph")
                od.append((nb, S * xm / geo.vol[i], S * omn / geo.vol[i]))
            else:
                patch = mesh.patches[-1 - nb]
                if patch.kind == SYMMETRY:
                    # specular reflection: what enters with xi is what leaves with its mirror image
                    fL, fR = f[i], f[i][reflection_index(xi[:, :dim], n)]
                    IL, IR = I[i], I[i][reflection_index(om, np.pad(n, (0, 3 - dim)))]   # directions in 3-D
                else:
                    rw = wall_density(geo, f[i, :, 0], xi, w, dim, patch, n) if patch.kind == WALL else 1.0
                    fL, fR = f[i], incoming_gas(patch, rw, xi, dim, model)
                    IL, IR = I[i], incoming_photon(patch, model, om.shape[0])
            r -= (S / geo.vol[i]) * (xp[:, None] * fL + xm[:, None] * fR)
            rR -= (S / geo.vol[i]) * (op * IL + omn * IR)
            d += S * xp / geo.vol[i]
            dr_ += S * op / geo.vol[i]
        res[k], dg[k], resR[k], dR[k] = r, d, rR, dr_
        offdiag.append(od)

    return res, dg, resR, dR, offdiag


def kinetic_sweep(f, I, wl, geo=None, cells=None, relax_block=1, F=None):
    """One implicit kinetic step (Eq. dis_micro) for the gas planes and photons.

    For every cell i and discrete velocity (photon direction):
      r_i = (g_i - f_i)/tau_i + s_i - (1/V_i) sum_faces S (xi_n^+ f_L + xi_n^- f_R)
      d_i = 1/dt_i + 1/tau_i + (1/V_i) sum_faces S xi_n^+
    with the photon relaxation rate k_eff in place of 1/tau, g_R = sigma_R T_v^4/pi,
    and the radiative sink s = -(f0/rho) k_eff (4 sigma_R T_v^4 - int I dOmega) in
    the f2 equation.  Point relaxation: relax_block = 1 is Jacobi (neighbours keep
    their previous iterate); relax_block = B > 1 runs a forward and a backward
    Gauss-Seidel sweep inside each block of B consecutive cells (B = n_cells is the
    paper's natural-order symmetric sweep).

    With wl.solver.positivity = theta > 0 every value of the result is at least theta times
    its value in f (or I).

    Returns (f_new, I_new) for ``cells`` (default: all cells, in order).
    """
    mesh, model, solver = wl.mesh, wl.model, wl.solver
    dim, xi, w, om, wo = mesh.dim, wl.xi, wl.w, wl.omega, wl.wo
    geo = geo or Geometry(mesh)
    nc = mesh.n_cells
    cells = np.arange(nc) if cells is None else np.asarray(cells)
    if relax_block != 1:
        blocks = sorted(set(int(c) // relax_block for c in cells))
        want = np.concatenate([np.arange(b * relax_block, min((b + 1) * relax_block, nc)) for b in blocks])
        if len(want) != len(cells) or np.any(np.sort(cells) != want):
            raise ValueError("block relaxation needs whole blocks of consecutive cells")
        cells = want
    res, dg, resR, dR, offdiag = kinetic_residual(f, I, wl, geo, cells, F)

    if relax_block == 1:
        df = res / dg[..., None]
        dI = resR / dR
    else:
        pos = {int(c): k for k, c in enumerate(cells)}
        df = np.zeros_like(res)
        dI = np.zeros_like(resR)
        for b in sorted(set(int(c) // relax_block for c in cells)):
            b0, b1 = b * relax_block, min((b + 1) * relax_block, nc)
            for i in range(b0, b1):                               # forward
                k = pos[i]
                acc, accR = res[k].copy(), resR[k].copy()
                for j, a, aR in offdiag[k]:
                    if b0 <= j < i:
                        acc -= a[:, None] * df[pos[j]]
                        accR -= aR * dI[pos[j]]
                df[k], dI[k] = acc / dg[k][:, None], accR / dR[k]
            for i in range(b1 - 1, b0 - 1, -1):                   # backward
                k = pos[i]
                for j, a, aR in offdiag[k]:
                    if i < j < b1:
                        df[k] -= a[:, None] * df[pos[j]] / dg[k][:, None]
                        dI[k] -= aR * dI[pos[j]] / dR[k]
    f_new, I_new = f[cells] + df, I[cells] + dI
    theta = float(getattr(solver, "positivity", 0.0))
    if theta > 0.0:
        # positivity bound of the implicit update (an extension; 0 is the paper's scheme): no
        # value falls below theta times its previous value.  At a steady state df = 0, so the
        # fixed point is unchanged.
        f_new = np.maximum(f_new, theta * f[cells])
        I_new = np.maximum(I_new, theta * I[cells])
    return f_new, I_new
