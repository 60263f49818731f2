"""Pins of the oracle's kinetic half against what the paper and mathematics fix.

Each test checks a property that a plausible slip in the oracle (a dropped term,
a wrong sign, a transposed index) would break: quadrature closed forms, mesh
closure, the conservation built into the reference distributions, the heat-flux
relaxation rates that define the matrix A, the hidden-velocity reduction against
a full 3-D evaluation, the equilibrium fixed point, the gas-photon energy balance
and the free-molecular closed form of a slab.
"""
import numpy as np
import pytest

import gsis_inputs as gi
from gsis_inputs import quadrature as Q
from oracle import kinetic as K
from oracle import model as mdl


def _fields(n, dim, seed, u_scale=0.4, q_scale=0.1, sigma_R=0.01):
    M = gi.fields.random_macro_fields(n, dim, seed, u_scale=u_scale, q_scale=q_scale)
    return K.fields_from_record(M, sigma_R)


# ---------------------------------------------------------------- quadratures and meshes
def test_gauss_hermite_moments():
    xi, w = Q.gauss_hermite_1d(32)
    for T in (0.7, 1.0, 1.5):
        f = np.exp(-xi[:, 0] ** 2 / (2 * T)) / np.sqrt(2 * np.pi * T)
        assert abs(w @ f - 1.0) < 1e-12
        assert abs(w @ (xi[:, 0] ** 2 * f) - T) < 1e-12
        assert abs(w @ (xi[:, 0] ** 4 * f) - 3 * T * T) < 1e-11


def test_gauss_hermite_against_golub_welsch():
    # independent route: eigenvalues of the Jacobi matrix of probabilists' Hermite polynomials
    n = 32
    J = np.diag(np.sqrt(np.arange(1, n)), 1)
    lam, vec = np.linalg.eigh(J + J.T)
    w_gw = np.sqrt(2 * np.pi) * vec[0] ** 2 * np.exp(lam ** 2 / 2)
    xi, w = Q.gauss_hermite_1d(n)
    order = np.argsort(xi[:, 0])
    assert np.allclose(xi[order, 0], np.sort(lam), atol=1e-12)
    assert np.allclose(w[order] * np.exp(-xi[order, 0] ** 2 / 2),
                       (w_gw * np.exp(-lam ** 2 / 2))[np.argsort(lam)], rtol=1e-9, atol=1e-14)  # eigenvector entries carry absolute error


def test_newton_cotes_38_exact_for_cubics():
    x, w = Q.newton_cotes_38_weights(28, 2.0)
    for p in range(4):
        exact = (2.0 ** (p + 1) - (-2.0) ** (p + 1)) / (p + 1)
        assert abs(w @ x ** p - exact) < 1e-12


def test_photon_product_sums():
    for npol, naz in ((8, 8), (8, 12), (8, 16)):
        om, wo = Q.photon_product(npol, naz)
        assert abs(wo.sum() - 4 * np.pi) < 1e-13
        assert np.abs(om.T @ wo).max() < 1e-13
        assert np.abs((om * wo[:, None]).T @ om - 4 * np.pi / 3 * np.eye(3)).max() < 1e-13
    om, wo = Q.gauss_legendre_slab(16)
    assert abs(wo.sum() - 4 * np.pi) < 1e-13 and abs(om[:, 0] @ wo) < 1e-13
    assert abs((om[:, 0] ** 2) @ wo - 4 * np.pi / 3) < 1e-13


@pytest.mark.parametrize("mk", [lambda: gi.mesh.cavity_triangles(12, seed=5),
                                lambda: gi.mesh.slab_1d(10),
                                lambda: gi.mesh.cylinder_ogrid(24, 8),
                                lambda: gi.mesh.channel_triangles(8, seed=3),
                                lambda: gi.mesh.ring_1d(12, 3.0)])
def test_mesh_closure(mk):
    m = mk()
    acc = np.zeros((m.n_cells, m.dim))
    np.add.at(acc, m.face_owner, m.face_normal * m.face_area[:, None])
    inner = m.face_nbr >= 0
    np.add.at(acc, m.face_nbr[inner], -m.face_normal[inner] * m.face_area[inner, None])
    assert np.abs(acc).max() < 1e-13
    assert np.allclose(np.linalg.norm(m.face_normal, axis=1), 1.0)


def test_periodic_meshes_have_minimal_image_neighbours():
    """On the periodic channel and ring every interior face's normal points from owner to
    neighbour along the minimal-image centroid difference (the seam faces included), the
    neighbours are a cell width apart, and the cells tile the domain."""
    for m, h in ((gi.mesh.channel_triangles(8, seed=3), 1.0 / 8), (gi.mesh.ring_1d(12, 3.0), 3.0 / 12)):
        geo = K.Geometry(m)
        inner = m.face_nbr >= 0
        d = geo.delta(m.cell_centroid[m.face_nbr[inner], :m.dim] - m.cell_centroid[m.face_owner[inner], :m.dim])
        raw = m.cell_centroid[m.face_nbr[inner], 0] - m.cell_centroid[m.face_owner[inner], 0]
        assert np.all(np.sum(d * m.face_normal[inner], axis=1) > 0.0)
        assert np.linalg.norm(d, axis=1).max() < 1.5 * h
        assert np.abs(raw).max() > 0.5 * m.period          # the seam faces are there
        total = 1.0 if m.dim == 2 else m.period
        assert abs(m.cell_volume.sum() - total) < 1e-12


def test_cavity_volume():
    assert abs(gi.mesh.cavity_triangles(30, seed=2).cell_volume.sum() - 1.0) < 1e-12


# ---------------------------------------------------------------- reference distributions
def _fine_grid(dim, n=48, L=11.0):
    return Q.trapezoid_nd(n, L, dim)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_reference_conserves_mass_momentum_energy(dim):
    model = gi.workloads.ModelParams()
    xi, w = _fine_grid(dim, n=64, L=13.0)
    F = _fields(5, dim, seed=11)
    g = K.reference_planes(F, xi, dim, model)
    rho, u = F["rho"], F["u"]
    assert np.allclose(g[..., 0] @ w, rho, rtol=1e-10)
    for a in range(dim):
        assert np.allclose((g[..., 0] * w) @ xi[:, a], rho * u[:, a], rtol=1e-10, atol=1e-12)
    c2 = np.sum((xi[None, :, :dim] - u[:, None, :dim]) ** 2, axis=-1)
    E = 0.5 * ((c2 * g[..., 0]) @ w + g[..., 1] @ w) + g[..., 2] @ w + g[..., 3] @ w
    E_ref = rho * (1.5 * F["T_t"] + 0.5 * model.d_r * F["T_r"] + 0.5 * model.d_v * F["T_v"])
    assert np.allclose(E, E_ref, rtol=1e-10)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_reference_heat_flux_relaxation_rates(dim):
    """The first-order moments of g reproduce the relaxation law
    dq/dt = -(p_t/mu) A q with mu = p_t tau (Section 2.1):
    int c (c^2/2) g0 = q_t - (A q)_t,  int c g1 = q_r - (A q)_r,  int c g2 = q_v - (A q)_v."""
    model = gi.workloads.ModelParams()
    xi, w = _fine_grid(dim, n=64, L=13.0)
    F = _fields(4, dim, seed=12)
    g = K.reference_planes(F, xi, dim, model)
    A = mdl.mason_monchick_A(model.d_r, model.d_v, model.Z_r, model.Z_v, model.Sc)
    c = xi[None, :, :dim] - F["u"][:, None, :dim]
    c2 = np.sum(c * c, axis=-1)
    q = np.stack([F["q_t"], F["q_r"], F["q_v"]], 1)              # [n, 3 modes, 3]
    Aq = np.einsum("ij,njd->nid", A, q)
    for a in range(dim):
        qt = 0.5 * (c[..., a] * (c2 * g[..., 0] + g[..., 1])) @ w
        qr = (c[..., a] * g[..., 2]) @ w
        qv = (c[..., a] * g[..., 3]) @ w
        assert np.allclose(qt, q[:, 0, a] - Aq[:, 0, a], rtol=1e-9, atol=1e-11)
        assert np.allclose(qr, q[:, 1, a] - Aq[:, 1, a], rtol=1e-9, atol=1e-11)
        assert np.allclose(qv, q[:, 2, a] - Aq[:, 2, a], rtol=1e-9, atol=1e-11)


def test_mason_monchick_gives_prandtl_two_thirds_without_internal_modes():
    # Z_r, Z_v -> infinity: A_tt -> 2/3, the Shakhov Prandtl number of the translational mode
    A = mdl.mason_monchick_A(2.0, 1.16, 1e30, 1e30, 5.0 / 6.0)
    assert abs(A[0, 0] - 2.0 / 3.0) < 1e-15 and abs(A[1, 1] - 5.0 / 6.0) < 1e-15
    assert np.abs(A[[0, 0, 1, 2], [1, 2, 0, 0]]).max() < 1e-29


@pytest.mark.parametrize("dim_lo", [1, 2])
def test_reduction_matches_higher_dimensional_evaluation(dim_lo):
    """Reduced planes (dim_lo) equal the (dim_lo+1)-dimensional reference distribution
    integrated over the extra velocity component (reading of the paper's reduction)."""
    model = gi.workloads.ModelParams()
    dim_hi = dim_lo + 1
    n1, L = 56, 12.0
    x1, w1 = Q.trapezoid_weights(n1, L)
    xi_lo, w_lo = Q.trapezoid_nd(n1, L, dim_lo)
    xi_hi, _ = Q.trapezoid_nd(n1, L, dim_hi)
    F = _fields(3, dim_lo, seed=13)
    g_lo = K.reference_planes(F, xi_lo, dim_lo, model)
    g_hi = K.reference_planes(F, xi_hi, dim_hi, model)            # q, u have no extra component
    g_hi = g_hi.reshape(3, -1, n1, 4)                            # last velocity axis is the extra one
    xe = x1[None, None, :]
    red0 = (g_hi[..., 0] * w1).sum(-1)
    red1 = (g_hi[..., 1] * w1).sum(-1) + (xe ** 2 * g_hi[..., 0] * w1).sum(-1)
    red2 = (g_hi[..., 2] * w1).sum(-1)
    red3 = (g_hi[..., 3] * w1).sum(-1)
    scale = np.abs(g_lo).max()
    for p, red in enumerate((red0, red1, red2, red3)):
        assert np.abs(red - g_lo[..., p]).max() < 1e-10 * scale


def test_moments_of_maxwellian():
    model = gi.workloads.ModelParams()
    xi, w = _fine_grid(2, n=72, L=12.0)
    om, wo = Q.photon_product(8, 8)
    M = gi.fields.random_macro_fields(4, 2, seed=14, u_scale=0.5)
    F = K.fields_from_record(M, model.sigma_R)
    f = K.equilibrium_planes(F, xi, 2, model)
    I = K.photon_equilibrium(F["T_R"], om.shape[0], model.sigma_R)
    G = K.moments(f, I, xi, w, om, wo, 2, model)
    for k in ("rho", "T_t", "T_r", "T_v", "T_R"):
        assert np.allclose(G[k], F[k], rtol=1e-11)
    assert np.allclose(G["u"], F["u"], atol=1e-11)
    for k in ("q_t", "q_r", "q_v", "q_R"):
        assert np.abs(G[k]).max() < 1e-11
    assert np.abs(G["sigma"]).max() < 1e-11


def test_gas_photon_energy_exchange_balances():
    """int (f2 source) dxi + int (photon source) dOmega = 0 up to the gas relaxation,
    which conserves energy by itself (Eq. kinetic_equation, Eq. macroscopic_equation)."""
    wl = gi.workloads.cavity(n_side=2, n_v=40, Kn_p=1.0)
    wl.xi, wl.w = _fine_grid(2, n=64, L=12.0)
    M = gi.fields.random_macro_fields(wl.mesh.n_cells, 2, seed=15, u_scale=0.3)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 2, 2.0, 1.16, wl.model.sigma_R, seed=16)
    F = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, 2, wl.model)
    src, srcR, _, _ = K.relaxation_source(F, f, I, wl)
    c2 = np.sum((wl.xi[None, :, :2] - F["u"][:, None, :2]) ** 2, axis=-1)
    gas = 0.5 * ((c2 * src[..., 0]) @ wl.w + src[..., 1] @ wl.w) + src[..., 2] @ wl.w + src[..., 3] @ wl.w
    ph = srcR @ wl.wo
    exch = ph.copy()
    assert np.abs(exch).max() > 1e-4                              # the exchange is not trivially zero
    assert np.allclose(gas + ph, 0.0, atol=1e-9 * np.abs(exch).max())   # quadrature error ~1e-10
    # mass and momentum of the gas source vanish too
    assert np.abs(src[..., 0] @ wl.w).max() < 1e-10


# ---------------------------------------------------------------- sweep
def test_lsq_gradient_exact_for_linear_fields():
    m = gi.mesh.cavity_triangles(8, seed=3)
    geo = K.Geometry(m)
    q = 0.3 + 1.7 * m.cell_centroid[:, 0] - 0.9 * m.cell_centroid[:, 1]
    for i in range(m.n_cells):
        if len(geo.interior_neighbours(i)) >= 2:
            grad, _ = K.limited_slope(geo, i, q, 5.0)
            assert np.allclose(grad, [1.7, -0.9], atol=1e-12)


def test_venkatakrishnan_limits():
    assert abs(K.venkatakrishnan(1e8, 1.0, 0.0) - 1.0) < 1e-7    # far from extrema: unlimited
    assert abs(K.venkatakrishnan(0.0, 1.0, 0.0)) < 1e-15         # at a local extremum: first order
    assert abs(K.venkatakrishnan(2.0, 1.0, 0.0) - 1.0) < 1e-15   # (4+4)/(4+2+2)


@pytest.mark.parametrize("order", [1, 2])
def test_uniform_equilibrium_is_a_fixed_point(order):
    wl = gi.workloads.with_solver(gi.workloads.cavity(n_side=4, n_v=28, u_lid=0.0, T_lid=1.3), order=order)
    for p in wl.mesh.patches:
        p.T_t = 1.3
    M = gi.fields.uniform_fields(wl.mesh.n_cells, rho=0.8, T=1.3)
    F = K.fields_from_record(M, wl.model.sigma_R)
    f = K.equilibrium_planes(F, wl.xi, 2, wl.model)
    I = K.photon_equilibrium(F["T_R"], wl.omega.shape[0], wl.model.sigma_R)
    # the discrete temperature differs from 1.3 by the grid's quadrature error; take the
    # walls at the discrete value so that only round-off remains
    G = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, 2, wl.model)
    fn, In = K.kinetic_sweep(f, I, wl)
    assert np.abs(fn - f).max() < 2e-5 * np.abs(f).max()        # quadrature-level
    assert np.abs(In - I).max() < 1e-13 * np.abs(I).max()
    # and exactly with a Gauss-Hermite grid on a slab where quadrature is exact
    wls = gi.workloads.with_solver(gi.workloads.slab(n_cells=8, T_left=1.0, T_right=1.0), order=order)
    Ms = gi.fields.uniform_fields(8, rho=1.1, T=1.0)
    Fs = K.fields_from_record(Ms, wls.model.sigma_R)
    fs = K.equilibrium_planes(Fs, wls.xi, 1, wls.model)
    Is = K.photon_equilibrium(Fs["T_R"], wls.omega.shape[0], wls.model.sigma_R)
    fsn, Isn = K.kinetic_sweep(fs, Is, wls)
    assert np.abs(fsn - fs).max() < 1e-13 * np.abs(fs).max()
    assert np.abs(Isn - Is).max() < 1e-13 * np.abs(Is).max()


def test_free_molecular_slab_closed_form():
    """Kn -> infinity: the steady discrete solution between diffuse walls is uniform,
    half-range wall Maxwellians with n_R/n_L fixed by zero net mass flux."""
    wl = gi.workloads.with_model(gi.workloads.slab(n_cells=12, Kn=1e9, Kn_p=1e9, sigma_R=0.0),
                                 sigma_R=0.0)
    # a vanishing pseudo-time term makes each symmetric sweep an exact transport solve;
    # otherwise its lag feeds the neutral mode of two explicitly coupled walls
    wl = gi.workloads.with_solver(wl, order=1, cfl_meso=1e15)
    TL, TR = 1.0, 1.5
    M = gi.fields.uniform_fields(12, T=1.2)
    F = K.fields_from_record(M, 1.0)
    f = K.equilibrium_planes(F, wl.xi, 1, wl.model)
    I = np.zeros((12, wl.omega.shape[0]))
    for _ in range(6):
        f, I = K.kinetic_sweep(f, I, wl, relax_block=12)
    xi = wl.xi[:, 0]
    FL = np.exp(-xi ** 2 / (2 * TL)) / np.sqrt(2 * np.pi * TL)
    FR = np.exp(-xi ** 2 / (2 * TR)) / np.sqrt(2 * np.pi * TR)
    JL = np.sum(np.where(xi > 0, wl.w * xi * FL, 0.0))
    JR = -np.sum(np.where(xi < 0, wl.w * xi * FR, 0.0))
    nL = f[0, xi > 0, 0][0] / FL[xi > 0][0]
    closed = np.where(xi > 0, nL * FL, nL * JL / JR * FR)
    for i in range(12):
        assert np.allclose(f[i, :, 0], closed, rtol=1e-9, atol=1e-14)
        assert np.allclose(f[i, :, 2], np.where(xi > 0, TL, TR) * wl.model.d_r / 2 * closed, rtol=1e-9,
                           atol=1e-14)
    # internal temperature of a free-molecular slab: sqrt(T_L T_R) (continuous half-range
    # integrals; the Gauss-Hermite grid integrates half ranges only approximately)
    G = K.moments(f[:1], I[:1], wl.xi, wl.w, wl.omega, wl.wo, 1, wl.model)
    assert abs(G["T_r"][0] - np.sqrt(TL * TR)) < 5e-3
