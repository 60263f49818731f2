"""Pins that tie the kinetic oracle to the Fourier stability analysis of Section 4.

On a uniform periodic row of cells (first-order upwind transport, so the row is exactly
periodic) the conventional iteration with the transport solved exactly (the sweeps of
``kinetic_sweep`` repeated with the fields held fixed until they stop changing) is, for
small perturbations of the global equilibrium, a linear map of one Fourier mode's
macroscopic amplitudes onto the next iteration's.  That map is measured here from the
oracle's own moments, reference distributions, relaxation sources and sweeps (central
differences of seeded perturbations), and compared element by element with the
eigen-equation of Section 4 (Eq. eigenfunction_cis) evaluated with the same discrete
velocities and photon directions and the upwind symbol of the row (oracle/fourier.py,
``transport_symbol``).  A dropped or misplaced term in either oracle, a wrong relaxation
rate, Shakhov factor or radiative coupling, breaks the agreement.

The decay factor per iteration (the spectral radius) then follows for both, and the
upwind symbol's factor approaches the continuous analysis of the paper as the cells
shrink.
"""
import math

import numpy as np
import pytest

import gsis_inputs as gi
from gsis_inputs import quadrature as Q
from oracle import fourier as FO
from oracle import kinetic as K

# longitudinal amplitudes of a mode along x: the 1-D problem carries these nine
LONG = [FO.RHO, FO.UX, FO.TT, FO.TR, FO.TV, FO.ER, FO.QT, FO.QR, FO.QV]


def _setup(kn_theta, ratio, sigma_R, n_cells, n_gh=48, n_mu=16):
    theta = kn_theta                                   # Kn = 1
    L = 2.0 * math.pi / theta
    mesh = gi.mesh.ring_1d(n_cells, L)
    xi, w = Q.gauss_hermite_1d(n_gh)
    om, wo = Q.gauss_legendre_slab(n_mu)
    model = gi.workloads.ModelParams(d_r=2.0, d_v=1.0, Z_r=2.67, Z_v=26.7, Kn=1.0, Kn_p=1.0 / ratio,
                                     sigma_R=sigma_R)
    solver = gi.workloads.SolverParams(precision="fp64", order=1, relax_block=n_cells)
    wl = gi.workloads.Workload("ring", mesh, xi, w, om, wo, model, solver)
    p = FO.Params(ratio, sigma_R, d_r=2.0, d_v=1.0, Z_r=2.67, Z_v=26.7)
    grid = FO.velocity_grid(x_nodes=(xi[:, 0], w))
    return wl, p, grid, theta


def _base_fields(n):
    M = gi.fields.uniform_fields(n)
    return M


def _fields(M, wl, comp, amp):
    """Fields of the record M with amplitude ``amp`` (per cell) added to the Fourier
    component ``comp``."""
    F = K.fields_from_record(M, wl.model.sigma_R)
    key = {FO.RHO: ("rho", None), FO.UX: ("u", 0), FO.TT: ("T_t", None), FO.TR: ("T_r", None),
           FO.TV: ("T_v", None), FO.ER: ("e_R", None), FO.QT: ("q_t", 0), FO.QR: ("q_r", 0),
           FO.QV: ("q_v", 0)}[comp]
    if key[1] is None:
        F[key[0]] = F[key[0]] + amp
    else:
        F[key[0]][:, key[1]] += amp
    return F


def _exact_transport(F, wl, geo, f, I):
    """Distributions that the sweeps reach with the fields held at F (the transport with
    relaxation to the reference distribution of F solved exactly)."""
    scale = np.abs(f).max()
    for _ in range(600):
        fn, In = K.kinetic_sweep(f, I, wl, geo=geo, F=F, relax_block=wl.mesh.n_cells)
        d = max(np.abs(fn - f).max() / scale, np.abs(In - I).max() / max(np.abs(I).max(), 1e-300))
        f, I = fn, In
        if d < 1e-15:
            return f, I
    raise AssertionError("transport sweeps did not converge")


def _amplitudes(F, theta, x):
    """Complex amplitude of e^{i theta x} of each longitudinal field: F(x) = Re(a e^{i theta x})."""
    e = np.exp(-1j * theta * x) * (2.0 / x.shape[0])
    vals = {FO.RHO: F["rho"], FO.UX: F["u"][:, 0], FO.TT: F["T_t"], FO.TR: F["T_r"], FO.TV: F["T_v"],
            FO.ER: F["e_R"], FO.QT: F["q_t"][:, 0], FO.QR: F["q_r"][:, 0], FO.QV: F["q_v"][:, 0]}
    return np.array([vals[c] @ e for c in LONG])


def _measured_map(wl, theta, eps=1e-6, phase=0.0):
    """Columns: the next iteration's amplitudes per unit amplitude e^{i phase} of each
    longitudinal component, by central differences."""
    geo = K.Geometry(wl.mesh)
    x = wl.mesh.cell_centroid[:, 0]
    M = _base_fields(wl.mesh.n_cells)
    F0 = K.fields_from_record(M, wl.model.sigma_R)
    f0 = K.equilibrium_planes(F0, wl.xi, 1, wl.model)
    I0 = K.photon_equilibrium(F0["T_R"], wl.omega.shape[0], wl.model.sigma_R)
    wave = np.cos(theta * x + phase)
    A = np.zeros((len(LONG), len(LONG)), complex)
    for n, comp in enumerate(LONG):
        amps = []
        for sgn in (1.0, -1.0):
            F = _fields(M, wl, comp, sgn * eps * wave)
            f, I = _exact_transport(F, wl, geo, f0, I0)
            G = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, 1, wl.model)
            amps.append(_amplitudes(G, theta, x))
        A[:, n] = (amps[0] - amps[1]) / (2.0 * eps) * np.exp(-1j * phase)
    return A


CASES = [(0.3, 1.0, 0.01), (1.0, 0.1, 0.1), (0.1, 10.0, 0.005)]


@pytest.mark.parametrize("kn_theta,ratio,sigma_R", CASES)
def test_kinetic_oracle_iteration_equals_the_fourier_matrix(kn_theta, ratio, sigma_R):
    n_cells = 24
    wl, p, grid, theta = _setup(kn_theta, ratio, sigma_R, n_cells)
    h = theta * (2.0 * math.pi / theta) / n_cells
    A = _measured_map(wl, theta)
    C = FO.cis_matrix(p, kn_theta, grid, h=h, photons=(wl.omega[:, 0], wl.wo))[np.ix_(LONG, LONG)]
    assert np.abs(C).max() > 0.1
    err = np.abs(A - C).max()
    assert err < 1e-7 * np.abs(C).max(), "max |A - C| = %.3e" % err
    rho_m = np.abs(np.linalg.eigvals(A)).max()
    rho_f = np.abs(np.linalg.eigvals(C)).max()
    assert abs(rho_m - rho_f) < 1e-7


def test_the_map_does_not_depend_on_the_phase_of_the_mode():
    """Translation invariance of the periodic row: a sine-phase perturbation gives the same
    complex map as a cosine-phase one."""
    wl, p, grid, theta = _setup(0.3, 1.0, 0.01, 24)
    A0 = _measured_map(wl, theta)
    A1 = _measured_map(wl, theta, phase=0.7)
    assert np.abs(A0 - A1).max() < 1e-8 * np.abs(A0).max()


@pytest.mark.parametrize("kn_theta,ratio,sigma_R", CASES)
def test_upwind_decay_factor_tends_to_the_continuous_one(kn_theta, ratio, sigma_R):
    """The spectral radius with the upwind symbol approaches that of the paper's continuous
    analysis at first order in the cell size (same velocity and direction sets)."""
    wl, p, grid, theta = _setup(kn_theta, ratio, sigma_R, 24)
    ph = (wl.omega[:, 0], wl.wo)
    rho_c = FO.spectral_radius_cis(p, kn_theta, grid, h=None, photons=ph)
    errs = []
    for n in (24, 96, 384):
        rho_h = FO.spectral_radius_cis(p, kn_theta, grid, h=2.0 * math.pi / n, photons=ph)
        errs.append(abs(rho_h - rho_c))
    assert errs[2] < errs[1] < errs[0]
    assert 2.5 < errs[0] / errs[1] < 6.0 and 2.5 < errs[1] / errs[2] < 6.0   # first order: 4x per 4x cells
    # the discrete direction set agrees with the exact sphere integral of the paper's analysis
    assert abs(rho_c - FO.spectral_radius_cis(p, kn_theta, grid)) < 1e-6


# ---------------------------------------------------------------------------- GSIS
def _solve_synthetic(W0, faces, hot, wl, newton=3):
    """W with R(W) = 0 (the synthetic equations with the high-order terms held fixed), by
    Newton steps on a finite-difference Jacobian of the oracle's residual.  On a periodic
    row the Jacobian is singular along the uniform states (total mass, momentum and energy
    are not fixed by the steady equations); the least-squares step of least norm keeps
    their totals, as the solver's point relaxation does for a single Fourier mode."""
    from oracle import macro as MA
    W = W0.copy()
    n, m = W.shape
    for _ in range(newton):
        R0 = MA.residual(W, faces, hot, wl).ravel()
        J = np.empty((n * m, n * m))
        for k in range(n * m):
            dW = np.zeros(n * m)
            st = 1e-7 * max(1.0, abs(W.ravel()[k]))
            dW[k] = st
            J[:, k] = (MA.residual(W + dW.reshape(n, m), faces, hot, wl).ravel() - R0) / st
        W = W + np.linalg.lstsq(J, -R0, rcond=1e-11)[0].reshape(n, m)
    return W


def _measured_gsis_map(wl, theta, eps=1e-6):
    """One GSIS step of the oracle (Section 3) on the periodic row, with the transport and
    the synthetic equations solved exactly: kinetic half step, moments and high-order terms
    (macro.high_order_terms), synthetic solve, synchronisation f + f_eq(M^{k+1}) -
    f_eq(M^{k+1/2}) (and likewise I), moments of the result."""
    from oracle import macro as MA
    geo = K.Geometry(wl.mesh)
    faces = MA.Faces(geo)
    x = wl.mesh.cell_centroid[:, 0]
    M = _base_fields(wl.mesh.n_cells)
    F0 = K.fields_from_record(M, wl.model.sigma_R)
    f0 = K.equilibrium_planes(F0, wl.xi, 1, wl.model)
    I0 = K.photon_equilibrium(F0["T_R"], wl.omega.shape[0], wl.model.sigma_R)
    wave = np.cos(theta * x)
    A = np.zeros((len(LONG), len(LONG)), complex)
    nO = wl.omega.shape[0]
    for n, comp in enumerate(LONG):
        amps = []
        for sgn in (1.0, -1.0):
            F = _fields(M, wl, comp, sgn * eps * wave)
            f, I = _exact_transport(F, wl, geo, f0, I0)
            Fh = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, 1, wl.model)
            hot = MA.high_order_terms(faces, Fh, MA.kinetic_boundary_flux(faces, f, I, wl), wl)
            W = _solve_synthetic(MA.conservative(Fh, 1, wl.model), faces, hot, wl)
            Fn = MA.fields_from_W(W, 1, wl.model)
            fn = f + K.equilibrium_planes(Fn, wl.xi, 1, wl.model) - K.equilibrium_planes(Fh, wl.xi, 1, wl.model)
            In = I + (K.photon_equilibrium(Fn["T_R"], nO, wl.model.sigma_R)
                      - K.photon_equilibrium(Fh["T_R"], nO, wl.model.sigma_R))
            G = K.moments(fn, In, wl.xi, wl.w, wl.omega, wl.wo, 1, wl.model)
            amps.append(_amplitudes(G, theta, x))
        A[:, n] = (amps[0] - amps[1]) / (2.0 * eps)
    return A


@pytest.mark.parametrize("kn_theta,ratio,sigma_R,sizes,max_rich", [
    (1.0, 0.1, 0.1, (32, 64), 0.008),        # case B
    (0.3, 1.0, 0.01, (24, 48), 0.045),       # case A
])
def test_gsis_iteration_tends_to_the_fourier_gsis_matrix(kn_theta, ratio, sigma_R, sizes, max_rich):
    """The oracle's GSIS step on a periodic row (exact transport, exact synthetic solve)
    against the Section-4 GSIS matrices (Eqs. eigenfunction_gsis, eigenfunction_gsis_S) with
    the same velocities, directions and upwind symbol in the kinetic half step, and with the
    heat fluxes that the algorithm's synchronisation keeps: those of the half step
    (oracle/fourier.py, ``gsis_algorithm_matrix``).  The synthetic equations are finite
    volume on the cells and continuous in the analysis; the Rusanov dissipation of their
    convective flux is first order in the cell size, their central terms second order.  So
    the difference falls at first order, and its Richardson extrapolation 2 E(2n) - E(n)
    is small.  A 5 % slip of the viscosity or the conductivity, or the stress or a heat flux
    dropped from the high-order terms, multiplies that extrapolated difference by 2 to 60."""
    E, rho = {}, {}
    for n_cells in sizes:
        wl, p, grid, theta = _setup(kn_theta, ratio, sigma_R, n_cells)
        h = 2.0 * math.pi / n_cells
        ph = (wl.omega[:, 0], wl.wo)
        A = _measured_gsis_map(wl, theta)
        G = FO.gsis_algorithm_matrix(p, kn_theta, grid, h=h, photons=ph)[np.ix_(LONG, LONG)]
        C = FO.cis_matrix(p, kn_theta, grid, h=h, photons=ph)[np.ix_(LONG, LONG)]
        # the synchronisation adds equilibria only: the heat-flux rows are the CIS step's
        assert np.abs(A[6:] - C[6:]).max() < 1e-7 * np.abs(C).max()
        E[n_cells] = A - G
        rho[n_cells] = (np.abs(np.linalg.eigvals(A)).max(), np.abs(np.linalg.eigvals(G)).max())
    a, b = sizes
    ea, eb = np.abs(E[a]).max(), np.abs(E[b]).max()
    assert 1.5 < ea / eb < 2.4, "difference falls by %.2f per halving of the cells" % (ea / eb)
    rich = np.abs(2.0 * E[b] - E[a]).max()
    assert rich < max_rich, "extrapolated difference %.3e" % rich
    # decay factors: the extrapolated discrete factor against the analysis
    ext_A = 2.0 * rho[b][0] - rho[a][0]
    ext_G = 2.0 * rho[b][1] - rho[a][1]
    assert abs(ext_A - ext_G) < 2.0 * max_rich
