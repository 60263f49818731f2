"""Oracle (test infrastructure only): linear Fourier stability analysis of Section 4.

The kinetic model is linearised about the global equilibrium (rho = T = 1, u = 0) with
continuous space, and the iteration error is a single Fourier mode exp(i theta x) with
theta along x.  With the 17 macroscopic perturbations
    alpha = [d rho, u_x, u_y, u_z, dT_t, dT_r, dT_v, de_R, q_t (3), q_r (3), q_v (3)],
one CIS step maps alpha to C alpha (Eq. eigenfunction_cis) and one GSIS step solves
e L alpha = R alpha (Eqs. eigenfunction_gsis, eigenfunction_gsis_S); the error decay factor
is the spectral radius of C or of L^-1 R.

Every quantity depends on Kn theta, Kn/Kn_p and sigma_R only; Kn = 1 is used.

Discrete space: on a uniform periodic row of cells of width dx, first-order upwinding
turns the transport symbol i a xi_x (continuous) into a |xi_x| (1 - exp(-i sgn(xi_x) h)) / h
with h = theta dx, which tends to i a xi_x as h -> 0 (``transport_symbol``).  With
``h`` given, ``cis_matrix`` uses that symbol for the gas and the photons; with the solver's
own velocity nodes (``velocity_grid(x_nodes=...)``) and photon directions it is the
iteration matrix of the discrete-velocity, finite-volume CIS step with exact transport
(tests/test_oracle_fourier_link_pins.py).  ``gsis_matrices`` takes the same options for
its kinetic half step; ``gsis_algorithm_matrix`` is the GSIS step with the heat fluxes
that the algorithm's synchronisation keeps, which the oracle's GSIS step on a periodic row
approaches at first order in the cell size (the same test file).

Velocity integrals: the kinetic responses are (polynomial x Gaussian) / (1 + i a xi_x)
with a = sqrt(2/pi) Kn theta.  They are evaluated on a tensor grid (dense trapezoid in
xi_x, Gauss-Hermite in xi_y, xi_z); the tests cross-check the xi_x integrals against the
plasma-dispersion (Faddeeva) closed form.  Photon integrals over the sphere use the closed
forms int dOmega / (1 + i b mu) = 4 pi arctan(b) / b and its first moment.

Readings:
  * the constitutive relations of the GSIS step take the full conductivity matrix
    kappa_gas = (sqrt(2/pi) Kn / 2) A^-1 diag(5, d_r, d_v) of Eq. (linear_constitutive)
    (the eigen-equations print one conductivity per mode, which is its diagonal);
  * kappa_R = Kn_p / 3 (photon diffusion).
Pins: tests/test_oracle_fourier_pins.py.
"""
from __future__ import annotations

import math

import numpy as np

from . import model as mdl

NM = 17
RHO, UX, TT, TR, TV, ER, QT, QR, QV = 0, 1, 4, 5, 6, 7, 8, 11, 14


class Params:
    def __init__(self, ratio, sigma_R, d_r=2.0, d_v=1.0, Z_r=2.67, Z_v=26.7, Sc=5.0 / 6.0):
        self.ratio = ratio            # Kn / Kn_p
        self.sigma_R = sigma_R
        self.d_r, self.d_v, self.Z_r, self.Z_v = d_r, d_v, Z_r, Z_v
        self.A = mdl.mason_monchick_A(d_r, d_v, Z_r, Z_v, Sc)


def velocity_grid(n_x=4001, L=12.0, n_t=8, x_nodes=None):
    """Tensor grid: trapezoid in xi_x on [-L, L] (or the given (nodes, weights) with
    sum w g(x) ~ int g dx), Gauss-Hermite (weight exp(-x^2/2)) in xi_y and xi_z.
    Returns (xi [n, 3], w [n]) with sum w g(xi) ~ int g."""
    if x_nodes is None:
        x = np.linspace(-L, L, n_x)
        wx = np.full(n_x, x[1] - x[0])
        wx[0] = wx[-1] = 0.5 * (x[1] - x[0])
    else:
        x, wx = (np.asarray(a, np.float64).ravel() for a in x_nodes)
    t, wt = np.polynomial.hermite_e.hermegauss(n_t)
    wt = wt * np.exp(0.5 * t * t)          # the integrands carry their own exp(-xi^2/2)
    X, Y, Z = np.meshgrid(x, t, t, indexing="ij")
    W = wx[:, None, None] * wt[None, :, None] * wt[None, None, :]
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1), W.ravel()


def _feq(xi):
    return (2.0 * math.pi) ** -1.5 * np.exp(-0.5 * np.sum(xi * xi, axis=1))


def transport_symbol(s, h=None):
    """Fourier symbol of tau xi_x d/dx for s = tau theta xi_x: i s in continuous space,
    |s| (1 - exp(-i sgn(s) h)) / h for first-order upwinding on cells of width h / theta."""
    s = np.asarray(s, np.float64)
    if h is None:
        return 1j * s
    return np.abs(s) * (1.0 - np.exp(-1j * np.sign(s) * h)) / h


def kinetic_response(p, alpha, Kn_theta, xi, h=None):
    """y_0, y_1, y_2 on the grid and the photon amplitude (4 sigma_R / pi) alpha_Tv of one
    CIS kinetic step driven by the macroscopic error alpha (Eq. error_function_propagation);
    ``h``: the upwind symbol of a periodic row of cells (see transport_symbol)."""
    a = math.sqrt(2.0 / math.pi) * Kn_theta
    f0 = _feq(xi)
    x2 = np.sum(xi * xi, axis=1)
    A = p.A
    cr, cv = p.d_r / ((3 + p.d_r) * p.Z_r), p.d_v / ((3 + p.d_v) * p.Z_v)
    u = alpha[1:4]
    qt, qr, qv = alpha[QT:QT + 3], alpha[QR:QR + 3], alpha[QV:QV + 3]
    base = (alpha[RHO] + xi @ u + alpha[TT] * (1 - cr - cv) * (0.5 * x2 - 1.5)
            + (cr * alpha[TR] + cv * alpha[TV]) * (0.5 * x2 - 1.5)
            + (xi @ ((3 - 3 * A[0, 0]) * qt - 3 * A[0, 1] * qr - 3 * A[0, 2] * qv)) * (2.0 / 15.0) * (0.5 * x2 - 2.5))
    r1 = (base + 3 / ((3 + p.d_r) * p.Z_r) * alpha[TT] + (1 - 3 / ((3 + p.d_r) * p.Z_r)) * alpha[TR]
          + (xi @ (-A[1, 0] * qt + (1 - A[1, 1]) * qr - A[1, 2] * qv)) * (2.0 / p.d_r))
    r2 = (base + 3 / ((3 + p.d_v) * p.Z_v) * alpha[TT] + (1 - 3 / ((3 + p.d_v) * p.Z_v)) * alpha[TV]
          + (xi @ (-A[2, 0] * qt - A[2, 1] * qr + (1 - A[2, 2]) * qv)) * (2.0 / p.d_v))
    den = 1.0 + transport_symbol(a * xi[:, 0], h)
    y0 = f0 * base / den
    y1 = 0.5 * p.d_r * f0 * r1 / den
    y2 = (0.5 * p.d_v * f0 * r2 - math.sqrt(2.0 / math.pi) * p.ratio * f0
          * (16 * p.sigma_R * alpha[TV] - alpha[ER])) / den
    return y0, y1, y2, 4.0 * p.sigma_R / math.pi * alpha[TV]


def photon_integrals(b):
    """(int dOmega / (1 + i b mu), int mu dOmega / (1 + i b mu)) over the unit sphere."""
    if abs(b) < 1e-8:
        return 4.0 * math.pi, 0.0
    i0 = 4.0 * math.pi * math.atan(b) / b
    i1 = 2.0 * math.pi / (1j * b) * (2.0 - 2.0 * math.atan(b) / b)
    return i0, i1


def cis_matrix(p, Kn_theta, grid=None, h=None, photons=None):
    """C (17 x 17) of Eq. eigenfunction_cis.  ``h`` = theta dx selects the upwind symbol
    of a periodic row of cells; ``photons`` = (mu, w), the x-cosines and weights of a
    discrete direction set, replaces the exact sphere integral."""
    xi, w = grid if grid is not None else velocity_grid()
    x2 = np.sum(xi * xi, axis=1)
    b = Kn_theta / p.ratio                      # Kn_p theta with Kn = 1
    if photons is None and h is None:
        i0, _ = photon_integrals(b)
    else:
        mu, wmu = photons if photons is not None else np.polynomial.legendre.leggauss(400)
        if photons is None:
            wmu = 2.0 * math.pi * wmu
        i0 = np.sum(wmu / (1.0 + transport_symbol(b * np.asarray(mu), h)))
    C = np.zeros((NM, NM), complex)
    for n in range(NM):
        e = np.zeros(NM)
        e[n] = 1.0
        y0, y1, y2, yR = kinetic_response(p, e, Kn_theta, xi, h)
        col = np.zeros(NM, complex)
        col[RHO] = w @ y0
        col[1:4] = (w * y0) @ xi
        col[TT] = w @ ((x2 / 3 - 1) * y0)
        col[TR] = w @ (2 / p.d_r * y1 - y0)
        col[TV] = w @ (2 / p.d_v * y2 - y0)
        col[ER] = yR * i0
        col[QT:QT + 3] = (w * (0.5 * x2 - 2.5) * y0) @ xi
        col[QR:QR + 3] = (w * (y1 - 0.5 * p.d_r * y0)) @ xi
        col[QV:QV + 3] = (w * (y2 - 0.5 * p.d_v * y0)) @ xi
        C[:, n] = col
    return C


def gsis_matrices(p, Kn_theta, grid=None, h=None, photons=None):
    """L and R (17 x 17) of Eq. eigenfunction_gsis_matrix, with Kn = 1 and theta = Kn theta
    along x.  ``h`` and ``photons`` act on the kinetic half step only, as in cis_matrix (the
    synthetic equations stay continuous)."""
    xi, w = grid if grid is not None else velocity_grid()
    x2 = np.sum(xi * xi, axis=1)
    th = Kn_theta
    kn, knp = 1.0, 1.0 / p.ratio
    b = knp * th
    if photons is None and h is None:
        i0, i1 = photon_integrals(b)
    else:
        mu, wmu = photons if photons is not None else np.polynomial.legendre.leggauss(400)
        mu = np.asarray(mu, np.float64)
        if photons is None:
            wmu = 2.0 * math.pi * wmu
        den = 1.0 + transport_symbol(b * mu, h)
        i0, i1 = np.sum(wmu / den), np.sum(wmu * mu / den)
    kap = math.sqrt(2.0 / math.pi) * kn / 2.0 * np.linalg.inv(p.A) @ np.diag([5.0, p.d_r, p.d_v])
    kR = knp / 3.0
    mu = math.sqrt(2.0 / math.pi) * kn
    cr = math.sqrt(math.pi / 2.0) / kn * 3 * p.d_r / (2 * (3 + p.d_r) * p.Z_r)
    cv = math.sqrt(math.pi / 2.0) / kn * 3 * p.d_v / (2 * (3 + p.d_v) * p.Z_v)
    T_rows = (TT, TR, TV)
    L = np.zeros((NM, NM), complex)
    # 1 continuity, 2-4 momentum, 5 energy, 6 rotational, 7 vibrational, 8 radiation,
    # 9-17 constitutive relations of q_t, q_r, q_v
    L[0, UX] = 1j * th
    for a in range(3):
        L[1 + a, 1 + a] = mu * th * th
    L[1, RHO] += 1j * th
    L[1, TT] += 1j * th
    L[4, QT] = L[4, QR] = L[4, QV] = 1j * th
    L[4, ER] = th * th * kR
    L[5, QR] = 1j * th
    L[5, TR] += cr
    L[5, TT] -= cr
    L[6, QV] = 1j * th
    L[6, TV] += cv + 16 * p.sigma_R / knp
    L[6, TT] -= cv
    L[6, ER] -= 1.0 / knp
    L[7, ER] = th * th * kR + 1.0 / knp
    L[7, TV] = -16 * p.sigma_R / knp
    for m, qb in enumerate((QT, QR, QV)):
        for a in range(3):
            L[8 + 3 * m + a, qb + a] = 1.0
        for l, tr in enumerate(T_rows):
            L[8 + 3 * m, tr] += 1j * th * kap[m, l]          # x component only
    Rm = np.zeros((NM, NM), complex)
    for n in range(NM):
        e = np.zeros(NM)
        e[n] = 1.0
        y0, y1, y2, yR = kinetic_response(p, e, th, xi, h)
        col = np.zeros(NM, complex)
        # momentum: int [-i theta x (xi xi - xi^2/3 I) + mu (theta^2 xi + theta (theta . xi)/3)] y0
        for a in range(3):
            sxx = xi[:, 0] * xi[:, a] - (x2 / 3 if a == 0 else 0.0)
            col[1 + a] = w @ ((-1j * th * sxx + mu * (th * th * xi[:, a] + (th * th * xi[:, 0] / 3 if a == 0 else 0.0)))
                              * y0)
        col[4] = yR * (-1j * th * i1 + kR * th * th * i0)
        col[7] = col[4]
        Tmom = [(x2 / 3 - 1) * y0, 2 / p.d_r * y1 - y0, 2 / p.d_v * y2 - y0]
        qmom = [(0.5 * x2 - 2.5) * y0, y1 - 0.5 * p.d_r * y0, y2 - 0.5 * p.d_v * y0]
        for m in range(3):
            for a in range(3):
                col[8 + 3 * m + a] = w @ (xi[:, a] * qmom[m])
            col[8 + 3 * m] += sum(1j * th * kap[m, l] * (w @ Tmom[l]) for l in range(3))
        Rm[:, n] = col
    return L, Rm


def spectral_radius_cis(p, Kn_theta, grid=None, h=None, photons=None):
    return float(np.max(np.abs(np.linalg.eigvals(cis_matrix(p, Kn_theta, grid, h, photons)))))


def gsis_algorithm_matrix(p, Kn_theta, grid=None, h=None, photons=None):
    """The GSIS step as the algorithm of Section 3 takes it (step 3, the synchronisation):
    the synthetic equations (L alpha' = R alpha) give the next density, velocity,
    temperatures and e_R, and the equilibria that the synchronisation adds carry no heat
    flux, so the next heat fluxes are those of the kinetic half step, the q rows of the CIS
    matrix.  (The eigen-equation of Section 4 takes them from the constitutive rows of L.)"""
    L, R = gsis_matrices(p, Kn_theta, grid, h, photons)
    G = np.linalg.solve(L, R)
    G[QT:QV + 3] = cis_matrix(p, Kn_theta, grid, h, photons)[QT:QV + 3]
    return G


def spectral_radius_gsis(p, Kn_theta, grid=None, h=None, photons=None, algorithm=False):
    if algorithm:
        return float(np.max(np.abs(np.linalg.eigvals(gsis_algorithm_matrix(p, Kn_theta, grid, h, photons)))))
    L, R = gsis_matrices(p, Kn_theta, grid, h, photons)
    return float(np.max(np.abs(np.linalg.eigvals(np.linalg.solve(L, R)))))


def xi_x_integral_faddeeva(k, a):
    """int g(x) x^k / (1 + i a x) dx for the standard normal density g, from the Faddeeva
    function: the k = 0 integral is sqrt(pi/2)/a w(i/(a sqrt 2)); higher k follow from
    x^(k+1)/(1 + i a x) = (x^k - x^k/(1 + i a x)) / (i a)."""
    from scipy.special import wofz
    J = math.sqrt(math.pi / 2.0) / a * wofz(1j / (a * math.sqrt(2.0)))
    moments = [1.0, 0.0, 1.0, 0.0, 3.0, 0.0, 15.0, 0.0, 105.0]
    for j in range(k):
        J = (moments[j] - J) / (1j * a)
    return J
