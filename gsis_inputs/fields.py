"""Seeded per-cell macroscopic states and distribution functions (inputs only).

The per-cell field record (the library's I/O layout, NF = 26 doubles per cell):
  0 rho | 1..3 u | 4 T_t | 5 T_r | 6 T_v | 7 T_R | 8..10 q_t | 11..13 q_r |
  14..16 q_v | 17..19 q_R | 20..25 sigma (xx, yy, zz, xy, xz, yz)
"""
from __future__ import annotations

import numpy as np

NF = 26
RHO, UX, UY, UZ, TT, TR, TV, TRAD = 0, 1, 2, 3, 4, 5, 6, 7
QT, QR, QV, QRAD, SIG = 8, 11, 14, 17, 20


def random_macro_fields(n_cells: int, dim: int, seed: int, u_scale: float = 1.0,
                        q_scale: float = 0.1) -> np.ndarray:
    """rho ~ U(0.5, 2), in-plane u ~ U(-1, 1)*u_scale, temperatures ~ U(0.5, 3),
    in-plane heat fluxes ~ U(-1, 1)*q_scale*rho*T^1.5; everything else zero."""
    rng = np.random.default_rng(seed)
    M = np.zeros((n_cells, NF))
    M[:, RHO] = rng.uniform(0.5, 2.0, n_cells)
    M[:, UX:UX + dim] = rng.uniform(-1.0, 1.0, (n_cells, dim)) * u_scale
    M[:, TT:TRAD + 1] = rng.uniform(0.5, 3.0, (n_cells, 4))
    for base, T in ((QT, TT), (QR, TR), (QV, TV), (QRAD, TRAD)):
        amp = q_scale * M[:, RHO] * M[:, T] ** 1.5
        M[:, base:base + dim] = rng.uniform(-1.0, 1.0, (n_cells, dim)) * amp[:, None]
    return M


def smooth_random_fields(x, seed: int, u_scale: float = 0.3, q_scale: float = 0.05) -> np.ndarray:
    """Per-cell states from a few seeded low-wavenumber Fourier modes of the cell
    centroids x [n, dim]: rho in [0.6, 1.4], temperatures in [0.8, 2.2], |u| <= u_scale,
    heat fluxes up to q_scale rho T^1.5."""
    rng = np.random.default_rng(seed)
    n, dim = x.shape

    def field():
        acc = np.zeros(n)
        for _ in range(3):
            k = rng.uniform(-2.0 * np.pi, 2.0 * np.pi, dim)
            acc += np.sin(x @ k + rng.uniform(0.0, 2.0 * np.pi)) / 3.0
        return acc                                    # in [-1, 1]

    M = np.zeros((n, NF))
    M[:, RHO] = 1.0 + 0.4 * field()
    for a in range(dim):
        M[:, UX + a] = u_scale * field()
    for k in (TT, TR, TV, TRAD):
        M[:, k] = 1.5 + 0.7 * field()
    for base, T in ((QT, TT), (QR, TR), (QV, TV), (QRAD, TRAD)):
        for a in range(dim):
            M[:, base + a] = q_scale * M[:, RHO] * M[:, T] ** 1.5 * field()
    return M


def uniform_fields(n_cells: int, rho=1.0, u=(0.0, 0.0, 0.0), T=1.0, T_R=None) -> np.ndarray:
    M = np.zeros((n_cells, NF))
    M[:, RHO] = rho
    M[:, UX:UZ + 1] = np.asarray(u, np.float64)
    M[:, TT:TV + 1] = T
    M[:, TRAD] = T if T_R is None else T_R
    return M


def shock_fields(wl) -> np.ndarray:
    """Step initial state of the normal shock: the upstream patch state for x <= 0, the
    downstream patch state for x > 0 (all temperatures equal on each side)."""
    up, down = wl.mesh.patches[0], wl.mesh.patches[1]
    x = wl.mesh.cell_centroid[:, 0]
    M = np.zeros((wl.mesh.n_cells, NF))
    for sel, P in ((x <= 0.0, up), (x > 0.0, down)):
        M[sel, RHO] = P.rho
        M[sel, UX:UZ + 1] = np.asarray(P.u, np.float64)
        M[sel, TT], M[sel, TR], M[sel, TV], M[sel, TRAD] = P.T_t, P.T_r, P.T_v, P.T_R
    return M


def noisy_equilibrium(M, xi, omega, dim, d_r, d_v, sigma_R, seed, noise=0.05):
    """Multi-temperature local equilibrium of each cell's (rho, u, T_t, T_r, T_v, T_R),
    each value multiplied by (1 + noise*U(-1, 1)).

    Returns f of shape [n_cells, V, 4] (planes: f0, f0-perp, f1, f2) and I of shape
    [n_cells, n_omega].  In 3-D the f0-perp plane is zero.
    """
    rng = np.random.default_rng(seed)
    n, V = M.shape[0], xi.shape[0]
    m_hidden = 3 - dim
    rho, T_t = M[:, RHO][:, None], M[:, TT][:, None]
    c2 = np.zeros((n, V))
    for a in range(dim):
        c2 += (xi[None, :, a] - M[:, UX + a][:, None]) ** 2
    F = rho * (2.0 * np.pi * T_t) ** (-0.5 * dim) * np.exp(-c2 / (2.0 * T_t))
    f = np.empty((n, V, 4))
    f[:, :, 0] = F
    f[:, :, 1] = m_hidden * T_t * F
    f[:, :, 2] = 0.5 * d_r * M[:, TR][:, None] * F
    f[:, :, 3] = 0.5 * d_v * M[:, TV][:, None] * F
    f *= 1.0 + noise * rng.uniform(-1.0, 1.0, f.shape)
    I = np.repeat((sigma_R * M[:, TRAD] ** 4 / np.pi)[:, None], omega.shape[0], axis=1)
    I *= 1.0 + noise * rng.uniform(-1.0, 1.0, I.shape)
    return f, I
