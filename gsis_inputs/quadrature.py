"""Seeded/deterministic quadrature generators (inputs only, no method arithmetic).

Velocity grids are returned as ``(xi, w)`` with ``xi`` of shape ``[n, vdim]`` and
``w`` of shape ``[n]`` such that ``sum_i w_i phi(xi_i)`` approximates the integral
of ``phi`` over the (reduced) velocity space.  Photon grids are ``(omega, w)``
with unit directions ``omega`` of shape ``[n, 3]`` and ``sum w = 4*pi``.

These rules are the inputs that the solver and the oracle both consume: the
velocity grids of the paper's cases are uniform Cartesian grids in a reduced
velocity space (Section 6) and the photon grids cover the unit sphere.
"""
from __future__ import annotations

import numpy as np


def gauss_hermite_1d(n: int):
    """n-point Gauss-Hermite rule for the weight exp(-xi^2/2) on the real line.

    The stored weights absorb exp(+xi^2/2), so ``sum w_i f(xi_i)`` approximates
    ``int f dxi`` for Maxwellian-like ``f``.
    """
    x, wx = np.polynomial.hermite.hermgauss(n)      # weight exp(-x^2)
    xi = np.sqrt(2.0) * x
    w = np.sqrt(2.0) * wx * np.exp(x * x)
    return xi.reshape(n, 1), w


def newton_cotes_38_weights(n: int, half_width: float):
    """Composite Simpson-3/8 rule with n points on [-L, L]; n-1 must be a multiple of 3."""
    if (n - 1) % 3 != 0:
        raise ValueError("composite 3/8 rule needs n = 3k + 1 points")
    x = np.linspace(-half_width, half_width, n)
    h = x[1] - x[0]
    w = np.zeros(n)
    for p in range((n - 1) // 3):
        w[3 * p: 3 * p + 4] += np.array([1.0, 3.0, 3.0, 1.0]) * (3.0 * h / 8.0)
    return x, w


def trapezoid_weights(n: int, half_width: float):
    """Uniform trapezoid rule with n points on [-L, L]."""
    x = np.linspace(-half_width, half_width, n)
    h = x[1] - x[0]
    w = np.full(n, h)
    w[0] = w[-1] = 0.5 * h
    return x, w


def tensor_grid(nodes_w_list):
    """Tensor product of 1-D rules; the first axis varies slowest."""
    xs = [nw[0] for nw in nodes_w_list]
    ws = [nw[1] for nw in nodes_w_list]
    mesh = np.meshgrid(*xs, indexing="ij")
    wmesh = np.meshgrid(*ws, indexing="ij")
    xi = np.stack([m.ravel() for m in mesh], axis=1)
    w = np.ones(xi.shape[0])
    for wm in wmesh:
        w = w * wm.ravel()
    return xi, w


def newton_cotes_2d(n: int, half_width: float):
    """n x n composite Newton-Cotes (3/8) product grid on [-L, L]^2."""
    r = newton_cotes_38_weights(n, half_width)
    return tensor_grid([r, r])


def trapezoid_nd(n: int, half_width: float, dim: int):
    r = trapezoid_weights(n, half_width)
    return tensor_grid([r] * dim)


def gauss_legendre_slab(n: int):
    """Photon directions for a plane-parallel slab: Gauss-Legendre in mu = Omega_x.

    Each node stands for the ring of directions with the same mu, so its weight
    is 2*pi times the Gauss-Legendre weight; the direction stored for the ring is
    (mu, sqrt(1-mu^2), 0).
    """
    mu, wmu = np.polynomial.legendre.leggauss(n)
    om = np.stack([mu, np.sqrt(1.0 - mu * mu), np.zeros(n)], axis=1)
    return om, 2.0 * np.pi * wmu


def uniform_polar_slab(n: int):
    """Photon directions for a plane-parallel slab from n uniform cells of the polar angle
    theta in [0, pi] (the azimuth integrates out): each cell is one ring of directions at
    its mid angle, weighted by the exact solid angle 2 pi (cos theta_lo - cos theta_hi)."""
    edges = np.linspace(0.0, np.pi, n + 1)
    th = 0.5 * (edges[1:] + edges[:-1])
    w = 2.0 * np.pi * (np.cos(edges[:-1]) - np.cos(edges[1:]))
    om = np.stack([np.cos(th), np.sin(th), np.zeros(n)], axis=1)
    return om, w


def photon_product(n_polar: int, n_azim: int):
    """Gauss-Legendre in cos(polar angle about z) x uniform azimuth in the x-y plane."""
    mu, wmu = np.polynomial.legendre.leggauss(n_polar)
    phi = (np.arange(n_azim) + 0.5) * (2.0 * np.pi / n_azim)
    M, P = np.meshgrid(mu, phi, indexing="ij")
    W = np.meshgrid(wmu, np.full(n_azim, 2.0 * np.pi / n_azim), indexing="ij")
    s = np.sqrt(1.0 - M * M)
    om = np.stack([(s * np.cos(P)).ravel(), (s * np.sin(P)).ravel(), M.ravel()], axis=1)
    return om, (W[0] * W[1]).ravel()


def disc_velocity_mesh(n_rings: int, r_max: float, stretch: float = 1.5, seed: int = 0):
    """Unstructured 2-D velocity mesh on the disc |xi| <= r_max (no tensor product).

    The disc is cut into n_rings annuli with edges r_k = r_max (k / n_rings)^stretch, so
    that the rings cluster near low speeds. Annulus k is cut into n_k ~ 2 pi r_mid / dr
    near-square sectors, and each ring is rotated by a seeded offset. A point sits at its
    sector's area centroid and carries the sector's area. The rule is therefore exact for
    polynomials of degree one on every sector, and its weights sum to pi r_max^2.
    """
    rng = np.random.default_rng(seed)
    edges = r_max * (np.arange(n_rings + 1) / n_rings) ** stretch
    pts, ws = [], []
    for k in range(n_rings):
        a, b = edges[k], edges[k + 1]
        n = max(6, int(round(np.pi * (a + b) / (b - a))))
        dth = 2.0 * np.pi / n
        # area-centroid radius of an annular sector of opening angle dth
        rc = (2.0 / 3.0) * (b ** 3 - a ** 3) / (b ** 2 - a ** 2) * np.sin(0.5 * dth) / (0.5 * dth)
        th = (np.arange(n) + 0.5 + rng.uniform(-0.5, 0.5)) * dth
        pts.append(np.stack([rc * np.cos(th), rc * np.sin(th)], axis=1))
        ws.append(np.full(n, 0.5 * (b * b - a * a) * dth))
    return np.concatenate(pts), np.concatenate(ws)
