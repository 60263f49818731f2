"""Named synthetic workloads: mesh + velocity/photon grids + model/solver parameters.

Gas parameters follow the paper's test section (d_r = 2, d_v = 1.16, Z_r = 2.67,
Z_v = 26.7, omega = 0.74); the geometries are seeded synthetic stand-ins for the
paper's cases.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

from . import mesh as _mesh
from . import quadrature as _q


@dataclass
class ModelParams:
    d_r: float = 2.0
    d_v: float = 1.16
    Z_r: float = 2.67
    Z_v: float = 26.7
    omega: float = 0.74
    Sc: float = 5.0 / 6.0
    Kn: float = 0.1
    Kn_p: float = 1.0
    sigma_R: float = 0.01
    k_eff_density_scaled: bool = False
    dv_temperature_dependent: bool = False   # d_v(T_v) = 2 x / (e^x - 1), x = Tv_ref / T_v (else d_v constant)
    Tv_ref: float = 0.0                      # characteristic vibrational temperature (units of T_0)
    A: np.ndarray | None = None          # 3x3 relaxation-rate matrix, None = Mason-Monchick form


@dataclass
class SolverParams:
    precision: str = "fp32"              # "fp32" or "fp64" storage/arithmetic of f and I
    order: int = 2                       # 1 = first-order upwind, 2 = limited linear reconstruction
    relax_block: int = 16                # Gauss-Seidel block of consecutive cells (1 = Jacobi)
    cfl_meso: float = 1e5
    cfl_macro: float = 1e3
    venkat_K: float = 5.0
    n_cis_precond: int = 10
    max_outer: int = 200
    max_inner: int = 100
    macro_sweeps: int = 6
    tol_outer: float = 1e-6
    tol_inner: float = 1e-7
    sync_relax: float = 1.0              # weight of the equilibrium correction in the synchronisation
    macro_fp32: int = 0                  # library FP32 path: synthetic residual side in FP32
    tc_moments: int = 1                  # library FP32 path: 0 CUDA cores, 1 tensor cores in the moment/sync
                                         # passes, 2 also in the sweep epilogue
    positivity: float = 0.0              # 0 <= theta < 1: the implicit update keeps f >= theta f_old (0: off)
    defect_correction: int = 0           # 1: synthetic residual R(W) - R(W_h) + kinetic residual moments (0: off)


@dataclass
class Workload:
    name: str
    mesh: _mesh.Mesh
    xi: np.ndarray
    w: np.ndarray
    omega: np.ndarray
    wo: np.ndarray
    model: ModelParams
    solver: SolverParams = field(default_factory=SolverParams)

    @property
    def dim(self) -> int:
        return self.mesh.dim


def slab(n_cells: int = 64, n_xi: int = 32, n_mu: int = 16, Kn: float = 0.1,
         Kn_p: float = 1.0, sigma_R: float = 0.01, T_left: float = 1.0, T_right: float = 1.5) -> Workload:
    """1-D Fourier slab between diffuse/black walls at T_left and T_right."""
    m = _mesh.slab_1d(n_cells, 1.0, patches=[_mesh.Patch(_mesh.WALL, T_t=T_left),
                                             _mesh.Patch(_mesh.WALL, T_t=T_right)])
    xi, w = _q.gauss_hermite_1d(n_xi)
    om, wo = _q.gauss_legendre_slab(n_mu)
    return Workload("slab%d" % n_cells, m, xi, w, om, wo,
                    ModelParams(Kn=Kn, Kn_p=Kn_p, sigma_R=sigma_R),
                    SolverParams(precision="fp64", tol_outer=1e-8))


def cavity(n_side: int = 100, n_v: int = 28, n_polar: int = 8, n_azim: int = 8, Kn: float = 0.1,
           Kn_p: float = 10.0, sigma_R: float = 0.005, u_lid: float = 0.18, T_lid: float = 3.0,
           seed: int = 0, rule: str = "trapezoid") -> Workload:
    """2-D lid-driven, heated cavity on a seeded triangle mesh (2*n_side^2 cells).

    The n_v x n_v uniform velocity grid spans +-(|u_lid| + 5 sqrt(T_lid)) with the
    composite closed Newton-Cotes rule of degree one (trapezoid) by default; "nc38"
    selects the composite 3/8 rule, and "disc" an unstructured mesh of n_v rings on the
    disc of that radius (no tensor product)."""
    m = _mesh.cavity_triangles(n_side, seed=seed, patches=[
        _mesh.Patch(_mesh.WALL, T_t=1.0), _mesh.Patch(_mesh.WALL, T_t=1.0),
        _mesh.Patch(_mesh.WALL, u=(u_lid, 0.0, 0.0), T_t=T_lid), _mesh.Patch(_mesh.WALL, T_t=1.0)])
    L = abs(u_lid) + 5.0 * np.sqrt(max(T_lid, 1.0))
    if rule == "trapezoid":
        xi, w = _q.trapezoid_nd(n_v, L, 2)
    elif rule == "nc38":
        xi, w = _q.newton_cotes_2d(n_v, L)
    elif rule == "disc":
        xi, w = _q.disc_velocity_mesh(n_v, L, stretch=1.3, seed=seed)
    else:
        raise ValueError("unknown velocity rule %r" % rule)
    om, wo = _q.photon_product(n_polar, n_azim)
    return Workload("cavity%d" % (2 * n_side * n_side), m, xi, w, om, wo,
                    ModelParams(Kn=Kn, Kn_p=Kn_p, sigma_R=sigma_R))


def couette(n_side: int = 8, n_v: int = 16, n_polar: int = 4, n_azim: int = 8, Kn: float = 0.1,
            Kn_p: float = 1.0, sigma_R: float = 0.005, u_wall: float = 0.2, seed: int = 0) -> Workload:
    """2-D planar Couette flow: the unit square periodic in x (``channel_triangles``)
    between a wall at rest (bottom, T = 1) and a wall moving at u_wall along x (top, T = 1);
    n_v x n_v trapezoid velocities on +-(|u_wall| + 5)."""
    m = _mesh.channel_triangles(n_side, seed=seed, patches=[
        _mesh.Patch(_mesh.WALL, T_t=1.0), _mesh.Patch(_mesh.WALL, u=(u_wall, 0.0, 0.0), T_t=1.0)])
    xi, w = _q.trapezoid_nd(n_v, abs(u_wall) + 5.0, 2)
    om, wo = _q.photon_product(n_polar, n_azim)
    return Workload("couette%d" % m.n_cells, m, xi, w, om, wo, ModelParams(Kn=Kn, Kn_p=Kn_p, sigma_R=sigma_R))


def cylinder(n_theta: int = 200, n_radial: int = 100, n_v: int = 48, n_polar: int = 8,
             n_azim: int = 12, Mach: float = 5.0, T_inf: float = 0.5, Kn: float = 0.01,
             Kn_p: float = 1000.0, sigma_R: float = 0.1, seed: int = 1) -> Workload:
    """2-D hypersonic flow past a cylinder (diameter 1) on a seeded triangulated O-grid."""
    gamma = (5.0 + 2.0 + 1.16) / (3.0 + 2.0 + 1.16)
    u_inf = Mach * np.sqrt(gamma * T_inf)
    T0 = T_inf * (1.0 + 0.5 * (gamma - 1.0) * Mach * Mach)
    m = _mesh.cylinder_ogrid(n_theta, n_radial, seed=seed, patches=[
        _mesh.Patch(_mesh.WALL, T_t=T_inf),
        _mesh.Patch(_mesh.FARFIELD, rho=1.0, u=(u_inf, 0.0, 0.0), T_t=T_inf, T_r=T_inf,
                    T_v=T_inf, T_R=T_inf)])
    L = 8.0 * np.sqrt(2.0 * T0)
    xi, w = _q.trapezoid_nd(n_v, L, 2)
    om, wo = _q.photon_product(n_polar, n_azim)
    return Workload("cylinder%d" % (2 * n_theta * n_radial), m, xi, w, om, wo,
                    ModelParams(Kn=Kn, Kn_p=Kn_p, sigma_R=sigma_R, k_eff_density_scaled=True))


def capsule(n: int = 32, n_v: int = 24, n_polar: int = 8, n_azim: int = 16, Mach: float = 10.0,
            T_inf: float = 0.5, T_wall: float = 0.5, Kn: float = 0.01, Kn_p: float = 1000.0,
            sigma_R: float = 0.1, seed: int = 2) -> Workload:
    """3-D hypersonic flow past a sphere-cone re-entry capsule (60-degree forebody, shoulder
    radius 0.1 D; mesh.capsule_tetrahedra) on a seeded tetrahedral mesh of the unit cube
    (about 6 n^3 cells, 193 009 at n = 32); the free stream flows along +x.  The n_v^3 uniform velocity grid (trapezoid weights) spans
    +-(u_inf + 4 sqrt(T_0)), T_0 the stagnation temperature; n_polar x n_azim photon
    directions.  FP32, order 2, CUDA-core moments."""
    gamma = (5.0 + 2.0 + 1.16) / (3.0 + 2.0 + 1.16)
    u_inf = Mach * np.sqrt(gamma * T_inf)
    T0 = T_inf * (1.0 + 0.5 * (gamma - 1.0) * Mach * Mach)
    m = _mesh.capsule_tetrahedra(n, seed=seed, patches=[
        _mesh.Patch(_mesh.WALL, T_t=T_wall),
        _mesh.Patch(_mesh.FARFIELD, rho=1.0, u=(u_inf, 0.0, 0.0), T_t=T_inf, T_r=T_inf,
                    T_v=T_inf, T_R=T_inf)])
    L = u_inf + 4.0 * np.sqrt(T0)
    xi, w = _q.trapezoid_nd(n_v, L, 3)
    om, wo = _q.photon_product(n_polar, n_azim)
    return Workload("capsule%d" % m.n_cells, m, xi, w, om, wo,
                    ModelParams(Kn=Kn, Kn_p=Kn_p, sigma_R=sigma_R, k_eff_density_scaled=True),
                    SolverParams(tc_moments=0))


def rankine_hugoniot(Mach: float, gamma: float):
    """Downstream (rho, u, T) of a normal shock with upstream rho = T = 1 and
    u = sqrt(gamma) Mach (velocity unit sqrt(R T0)), from the Rankine-Hugoniot relations
    as the paper's normal-shock case states them (Section 'Normal shock wave')."""
    M2 = Mach * Mach
    rho_d = (gamma + 1.0) * M2 / (2.0 + (gamma - 1.0) * M2)
    u_u = np.sqrt(gamma) * Mach
    T_d = (2.0 + (gamma - 1.0) * M2) * (2.0 * gamma * M2 - (gamma - 1.0)) / ((gamma + 1.0) ** 2 * M2)
    return rho_d, u_u / rho_d, T_d


def normal_shock(Z_r: float = 2.6, Z_v: float = 26.0, length: float = 200.0, dx: float = 0.25,
                 Mach: float = 5.0, n_xi: int = 64, xi_max: float = 15.0, n_theta: int = 48,
                 x_shock: float = 0.25) -> Workload:
    """The paper's Mach-5 normal shock (Section 'Normal shock wave'): a uniform 1-D mesh of
    spacing dx over `length` (in the unit L0 of the paper, so Kn = 5 pi / 16), fixed
    upstream and Rankine-Hugoniot downstream equilibrium states at the two ends (far-field
    patches), Kn_p = 10, sigma_R = 0.01, n_xi uniform velocities on [-xi_max, xi_max]
    (trapezoid weights) and n_theta uniform polar cells for the photons.  The initial
    discontinuity sits at the fraction `x_shock` of the domain."""
    d_r, d_v = 2.0, 1.16
    gamma = (5.0 + d_r + d_v) / (3.0 + d_r + d_v)
    rho_d, u_d, T_d = rankine_hugoniot(Mach, gamma)
    u_u = np.sqrt(gamma) * Mach
    n = int(round(length / dx))
    m = _mesh.slab_1d(n, length, patches=[
        _mesh.Patch(_mesh.FARFIELD, rho=1.0, u=(u_u, 0.0, 0.0), T_t=1.0, T_r=1.0, T_v=1.0, T_R=1.0),
        _mesh.Patch(_mesh.FARFIELD, rho=rho_d, u=(u_d, 0.0, 0.0), T_t=T_d, T_r=T_d, T_v=T_d, T_R=T_d)])
    m.cell_centroid = m.cell_centroid - x_shock * length
    m.face_centroid = m.face_centroid - x_shock * length
    xi, w = _q.trapezoid_nd(n_xi, xi_max, 1)
    om, wo = _q.uniform_polar_slab(n_theta)
    return Workload("shock_Zv%g_%d" % (Z_v, n), m, xi, w, om, wo,
                    ModelParams(d_r=d_r, d_v=d_v, Z_r=Z_r, Z_v=Z_v, Kn=5.0 * np.pi / 16.0, Kn_p=10.0,
                                sigma_R=0.01),
                    SolverParams(precision="fp64", tol_outer=2e-6, max_outer=4000))


def with_solver(wl: Workload, **kw) -> Workload:
    return replace(wl, solver=replace(wl.solver, **kw))


def with_model(wl: Workload, **kw) -> Workload:
    return replace(wl, model=replace(wl.model, **kw))
