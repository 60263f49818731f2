"""GPU parity of one GSIS iteration (Section 3: kinetic step, high-order terms, synthetic
equations, synchronisation) against the FP64 oracle on the same seeded inputs.

The synthetic solve runs a fixed number of inner iterations (tol_inner = 0), so both
sides take exactly the same steps.  Tolerances: FP64 1e-10 relative (distributions per
plane, fields as in the conventional-iteration tests); FP32 distributions 1e-5.
"""
import numpy as np
import pytest

import gsis_inputs as gi
from oracle import gsis as OG
from oracle import kinetic as K
from oracle import macro as MA
from paper_2601_03935_gb300 import build
from paper_2601_03935_gb300 import gsis as G

from _ctx import assert_fields_close, assert_planes_close, create

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    G.load()


def _inputs(wl, seed, precision):
    M = gi.fields.smooth_random_fields(wl.mesh.cell_centroid, seed, u_scale=0.2)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, wl.dim, wl.model.d_r, wl.model.d_v,
                                       wl.model.sigma_R, seed + 1, noise=0.02)
    if precision == "fp32":
        f, I = f.astype(np.float32).astype(np.float64), I.astype(np.float32).astype(np.float64)
    return f, I


CASES = {
    # 16 cells between walls: the closed-domain mass rescaling, 1-D reduced planes
    "slab16": lambda: gi.workloads.slab(16, Kn=0.05),
    # 72 triangles, heated moving lid: 2-D walls, a ragged relaxation block
    "cavity72": lambda: gi.workloads.cavity(n_side=6, Kn=0.05, Kn_p=1.0),
    # the same cavity on an unstructured disc velocity mesh (245 velocities, no tensor product)
    "cavity72_disc": lambda: gi.workloads.cavity(n_side=6, n_v=10, Kn=0.05, Kn_p=1.0, rule="disc"),
    # 64 triangles around a cylinder: a far-field patch (no mass rescaling)
    "cylinder64": lambda: gi.workloads.cylinder(n_theta=8, n_radial=4, n_v=16, n_polar=4, n_azim=8, Mach=0.5,
                                                Kn=0.05, Kn_p=1.0),
}


def _run(wl, f, I, steps):
    ctx = create(wl)
    try:
        G.gsis_set_distributions(ctx, f, I)
        eps = [G.gsis_step(ctx, G.GSIS_MODE_GSIS) for _ in range(steps)]
        fg, Ig = G.gsis_get_distributions(ctx, wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0])
        rec = G.gsis_get_fields(ctx, wl.mesh.n_cells)
        return fg, Ig, rec, eps
    finally:
        G.gsis_destroy(ctx)


def _oracle(wl, f, I, steps):
    geo = K.Geometry(wl.mesh)
    faces = MA.Faces(geo)
    eps = []
    for _ in range(steps):
        f, I, e, F = OG.gsis_step(f, I, wl, geo, faces)
        eps.append(e)
    return f, I, F, eps


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("case", sorted(CASES))
def test_gsis_step_matches_oracle_fp64(case, order):
    wl = gi.workloads.with_solver(CASES[case](), precision="fp64", order=order, relax_block=16, max_inner=12,
                                  tol_inner=0.0, macro_sweeps=4, cfl_macro=200.0)
    f, I = _inputs(wl, 11, "fp64")
    fg, Ig, rec, eps = _run(wl, f, I, 1)
    fo, Io, Fo, eps_o = _oracle(wl, f, I, 1)
    assert_planes_close(fg, fo, TOL["fp64"], "f^{k+1}")
    assert_planes_close(Ig, Io, TOL["fp64"], "I^{k+1}")
    assert_fields_close(rec, Fo, TOL["fp64"], wl.dim, "moments of f^{k+1}")
    assert abs(eps[0] - eps_o[0]) <= 1e-9 * eps_o[0]


def test_normal_shock_steps_match_oracle():
    """The Mach-5 normal shock (1-D, far-field upstream state and Rankine-Hugoniot
    downstream state at the two ends) from its step initial state: two CIS and one GSIS
    iteration in FP64, order 2, on 24 cells x 48 velocities (one ragged chunk) x 8 polar
    cells."""
    wl = gi.workloads.with_solver(gi.workloads.normal_shock(length=12.0, dx=0.5, n_xi=48, n_theta=8),
                                  precision="fp64", order=2, relax_block=16, max_inner=12, tol_inner=0.0,
                                  venkat_K=0.01)
    M = gi.fields.shock_fields(wl)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 1, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 0,
                                       noise=0.0)
    ctx = create(wl)
    try:
        G.gsis_set_distributions(ctx, f, I)
        eps = [G.gsis_step(ctx, m) for m in (G.GSIS_MODE_CIS, G.GSIS_MODE_CIS, G.GSIS_MODE_GSIS)]
        fg, Ig = G.gsis_get_distributions(ctx, wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0])
        rec = G.gsis_get_fields(ctx, wl.mesh.n_cells)
    finally:
        G.gsis_destroy(ctx)
    geo = K.Geometry(wl.mesh)
    faces = MA.Faces(geo)
    eps_o = []
    fo, Io = f, I
    for _ in range(2):
        fo, Io, e, Fo = OG.cis_step(fo, Io, wl, geo)
        eps_o.append(e)
    fo, Io, e, Fo = OG.gsis_step(fo, Io, wl, geo, faces)
    eps_o.append(e)
    assert_planes_close(fg, fo, TOL["fp64"], "f^{k+3}")
    assert_planes_close(Ig, Io, TOL["fp64"], "I^{k+3}")
    assert_fields_close(rec, Fo, TOL["fp64"], wl.dim, "moments of f^{k+3}")
    assert np.allclose(eps, eps_o, rtol=1e-9)


def test_gsis_two_steps_fp64():
    wl = gi.workloads.with_solver(CASES["cavity72"](), precision="fp64", order=2, relax_block=16, max_inner=10,
                                  tol_inner=0.0)
    f, I = _inputs(wl, 3, "fp64")
    fg, Ig, rec, eps = _run(wl, f, I, 2)
    fo, Io, Fo, eps_o = _oracle(wl, f, I, 2)
    assert_planes_close(fg, fo, TOL["fp64"], "f^{k+2}")
    assert_fields_close(rec, Fo, TOL["fp64"], wl.dim, "moments of f^{k+2}")
    assert np.allclose(eps, eps_o, rtol=1e-9)


def test_gsis_step_matches_oracle_fp32():
    wl = gi.workloads.with_solver(CASES["cavity72"](), precision="fp32", order=2, relax_block=16, max_inner=12,
                                  tol_inner=0.0)
    f, I = _inputs(wl, 5, "fp32")
    fg, Ig, rec, eps = _run(wl, f, I, 1)
    fo, Io, Fo, eps_o = _oracle(wl, f, I, 1)
    assert_planes_close(fg, fo, TOL["fp32"], "f^{k+1}")
    assert_planes_close(Ig, Io, TOL["fp32"], "I^{k+1}")
    assert_fields_close(rec, Fo, TOL["fp32"], wl.dim, "moments of f^{k+1}")


def test_gsis_inner_convergence_stops_early():
    """With a reachable inner tolerance the solve stops on the device flag and still
    matches the oracle, which stops at the same inner iteration."""
    wl = gi.workloads.with_solver(CASES["slab16"](), precision="fp64", order=2, relax_block=16, max_inner=100,
                                  tol_inner=1e-4)
    f, I = _inputs(wl, 13, "fp64")
    fg, Ig, rec, eps = _run(wl, f, I, 1)
    fo, Io, Fo, eps_o = _oracle(wl, f, I, 1)
    assert_planes_close(fg, fo, 1e-9, "f^{k+1}")


@pytest.mark.parametrize("tc", [0, 2])
def test_gsis_step_fp32_moment_engines(tc):
    """The synchronisation pass with its moments on CUDA cores (tc 0) and on the tensor
    cores (tc 2, also the sweep epilogue)."""
    wl = gi.workloads.with_solver(CASES["cavity72"](), precision="fp32", order=2, relax_block=16, max_inner=12,
                                  tol_inner=0.0, tc_moments=tc)
    f, I = _inputs(wl, 9, "fp32")
    fg, Ig, rec, _ = _run(wl, f, I, 1)
    fo, Io, Fo, _ = _oracle(wl, f, I, 1)
    assert_planes_close(fg, fo, TOL["fp32"], "f^{k+1}")
    assert_fields_close(rec, Fo, TOL["fp32"], wl.dim, "moments of f^{k+1}")


@pytest.mark.parametrize("mode", [1, 2])
def test_gsis_step_fp32_residual_side(mode):
    """FP32 contexts may evaluate the synthetic residual side and the relaxation sweeps' flux
    increments in FP32 (the diagonal solves and updates stay FP64):
    throughout (mode 1), or for all but the last 16 inner iterations (mode 2: 8 FP32 and 16
    FP64 iterations here)."""
    wl = gi.workloads.with_solver(CASES["cavity72"](), precision="fp32", order=2, relax_block=16, max_inner=24,
                                  tol_inner=0.0, macro_fp32=mode)
    f, I = _inputs(wl, 5, "fp32")
    fg, Ig, rec, eps = _run(wl, f, I, 1)
    fo, Io, Fo, eps_o = _oracle(wl, f, I, 1)
    assert_planes_close(fg, fo, TOL["fp32"], "f^{k+1}")
    assert_fields_close(rec, Fo, TOL["fp32"], wl.dim, "moments of f^{k+1}")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_hypersonic_cylinder_gsis_step_matches_oracle(precision):
    """Mach 5 past the cylinder from an impulsive start (far field and wall, Kn 0.1,
    Kn_p 1000, sigma_R 0.1): ten CIS iterations on the GPU empty the wake to a density of
    a few 1e-4; one GSIS iteration from that state matches the oracle's.  The
    synchronisation there subtracts Maxwellians whose exponents reach hundreds (FP32
    evaluation must not form 0 x inf)."""
    base = gi.workloads.cylinder(n_theta=24, n_radial=8, n_v=24, n_polar=4, n_azim=8, Mach=5.0, Kn=0.1,
                                 Kn_p=1000.0, sigma_R=0.1)
    wl = gi.workloads.with_solver(base, precision=precision, order=1, relax_block=16, max_inner=100,
                                  tol_inner=1e-7)
    M = gi.fields.uniform_fields(wl.mesh.n_cells)
    far = wl.mesh.patches[1]
    M[:, 0], M[:, 1], M[:, 4:8] = far.rho, far.u[0], far.T_t
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 2, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 0,
                                       noise=0.0)
    ctx = create(wl)
    try:
        G.gsis_set_distributions(ctx, f, I)
        for _ in range(10):
            G.gsis_step(ctx, G.GSIS_MODE_CIS)
        fk, Ik = G.gsis_get_distributions(ctx, wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0])
        G.gsis_step(ctx, G.GSIS_MODE_GSIS)
        fg, Ig = G.gsis_get_distributions(ctx, wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0])
        rec = G.gsis_get_fields(ctx, wl.mesh.n_cells)
    finally:
        G.gsis_destroy(ctx)
    geo = K.Geometry(wl.mesh)
    fo, Io, _, Fo = OG.gsis_step(fk, Ik, wl, geo, MA.Faces(geo))
    assert Fo["rho"].min() < 1e-2      # the near-vacuum wake is part of the case
    assert_planes_close(fg, fo, TOL[precision], "f^{k+1}")
    assert_planes_close(Ig, Io, TOL[precision], "I^{k+1}")
    assert_fields_close(rec, Fo, TOL[precision], wl.dim, "moments of f^{k+1}")


def test_normal_shock_conserves_fluxes_at_convergence():
    """A converged Mach-5 shock (the paper's case: 200 L0 at spacing 0.25 L0, Z_v = 26, CIS
    to its tolerance eps < 2e-6) carries uniform mass,
    momentum and energy fluxes through the domain: rho u, rho u^2 + rho T_t + sigma_xx and
    u (E + p + sigma_xx) + q (gas modes and radiation) from the library's field records;
    mass and momentum equal those of the upstream state.  Cell values of a resolved shock
    differ from the conserved face fluxes by the scheme's truncation error, hence 1e-2."""
    wl = gi.workloads.with_solver(gi.workloads.normal_shock(length=200.0, dx=0.25, n_xi=64, n_theta=48),
                                  precision="fp64", order=2, relax_block=16, venkat_K=0.01)
    M = gi.fields.shock_fields(wl)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 1, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 0,
                                       noise=0.0)
    ctx = create(wl)
    try:
        G.gsis_set_distributions(ctx, f, I)
        it, hist = G.gsis_solve(ctx, G.GSIS_MODE_CIS, 6000, 2e-6)
        F = G.gsis_get_fields(ctx, wl.mesh.n_cells)
    finally:
        G.gsis_destroy(ctx)
    assert hist[-1] < 2e-6, "CIS reached %.2e after %d iterations" % (hist[-1], it)
    d_r, d_v = wl.model.d_r, wl.model.d_v
    rho, u, Tt, Tr, Tv = F[:, 0], F[:, 1], F[:, 4], F[:, 5], F[:, 6]
    sxx = F[:, 20]
    q = F[:, 8] + F[:, 11] + F[:, 14] + F[:, 17]
    p = rho * Tt
    E = rho * (0.5 * u * u + 0.5 * (3.0 * Tt + d_r * Tr + d_v * Tv))
    fluxes = {"mass": rho * u, "momentum": rho * u * u + p + sxx, "energy": u * (E + p + sxx) + q}
    for name, fl in fluxes.items():
        dev = (fl.max() - fl.min()) / abs(fl.mean())
        assert dev < 1e-2, "%s flux varies by %.2e of its mean" % (name, dev)
    up = wl.mesh.patches[0]
    assert abs(fluxes["mass"].mean() - up.rho * up.u[0]) < 1e-2 * up.rho * up.u[0]
    assert abs(fluxes["momentum"].mean() - up.rho * (up.u[0] ** 2 + up.T_t)) < 1e-2 * up.rho * up.u[0] ** 2


@pytest.mark.parametrize("precision,mode", [("fp64", 0), ("fp32", 0), ("fp32", 1), ("fp32", 2)])
def test_graph_path_matches_stepwise_launches(precision, mode):
    """On a non-default stream the inner loop of the synthetic solve runs as captured CUDA
    graphs (two of them in the mixed schedule, mode 2); on the default stream it is launched
    kernel by kernel.  Both orders of work are the same, so the results are identical."""
    import torch
    wl = gi.workloads.with_solver(CASES["cavity72"](), precision=precision, order=2, relax_block=16, max_inner=40,
                                  tol_inner=1e-6, macro_fp32=mode)
    f, I = _inputs(wl, 7, precision)
    stream = torch.cuda.Stream()
    out = []
    for st in (0, stream.cuda_stream):
        ctx = create(wl, st)
        try:
            G.gsis_set_distributions(ctx, f, I)
            eps = [G.gsis_step(ctx, G.GSIS_MODE_GSIS) for _ in range(2)]
            fg, Ig = G.gsis_get_distributions(ctx, wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0])
            out.append((eps, fg, G.gsis_get_fields(ctx, wl.mesh.n_cells)))
        finally:
            G.gsis_destroy(ctx)
    (ea, fa, Fa), (eb, fb, Fb) = out
    assert ea == eb
    assert np.array_equal(fa, fb) and np.array_equal(Fa, Fb)
