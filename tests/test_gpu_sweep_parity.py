"""GPU parity of one conventional iteration (the kinetic sweep of Eq. dis_micro and the
moments of Eq. getmoment) against the FP64 oracle on the same seeded inputs.

Tolerances: FP64 path 1e-10 relative; FP32 path 1e-5 relative (macroscopic fields,
per plane of f against its largest value).  The FP32 oracle input is the FP32-rounded
distribution, so the comparison measures arithmetic only.
"""
import numpy as np
import pytest

import gsis_inputs as gi
from oracle import gsis as OG
from oracle import kinetic as K
from paper_2601_03935_gb300 import build
from paper_2601_03935_gb300 import gsis as G

from _ctx import assert_fields_close, assert_planes_close, create

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    G.load()


def _inputs(wl, seed, precision, u_scale=0.3, smooth=False):
    if smooth:
        M = gi.fields.smooth_random_fields(wl.mesh.cell_centroid, seed, u_scale=u_scale)
    else:
        M = gi.fields.random_macro_fields(wl.mesh.n_cells, wl.dim, seed, u_scale=u_scale)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, wl.dim, wl.model.d_r, wl.model.d_v,
                                       wl.model.sigma_R, seed + 1)
    if precision == "fp32":
        f, I = f.astype(np.float32).astype(np.float64), I.astype(np.float32).astype(np.float64)
    return f, I


def _run(wl, f, I):
    ctx = create(wl)
    try:
        G.gsis_set_distributions(ctx, f, I)
        rec0 = G.gsis_get_fields(ctx, wl.mesh.n_cells)
        eps = G.gsis_step(ctx, G.GSIS_MODE_CIS)
        fg, Ig = G.gsis_get_distributions(ctx, wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0])
        rec1 = G.gsis_get_fields(ctx, wl.mesh.n_cells)
        return rec0, rec1, fg, Ig, eps
    finally:
        G.gsis_destroy(ctx)


CASES = {
    # 338 cells: 21 blocks of 16 and a ragged block of 2; 784 velocities: 12 full chunks
    # of 64 and a ragged one; 64 photon directions
    "cavity338": lambda: gi.workloads.cavity(n_side=13),
    # the same mesh on an unstructured disc velocity mesh: 477 velocities (7 full chunks
    # and a ragged one), no tensor product
    "cavity338_disc": lambda: gi.workloads.cavity(n_side=13, n_v=14, rule="disc"),
    # 64 cells, 32 Gauss-Hermite velocities and 16 photon directions (one ragged chunk each)
    "slab64": lambda: gi.workloads.slab(64),
}


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_cis_step_matches_oracle(case, precision, order):
    wl = gi.workloads.with_solver(CASES[case](), precision=precision, order=order, relax_block=16)
    f, I = _inputs(wl, 7, precision)
    rec0, rec1, fg, Ig, eps = _run(wl, f, I)
    F0 = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, wl.dim, wl.model)
    fo, Io = K.kinetic_sweep(f, I, wl, relax_block=16, F=F0)
    F1 = K.moments(fo, Io, wl.xi, wl.w, wl.omega, wl.wo, wl.dim, wl.model)
    tol = TOL[precision]
    assert_fields_close(rec0, F0, tol, wl.dim, "moments of f^k")
    assert_planes_close(fg, fo, tol, "f^{k+1}")
    assert_planes_close(Ig, Io, tol, "I^{k+1}")
    assert_fields_close(rec1, F1, tol, wl.dim, "moments of f^{k+1}")
    eps_o = OG.epsilon(F1, F0, wl.mesh.cell_volume, wl.model, wl.dim)
    assert abs(eps - eps_o) <= 1e-4 * eps_o if precision == "fp32" else abs(eps - eps_o) <= 1e-9 * eps_o


@pytest.mark.parametrize("tc,block", [(0, 16), (1, 16), (2, 16), (2, 8), (2, 1), (2, 5), (2, 64)])
def test_fp32_moment_engines(tc, block):
    """Every place the FP32 gas moments are contracted: CUDA cores (tc 0), the tensor-core
    standalone pass (tc >= 1, the moments of f^k) and the tensor-core sweep epilogue (tc 2,
    blocks dividing 16; blocks 5 and 64 keep the CUDA-core epilogue), on 338 cells (ragged
    last tile) x 784 velocities (ragged last chunk), flow speeds up to 0.6."""
    wl = gi.workloads.with_solver(CASES["cavity338"](), precision="fp32", order=2, relax_block=block, tc_moments=tc)
    f, I = _inputs(wl, 17, "fp32", u_scale=0.6)
    rec0, rec1, fg, Ig, _ = _run(wl, f, I)
    F0 = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, wl.dim, wl.model)
    fo, Io = K.kinetic_sweep(f, I, wl, relax_block=block, F=F0)
    F1 = K.moments(fo, Io, wl.xi, wl.w, wl.omega, wl.wo, wl.dim, wl.model)
    assert_fields_close(rec0, F0, 1e-5, wl.dim, "moments of f^k")
    assert_planes_close(fg, fo, 1e-5, "f^{k+1}")
    assert_fields_close(rec1, F1, 1e-5, wl.dim, "moments of f^{k+1}")


@pytest.mark.parametrize("block", [1, 5, 49, 64])
def test_block_sizes_and_jacobi(block):
    wl = gi.workloads.with_solver(gi.workloads.cavity(n_side=9), precision="fp64", order=2, relax_block=block)
    f, I = _inputs(wl, 11, "fp64", smooth=True)
    _, rec1, fg, Ig, _ = _run(wl, f, I)
    fo, Io = K.kinetic_sweep(f, I, wl, relax_block=block)
    assert_planes_close(fg, fo, 1e-10, "f block=%d" % block)
    assert_planes_close(Ig, Io, 1e-10, "I block=%d" % block)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_zero_normal_velocity(precision):
    """An odd velocity grid contains xi = 0, where xi . n = 0 on every face: no side writes
    the face's upwind value and the sweep skips the face (order 2), as the oracle does."""
    wl = gi.workloads.with_solver(gi.workloads.cavity(n_side=9, n_v=15), precision=precision, order=2,
                                  relax_block=16)
    assert np.any(np.all(wl.xi == 0.0, axis=1))
    f, I = _inputs(wl, 13, precision)
    _, rec1, fg, Ig, _ = _run(wl, f, I)
    fo, Io = K.kinetic_sweep(f, I, wl, relax_block=16)
    assert_planes_close(fg, fo, TOL[precision], "f")
    assert_planes_close(Ig, Io, TOL[precision], "I")


def test_largest_fp32_block():
    wl = gi.workloads.with_solver(gi.workloads.cavity(n_side=9), precision="fp32", order=2, relax_block=64)
    f, I = _inputs(wl, 12, "fp32", smooth=True)
    _, _, fg, Ig, _ = _run(wl, f, I)
    fo, Io = K.kinetic_sweep(f, I, wl, relax_block=64)
    assert_planes_close(fg, fo, 1e-5, "f block=64")
    assert_planes_close(Ig, Io, 1e-5, "I block=64")


def test_mesh_smaller_than_one_block():
    wl = gi.workloads.with_solver(gi.workloads.slab(5), precision="fp64", order=2, relax_block=16)
    f, I = _inputs(wl, 3, "fp64")
    _, _, fg, Ig, _ = _run(wl, f, I)
    fo, Io = K.kinetic_sweep(f, I, wl, relax_block=16)
    assert_planes_close(fg, fo, 1e-10, "f")
    assert_planes_close(Ig, Io, 1e-10, "I")


def test_far_field_and_density_scaled_absorption():
    wl = gi.workloads.cylinder(n_theta=24, n_radial=6, n_v=24, n_azim=12, Mach=2.0)
    wl = gi.workloads.with_solver(wl, precision="fp64", order=2, relax_block=16)
    M = gi.fields.random_macro_fields(wl.mesh.n_cells, 2, 5, u_scale=1.0)
    M[:, 4:8] *= 0.5
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 2, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 6)
    _, rec1, fg, Ig, _ = _run(wl, f, I)
    fo, Io = K.kinetic_sweep(f, I, wl, relax_block=16)
    assert_planes_close(fg, fo, 1e-10, "f")
    assert_planes_close(Ig, Io, 1e-10, "I")


def test_full_size_cavity_sampled_blocks():
    """20 000 cells x 784 velocities x 64 directions in the benchmark's configuration
    (FP32, order 2, blocks of 16): whole blocks at the start, middle, on the lid and at
    the end are recomputed by the oracle."""
    wl = gi.workloads.with_solver(gi.workloads.cavity(n_side=100), precision="fp32", order=2, relax_block=16)
    f, I = _inputs(wl, 21, "fp32", smooth=True)
    _, _, fg, Ig, _ = _run(wl, f, I)
    nc = wl.mesh.n_cells
    lid = int(np.argmax(wl.mesh.cell_centroid[:, 1] + 1e-3 * wl.mesh.cell_centroid[:, 0]))
    blocks = sorted({0, nc // 32, lid // 16, (nc - 1) // 16})
    cells = np.concatenate([np.arange(b * 16, min(b * 16 + 16, nc)) for b in blocks])
    fo, Io = K.kinetic_sweep(f, I, wl, relax_block=16, cells=cells)
    assert_planes_close(fg[cells], fo, 1e-5, "f sampled")
    assert_planes_close(Ig[cells], Io, 1e-5, "I sampled")


def test_full_size_cylinder_sampled_blocks():
    """The Mach-5 cylinder at full size: 40 000 triangles x 2304 velocities (48 x 48,
    truncated at 8 sqrt(2 T_0)) x 96 photon directions, density-scaled absorption, FP32,
    order 2, blocks of 16, from a smooth state around the free stream.  Whole blocks at
    the start, next to the wall, next to the far field, in the middle and at the end are
    recomputed by the oracle."""
    wl = gi.workloads.with_solver(gi.workloads.cylinder(), precision="fp32", order=2, relax_block=16)
    assert wl.mesh.n_cells == 40000 and wl.xi.shape[0] == 2304 and wl.omega.shape[0] == 96
    far = wl.mesh.patches[1]
    M = gi.fields.smooth_random_fields(wl.mesh.cell_centroid / 8.0, 23, u_scale=0.5)
    M[:, 1] += far.u[0]
    M[:, 4:8] *= far.T_t
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 2, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 24)
    f, I = f.astype(np.float32).astype(np.float64), I.astype(np.float32).astype(np.float64)
    _, _, fg, Ig, _ = _run(wl, f, I)
    nc = wl.mesh.n_cells
    m = wl.mesh
    bnd = m.face_nbr < 0
    wall = m.face_owner[bnd & (m.face_nbr == -1)]
    farc = m.face_owner[bnd & (m.face_nbr == -2)]
    blocks = sorted({0, int(wall[len(wall) // 3]) // 16, int(farc[len(farc) // 2]) // 16, nc // 32,
                     (nc - 1) // 16})
    cells = np.concatenate([np.arange(b * 16, min(b * 16 + 16, nc)) for b in blocks])
    fo, Io = K.kinetic_sweep(f, I, wl, relax_block=16, cells=cells)
    assert_planes_close(fg[cells], fo, 1e-5, "f sampled")
    assert_planes_close(Ig[cells], Io, 1e-5, "I sampled")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_positivity_bound_on_the_impulsive_cylinder(precision):
    """Order 2 from the impulsive Mach-5 free stream around a cylinder with the positivity
    bound theta = 0.1: the bound is active on many values and the iteration equals the
    oracle's."""
    wl = gi.workloads.with_solver(gi.workloads.cylinder(n_theta=8, n_radial=4, n_v=16, n_polar=4, n_azim=8),
                                  precision=precision, order=2, relax_block=16, venkat_K=0.01, positivity=0.1)
    far = wl.mesh.patches[1]
    M = gi.fields.uniform_fields(wl.mesh.n_cells, rho=far.rho, u=far.u, T=far.T_t)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 2, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 0,
                                       noise=0.0)
    if precision == "fp32":
        f, I = f.astype(np.float32).astype(np.float64), I.astype(np.float32).astype(np.float64)
    _, rec1, fg, Ig, _ = _run(wl, f, I)
    F0 = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, 2, wl.model)
    fo, Io = K.kinetic_sweep(f, I, wl, relax_block=16, F=F0)
    fu, _ = K.kinetic_sweep(f, I, gi.workloads.with_solver(wl, positivity=0.0), relax_block=16, F=F0)
    assert np.mean(fo != fu) > 0.1
    assert_planes_close(fg, fo, TOL[precision], "f^{k+1}")
    assert_planes_close(Ig, Io, TOL[precision], "I^{k+1}")
    assert_fields_close(rec1, K.moments(fo, Io, wl.xi, wl.w, wl.omega, wl.wo, 2, wl.model), TOL[precision], 2,
                        "fields")


def test_twenty_iterations_follow_the_oracle():
    """Twenty CIS iterations on the 8 x 8 heated-lid cavity at Kn = 1, order 2, FP64: the
    convergence measure of every iteration and the final distributions equal the oracle's
    (fields, coefficients and sweeps accumulate over the iterations)."""
    wl = gi.workloads.with_solver(gi.workloads.cavity(n_side=8, Kn=1.0, Kn_p=10.0), precision="fp64", order=2,
                                  relax_block=16)
    M = gi.fields.uniform_fields(wl.mesh.n_cells)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 2, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 0,
                                       noise=0.0)
    ctx = create(wl)
    try:
        G.gsis_set_distributions(ctx, f, I)
        eps_g = [G.gsis_step(ctx, G.GSIS_MODE_CIS) for _ in range(20)]
        fg, Ig = G.gsis_get_distributions(ctx, wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0])
    finally:
        G.gsis_destroy(ctx)
    geo = K.Geometry(wl.mesh)
    eps_o = []
    for _ in range(20):
        f, I, e, _ = OG.cis_step(f, I, wl, geo)
        eps_o.append(e)
    assert np.allclose(eps_g, eps_o, rtol=1e-9, atol=0.0)
    assert_planes_close(fg, f, 1e-9, "f after 20 iterations")
    assert_planes_close(Ig, I, 1e-9, "I after 20 iterations")


def test_divergence_is_reported_and_cleared():
    """A non-finite distribution value (injected on the host) makes the next iteration
    report DIVERGED; a following valid state iterates normally again."""
    wl = gi.workloads.with_solver(gi.workloads.cavity(n_side=9), precision="fp64", order=2, relax_block=16)
    f, I = _inputs(wl, 11, "fp64", smooth=True)
    bad = f.copy()
    bad[37, 100, 0] = np.nan
    ctx = create(wl)
    try:
        G.gsis_set_distributions(ctx, bad, I)
        with pytest.raises(G.GsisError) as e:
            G.gsis_step(ctx, G.GSIS_MODE_CIS)
        assert e.value.code == G.GSIS_ERR_DIVERGED
        G.gsis_set_distributions(ctx, f, I)
        assert np.isfinite(G.gsis_step(ctx, G.GSIS_MODE_CIS))
    finally:
        G.gsis_destroy(ctx)
