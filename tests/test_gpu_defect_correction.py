"""GPU parity of the defect-corrected GSIS step (solver.defect_correction, an extension):
the synthetic equations R(W) - R(W_h) + r_h = 0, r_h the moments of the kinetic residual
at f^{k+1/2}.  One iteration against the FP64 oracle on the GSIS parity cases (closed and
far-field domains, 1-D, 2-D and 3-D, orders 1 and 2), the fixed-point property at a
kinetic steady state, and the refusal for velocity shards."""
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


CASES = {
    "slab16": lambda: gi.workloads.slab(16, Kn=0.05),
    "cavity72": lambda: gi.workloads.cavity(n_side=6, Kn=0.05, Kn_p=1.0),
    "cylinder64": lambda: gi.workloads.cylinder(n_theta=8, n_radial=4, n_v=16, n_polar=4, n_azim=8, Mach=0.5,
                                                Kn=0.05, Kn_p=1.0),
    "box162": lambda: gi.workloads.Workload("box162", gi.mesh.box_tetrahedra(3, seed=4),
                                            *gi.quadrature.trapezoid_nd(6, 4.5, 3),
                                            *gi.quadrature.photon_product(2, 4),
                                            gi.workloads.ModelParams(Kn=0.1, Kn_p=1.0)),
}


def _inputs(wl, seed, precision):
    M = gi.fields.smooth_random_fields(wl.mesh.cell_centroid, seed, u_scale=0.2)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, wl.dim, wl.model.d_r, wl.model.d_v,
                                       wl.model.sigma_R, seed + 1, noise=0.02)
    if precision == "fp32":
        f, I = f.astype(np.float32).astype(np.float64), I.astype(np.float32).astype(np.float64)
    return f, I


def _wl(case, precision, order):
    return gi.workloads.with_solver(CASES[case](), precision=precision, order=order, relax_block=16, max_inner=12,
                                    tol_inner=0.0, macro_sweeps=4, cfl_macro=200.0, defect_correction=1,
                                    tc_moments=0 if case == "box162" else 1)


def _gpu(wl, f, I, modes):
    ctx = create(wl)
    try:
        G.gsis_set_distributions(ctx, f, I)
        eps = [G.gsis_step(ctx, m) for m in modes]
        fg, Ig = G.gsis_get_distributions(ctx, wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0])
        return fg, Ig, G.gsis_get_fields(ctx, wl.mesh.n_cells), eps
    finally:
        G.gsis_destroy(ctx)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("case", sorted(CASES))
def test_corrected_gsis_step_matches_oracle_fp64(case, order):
    wl = _wl(case, "fp64", order)
    f, I = _inputs(wl, 21, "fp64")
    fg, Ig, rec, eps = _gpu(wl, f, I, [G.GSIS_MODE_GSIS])
    geo = K.Geometry(wl.mesh)
    fo, Io, eo, Fo = OG.gsis_step(f, I, wl, geo, MA.Faces(geo))
    assert_planes_close(fg, fo, TOL["fp64"], "f^{k+1}")
    assert_planes_close(Ig, Io, TOL["fp64"], "I^{k+1}")
    assert_fields_close(rec, Fo, TOL["fp64"], wl.dim, "fields")
    assert abs(eps[0] - eo) <= 1e-9 * eo


@pytest.mark.parametrize("case", ["cavity72", "cylinder64"])
def test_corrected_gsis_step_matches_oracle_fp32(case):
    wl = _wl(case, "fp32", 2)
    f, I = _inputs(wl, 23, "fp32")
    fg, Ig, rec, eps = _gpu(wl, f, I, [G.GSIS_MODE_GSIS])
    geo = K.Geometry(wl.mesh)
    fo, Io, eo, Fo = OG.gsis_step(f, I, wl, geo, MA.Faces(geo))
    assert_planes_close(fg, fo, TOL["fp32"], "f^{k+1}")
    assert_fields_close(rec, Fo, TOL["fp32"], wl.dim, "fields")


def test_kinetic_steady_state_is_kept_by_the_corrected_step():
    """From a kinetic steady state (CIS on the GPU to eps < 1e-12, FP64) one corrected GSIS
    step moves the fields by rounding only; the paper's step moves them by the synthetic
    equations' discretisation mismatch."""
    base = gi.workloads.with_solver(gi.workloads.slab(16, Kn=0.1), precision="fp64", order=2, relax_block=16,
                                    max_inner=400, tol_inner=1e-12)
    eps = {}
    for dc in (0, 1):
        wl = gi.workloads.with_solver(base, defect_correction=dc)
        ctx = create(wl)
        try:
            G.gsis_init_fields(ctx, gi.fields.uniform_fields(16, T=1.25))
            it, hist = G.gsis_solve(ctx, G.GSIS_MODE_CIS, 5000, 1e-12)
            assert hist[-1] < 1e-12
            eps[dc] = G.gsis_step(ctx, G.GSIS_MODE_GSIS)
        finally:
            G.gsis_destroy(ctx)
    assert eps[1] < 1e-10, eps
    assert eps[0] > 1e-4, eps


def test_velocity_shards_refuse_the_correction():
    wl = gi.workloads.with_solver(gi.workloads.slab(8), precision="fp64", defect_correction=1)
    ctx = create(wl)
    try:
        with pytest.raises(G.GsisError) as e:
            G.gsis_shard_setup(ctx, wl.xi[:, :1], wl.w, wl.omega, wl.wo)
        assert e.value.code == G.GSIS_ERR_UNSUPPORTED
    finally:
        G.gsis_destroy(ctx)


def test_corrected_gsis_converges_on_the_slab_where_the_paper_step_stalls():
    """The 64-cell slab at Kn = 0.1 (FP64, order 2, synchronisation weight 0.8): the paper's
    GSIS step stops near eps = 4e-7, the corrected one reaches 1e-8."""
    out = {}
    for dc in (0, 1):
        wl = gi.workloads.with_solver(gi.workloads.slab(64, Kn=0.1), precision="fp64", order=2, relax_block=16,
                                      max_inner=100, tol_inner=1e-7, n_cis_precond=3, sync_relax=0.8,
                                      defect_correction=dc)
        M = gi.fields.uniform_fields(64, T=1.25)
        f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 1, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 0,
                                           noise=0.0)
        ctx = create(wl)
        try:
            G.gsis_set_distributions(ctx, f, I)
            it, hist = G.gsis_solve(ctx, G.GSIS_MODE_GSIS, 300, 1e-8)
        finally:
            G.gsis_destroy(ctx)
        out[dc] = (it, hist[-1])
    assert out[1][1] < 1e-8, out
    assert out[0][1] > 1e-7, out
