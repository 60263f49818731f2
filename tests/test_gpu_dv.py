"""GPU parity with the temperature-dependent vibrational degrees of freedom
d_v(T_v) = 2 x / (e^x - 1), x = Tv_ref / T_v (Section 2.1), against the FP64 oracle on
the same seeded inputs: one CIS iteration (vibrational energy and its inverse in the
moments, T_tv by Newton and A, Mix at d_v(T_v) in the reference distributions, wall
re-emission) and one GSIS iteration (conservative/primitive conversion, the re-derived
source and its Jacobian, NSF conductivities at the face's d_v, synchronisation).
Tolerances as the other parity tests: FP64 1e-10, FP32 1e-5."""
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
TREF = 3.0


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    G.load()


def _dv(wl):
    return gi.workloads.with_model(wl, dv_temperature_dependent=True, Tv_ref=TREF)


def _inputs(wl, seed, precision):
    M = gi.fields.smooth_random_fields(wl.mesh.cell_centroid, seed, u_scale=0.2)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, wl.dim, wl.model.d_r, wl.model.d_v,
                                       wl.model.sigma_R, seed + 1, noise=0.02)
    if precision == "fp32":
        f, I = f.astype(np.float32).astype(np.float64), I.astype(np.float32).astype(np.float64)
    return f, I


CIS_CASES = {"slab64": lambda: gi.workloads.slab(64), "cavity338": lambda: gi.workloads.cavity(n_side=13)}


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("case", sorted(CIS_CASES))
def test_cis_step_with_dv_of_T_matches_oracle(case, precision):
    wl = _dv(gi.workloads.with_solver(CIS_CASES[case](), precision=precision, order=2, relax_block=16))
    f, I = _inputs(wl, 7, precision)
    ctx = create(wl)
    try:
        G.gsis_set_distributions(ctx, f, I)
        rec0 = G.gsis_get_fields(ctx, wl.mesh.n_cells)
        eps = G.gsis_step(ctx, G.GSIS_MODE_CIS)
        fg, Ig = G.gsis_get_distributions(ctx, wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0])
        rec1 = G.gsis_get_fields(ctx, wl.mesh.n_cells)
    finally:
        G.gsis_destroy(ctx)
    F0 = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, wl.dim, wl.model)
    fo, Io = K.kinetic_sweep(f, I, wl, relax_block=16, F=F0)
    F1 = K.moments(fo, Io, wl.xi, wl.w, wl.omega, wl.wo, wl.dim, wl.model)
    tol = TOL[precision]
    assert_fields_close(rec0, F0, tol, wl.dim, "moments of f^k")
    assert_planes_close(fg, fo, tol, "f^{k+1}")
    assert_planes_close(Ig, Io, tol, "I^{k+1}")
    assert_fields_close(rec1, F1, tol, wl.dim, "moments of f^{k+1}")
    geo = K.Geometry(wl.mesh)
    assert abs(eps - OG.epsilon(F1, F0, geo.vol, wl.model, wl.dim)) <= 10 * tol * eps
    # the model differs from constant d_v on these states
    const = gi.workloads.with_model(wl, dv_temperature_dependent=False)
    fc, _ = K.kinetic_sweep(f, I, const, relax_block=16)
    assert np.abs(fc[..., 3] - fo[..., 3]).max() > 1e-3 * np.abs(fo[..., 3]).max()


GSIS_CASES = {
    "slab16": lambda: gi.workloads.slab(16, Kn=0.05),
    "cavity72": lambda: gi.workloads.cavity(n_side=6, Kn=0.05, Kn_p=1.0),
    "cylinder64": lambda: gi.workloads.cylinder(n_theta=8, n_radial=4, n_v=16, n_polar=4, n_azim=8, Mach=0.5,
                                                Kn=0.05, Kn_p=1.0),
}


@pytest.mark.parametrize("case", sorted(GSIS_CASES))
def test_gsis_step_with_dv_of_T_matches_oracle_fp64(case):
    wl = _dv(gi.workloads.with_solver(GSIS_CASES[case](), precision="fp64", order=2, relax_block=16, max_inner=12,
                                      tol_inner=0.0, macro_sweeps=4, cfl_macro=200.0))
    f, I = _inputs(wl, 11, "fp64")
    ctx = create(wl)
    try:
        G.gsis_set_distributions(ctx, f, I)
        eps = G.gsis_step(ctx, G.GSIS_MODE_GSIS)
        fg, Ig = G.gsis_get_distributions(ctx, wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0])
        rec = G.gsis_get_fields(ctx, wl.mesh.n_cells)
    finally:
        G.gsis_destroy(ctx)
    geo = K.Geometry(wl.mesh)
    fo, Io, eps_o, Fo = OG.gsis_step(f, I, wl, geo, MA.Faces(geo))
    assert_planes_close(fg, fo, TOL["fp64"], "f^{k+1}")
    assert_planes_close(Ig, Io, TOL["fp64"], "I^{k+1}")
    assert_fields_close(rec, Fo, TOL["fp64"], wl.dim, "moments of f^{k+1}")
    assert abs(eps - eps_o) <= 1e-9 * eps_o
