"""GPU parity of mirror-plane (SYMMETRY) patches against the FP64 oracle: specular
reflection of molecules and photons in the kinetic sweep, the mirror flux of the
synthetic equations and the kinetic boundary flux, on a half slab (mirror at x = 0.5)
and a half cavity (mirror as the left side); and the mirror trajectory: with Jacobi
relaxation the half slab follows the symmetric full slab iterate by iterate."""
import dataclasses

import numpy as np
import pytest

import gsis_inputs as gi
from gsis_inputs import mesh as GM
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


def _half_slab(n=16, **kw):
    wl = gi.workloads.slab(2 * n, **kw)
    m = GM.slab_1d(n, 0.5, patches=[GM.Patch(GM.WALL, T_t=1.5), GM.Patch(GM.SYMMETRY)])
    return dataclasses.replace(wl, mesh=m, name="halfslab%d" % n)


def _half_cavity(n_side=8, **kw):
    wl = gi.workloads.cavity(n_side=n_side, **kw)
    p = list(wl.mesh.patches)
    p[3] = GM.Patch(GM.SYMMETRY)
    return dataclasses.replace(wl, mesh=dataclasses.replace(wl.mesh, patches=p), name="halfcavity")


CASES = {"halfslab16": lambda: _half_slab(16, Kn=0.05), "halfcavity128": lambda: _half_cavity(8, Kn=0.05, Kn_p=1.0)}


def _inputs(wl, seed, precision):
    M = gi.fields.smooth_random_fields(wl.mesh.cell_centroid, seed, u_scale=0.2)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, wl.dim, wl.model.d_r, wl.model.d_v,
                                       wl.model.sigma_R, seed + 1, noise=0.02)
    if precision == "fp32":
        f, I = f.astype(np.float32).astype(np.float64), I.astype(np.float32).astype(np.float64)
    return f, I


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_cis_step_with_a_mirror_plane_matches_oracle(case, precision, order):
    wl = gi.workloads.with_solver(CASES[case](), precision=precision, order=order, relax_block=16)
    f, I = _inputs(wl, 3, precision)
    ctx = create(wl)
    try:
        G.gsis_set_distributions(ctx, f, I)
        G.gsis_step(ctx, G.GSIS_MODE_CIS)
        fg, Ig = G.gsis_get_distributions(ctx, wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0])
        rec = G.gsis_get_fields(ctx, wl.mesh.n_cells)
    finally:
        G.gsis_destroy(ctx)
    fo, Io = K.kinetic_sweep(f, I, wl, relax_block=16)
    tol = TOL[precision]
    assert_planes_close(fg, fo, tol, "f^{k+1}")
    assert_planes_close(Ig, Io, tol, "I^{k+1}")
    assert_fields_close(rec, K.moments(fo, Io, wl.xi, wl.w, wl.omega, wl.wo, wl.dim, wl.model), tol, wl.dim, "fields")


@pytest.mark.parametrize("case", sorted(CASES))
def test_gsis_step_with_a_mirror_plane_matches_oracle_fp64(case):
    wl = gi.workloads.with_solver(CASES[case](), precision="fp64", order=2, relax_block=16, max_inner=12,
                                  tol_inner=0.0, macro_sweeps=4, cfl_macro=200.0)
    f, I = _inputs(wl, 5, "fp64")
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
    assert_fields_close(rec, Fo, TOL["fp64"], wl.dim, "fields")
    assert abs(eps - eps_o) <= 1e-9 * eps_o


def test_half_slab_follows_the_symmetric_full_slab():
    kw = dict(Kn=0.3, Kn_p=1.0)
    full = gi.workloads.with_solver(gi.workloads.slab(16, T_left=1.5, T_right=1.5, **kw), precision="fp64",
                                    order=1, relax_block=1)
    half = gi.workloads.with_solver(_half_slab(8, **kw), precision="fp64", order=1, relax_block=1)
    out = []
    for wl in (full, half):
        M = gi.fields.uniform_fields(wl.mesh.n_cells, T=1.0)
        f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 1, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 0,
                                           noise=0.0)
        ctx = create(wl)
        try:
            G.gsis_set_distributions(ctx, f, I)
            eps = [G.gsis_step(ctx, G.GSIS_MODE_CIS) for _ in range(10)]
            out.append((eps, G.gsis_get_distributions(ctx, wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0])))
        finally:
            G.gsis_destroy(ctx)
    (ef, (ff, If)), (eh, (fh, Ih)) = out
    assert np.allclose(ef, eh, rtol=1e-12, atol=0.0)
    assert np.abs(fh - ff[:8]).max() <= 1e-12 * np.abs(ff).max()
    assert np.abs(Ih - If[:8]).max() <= 1e-12 * np.abs(If).max()


def test_mirror_planes_refuse_velocity_sharding():
    wl = gi.workloads.with_solver(_half_slab(8), precision="fp64")
    ctx = create(wl)
    try:
        with pytest.raises(G.GsisError) as e:
            G.gsis_shard_setup(ctx, wl.xi, wl.w, wl.omega, wl.wo)
        assert e.value.code == G.GSIS_ERR_UNSUPPORTED
    finally:
        G.gsis_destroy(ctx)
