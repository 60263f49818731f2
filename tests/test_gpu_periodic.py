"""GPU parity on a periodic domain: a uniform row of cells closed into a ring by one face
from the last cell to the first (gsis_inputs.mesh.ring_1d), with period = L, so that
every centroid difference across that face (least-squares stencils, face offsets of the
second-order reconstruction, face distances of the synthetic equations) is the minimal
image.  One CIS and one GSIS iteration against the FP64 oracle on the same seeded
periodic state, orders 1 and 2; and the same mesh passed without its period, against the
oracle on that non-periodic geometry (at order 2 the two differ)."""
import dataclasses
import math

import numpy as np
import pytest

import gsis_inputs as gi
from gsis_inputs import quadrature as Q
from oracle import gsis as OG
from oracle import kinetic as K
from oracle import macro as MA
from paper_2601_03935_gb300 import build
from paper_2601_03935_gb300 import gsis as G

from _ctx import assert_fields_close, assert_planes_close, create

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-10}
L = 4.0


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    G.load()


def _ring(n, order, precision, periodic=True):
    mesh = gi.mesh.ring_1d(n, L)
    if not periodic:
        mesh = dataclasses.replace(mesh, period=0.0)
    xi, w = Q.gauss_hermite_1d(24)
    om, wo = Q.gauss_legendre_slab(8)
    model = gi.workloads.ModelParams(Kn=0.1, Kn_p=1.0, sigma_R=0.05)
    solver = gi.workloads.SolverParams(precision=precision, order=order, relax_block=8, max_inner=12,
                                       tol_inner=0.0, macro_sweeps=4, cfl_macro=200.0)
    return gi.workloads.Workload("ring%d" % n, mesh, xi, w, om, wo, model, solver)


def _state(wl, precision):
    """A smooth periodic state: one and two wavelengths of density, velocity and the
    temperatures along the ring, then a seeded perturbation of the distributions."""
    x = wl.mesh.cell_centroid[:, 0]
    k = 2.0 * math.pi / L
    M = gi.fields.uniform_fields(wl.mesh.n_cells)
    M[:, 0] = 1.0 + 0.2 * np.cos(k * x)
    M[:, 1] = 0.15 * np.sin(k * x)
    M[:, 4] = 1.0 + 0.1 * np.cos(2 * k * x + 0.3)
    M[:, 5] = 1.0 + 0.08 * np.sin(k * x + 0.7)
    M[:, 6] = 1.0 + 0.05 * np.cos(k * x + 1.1)
    M[:, 7] = 1.0 + 0.04 * np.sin(2 * k * x)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, wl.dim, wl.model.d_r, wl.model.d_v,
                                       wl.model.sigma_R, 5, noise=0.02)
    if precision == "fp32":
        f, I = f.astype(np.float32).astype(np.float64), I.astype(np.float32).astype(np.float64)
    return f, I


def _gpu(wl, f, I, mode):
    ctx = create(wl)
    try:
        G.gsis_set_distributions(ctx, f, I)
        eps = G.gsis_step(ctx, mode)
        fg, Ig = G.gsis_get_distributions(ctx, wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0])
        return fg, Ig, G.gsis_get_fields(ctx, wl.mesh.n_cells), eps
    finally:
        G.gsis_destroy(ctx)


def _oracle(wl, f, I, mode):
    geo = K.Geometry(wl.mesh)
    if mode == G.GSIS_MODE_GSIS:
        return OG.gsis_step(f, I, wl, geo, MA.Faces(geo))
    return OG.cis_step(f, I, wl, geo)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("mode", ["cis", "gsis"])
def test_periodic_ring_matches_oracle(mode, order, precision):
    md = G.GSIS_MODE_GSIS if mode == "gsis" else G.GSIS_MODE_CIS
    wl = _ring(24, order, precision)
    f, I = _state(wl, precision)
    fg, Ig, rec, eps = _gpu(wl, f, I, md)
    fo, Io, eo, Fo = _oracle(wl, f, I, md)
    tol = TOL[precision]
    assert_planes_close(fg, fo, tol, "f")
    assert_planes_close(Ig, Io, tol, "I")
    assert_fields_close(rec, Fo, tol, wl.dim, "fields")
    assert abs(eps - eo) <= max(tol, 1e-6 if precision == "fp32" else 0.0) * max(abs(eo), 1e-30)


@pytest.mark.parametrize("mode", ["cis", "gsis"])
def test_the_period_changes_the_second_order_path(mode):
    """Without its period the closing face joins cells L - dx apart: the least-squares
    stencils and face offsets there change, and the GPU follows the oracle either way."""
    md = G.GSIS_MODE_GSIS if mode == "gsis" else G.GSIS_MODE_CIS
    out = {}
    for periodic in (True, False):
        wl = _ring(24, 2, "fp64", periodic)
        f, I = _state(wl, "fp64")
        fg, Ig, rec, _ = _gpu(wl, f, I, md)
        fo, Io, _, Fo = _oracle(wl, f, I, md)
        assert_planes_close(fg, fo, 1e-10, "f")
        assert_fields_close(rec, Fo, 1e-10, wl.dim, "fields")
        out[periodic] = fg
    assert np.abs(out[True] - out[False]).max() > 1e-6 * np.abs(out[True]).max()


def _couette(order, precision):
    wl = gi.workloads.couette(n_side=6, n_v=12, Kn=0.1)
    return gi.workloads.with_solver(wl, precision=precision, order=order, relax_block=16, max_inner=12,
                                    tol_inner=0.0, macro_sweeps=4, cfl_macro=200.0)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("mode", ["cis", "gsis"])
def test_periodic_channel_matches_oracle(mode, order):
    """2-D: planar Couette flow in the unit square periodic in x (72 triangles, the seam
    faces joining cells at x = 1 and x = 0), FP64, one iteration against the oracle."""
    md = G.GSIS_MODE_GSIS if mode == "gsis" else G.GSIS_MODE_CIS
    wl = _couette(order, "fp64")
    M = gi.fields.uniform_fields(wl.mesh.n_cells)
    y = wl.mesh.cell_centroid[:, 1]
    x = wl.mesh.cell_centroid[:, 0]
    M[:, 1] = 0.2 * y + 0.03 * np.sin(2 * math.pi * x)
    M[:, 0] = 1.0 + 0.05 * np.cos(2 * math.pi * x) * np.sin(math.pi * y)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, wl.dim, wl.model.d_r, wl.model.d_v,
                                       wl.model.sigma_R, 9, noise=0.02)
    fg, Ig, rec, eps = _gpu(wl, f, I, md)
    fo, Io, eo, Fo = _oracle(wl, f, I, md)
    assert_planes_close(fg, fo, 1e-10, "f")
    assert_planes_close(Ig, Io, 1e-10, "I")
    assert_fields_close(rec, Fo, 1e-10, wl.dim, "fields")
    assert abs(eps - eo) <= 1e-10 * abs(eo)


def test_steady_couette_flow_has_uniform_shear_stress():
    """At the steady state of planar Couette flow the x-momentum flux through any plane
    y = const is the same (the shear stress sigma_xy is uniform) and there is no mean flow
    across the channel; GSIS in FP64 to eps < 1e-9 on the 12 x 12 channel (288 cells)."""
    wl = gi.workloads.with_solver(gi.workloads.couette(n_side=12, n_v=16, Kn=0.1), precision="fp64", order=2,
                                  relax_block=16, n_cis_precond=10, venkat_K=1.0)
    ctx = create(wl)
    try:
        G.gsis_init_fields(ctx, gi.fields.uniform_fields(wl.mesh.n_cells))
        it, hist = G.gsis_solve(ctx, G.GSIS_MODE_GSIS, 400, 1e-9)
        rec = G.gsis_get_fields(ctx, wl.mesh.n_cells)
    finally:
        G.gsis_destroy(ctx)
    assert hist[-1] < 1e-9, "eps %.2e after %d iterations" % (hist[-1], it)
    y, vol = wl.mesh.cell_centroid[:, 1], wl.mesh.cell_volume
    sxy = rec[:, 23]
    mean = np.sum(sxy * vol) / vol.sum()
    # the wall drags: sigma_xy = -mu du/dy < 0 for the lid moving along +x
    assert mean < 0.0
    # cells away from the walls, where the triangulation's face-flux errors are smallest
    core = (y > 0.2) & (y < 0.8)
    assert np.abs(sxy[core] - mean).max() < 0.05 * abs(mean)
    # no net flow across the channel: per cell u_y is of the triangulation's discretization
    # error (about 1e-4 of the wall speed on this mesh), the volume sum smaller still
    assert abs(np.sum(rec[:, 0] * rec[:, 2] * vol)) < 1e-4 * 0.2
