"""GPU parity of the conventional iteration on 3-D tetrahedral meshes (the sweeps of Eq.
dis_micro for f0, f1, f2 and I over the full 3-D velocity space, the moments of Eq.
getmoment, the fields and eps) against the FP64 oracle on the same seeded inputs.

Tolerances as in the 2-D parity tests: FP64 1e-10, FP32 1e-5 relative (per plane of f
against its largest value; fields against their magnitude).  The full-size capsule (about
193 000 tetrahedra x 13 824 velocities x 128 directions) is checked on the fields of
sampled relaxation blocks, recomputed by the oracle from the same equilibrium state.
"""
import numpy as np
import pytest

import gsis_inputs as gi
from gsis_inputs import quadrature as Q
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


def box162():
    """3 x 3 x 3 hexahedra cut into 162 tetrahedra (ten blocks of 16 and a ragged block of
    2), walls at three temperatures, one moving obliquely; 9^3 velocities (eleven full
    chunks of 64 and a ragged one), 32 photon directions (one ragged chunk)."""
    lid = gi.mesh.Patch(gi.mesh.WALL, u=(0.3, -0.2, 0.25), T_t=1.6)
    pats = [gi.mesh.Patch(gi.mesh.WALL, T_t=1.0), gi.mesh.Patch(gi.mesh.WALL, T_t=1.3)] + \
        [gi.mesh.Patch(gi.mesh.WALL, T_t=1.0) for _ in range(3)] + [lid]
    m = gi.mesh.box_tetrahedra(3, seed=7, patches=pats)
    xi, w = Q.trapezoid_nd(9, 6.5, 3)
    om, wo = Q.photon_product(4, 8)
    return gi.workloads.Workload("box162", m, xi, w, om, wo, gi.workloads.ModelParams(Kn=0.2, Kn_p=2.0),
                                 gi.workloads.SolverParams(tc_moments=0))


CASES = {
    "box162": box162,
    # 1270 tetrahedra around the capsule (79 blocks of 16 and a ragged one of 6), Mach 3
    # free stream, 8^3 velocities, 32 directions
    "capsule1270": lambda: gi.workloads.capsule(n=6, n_v=8, n_polar=4, n_azim=8, Mach=3.0, Kn=0.1, Kn_p=10.0),
}


def _inputs(wl, seed, precision, u_scale=0.3):
    M = gi.fields.random_macro_fields(wl.mesh.n_cells, 3, seed, u_scale=u_scale, q_scale=0.05)
    if wl.mesh.patches[-1].kind == gi.mesh.FARFIELD:
        M[:, 1] += 0.5 * wl.mesh.patches[-1].u[0]
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 3, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, seed + 1)
    if precision == "fp32":
        f, I = f.astype(np.float32).astype(np.float64), I.astype(np.float32).astype(np.float64)
    return f, I


def _run(wl, f, I, steps=1):
    ctx = create(wl)
    try:
        G.gsis_set_distributions(ctx, f, I)
        rec0 = G.gsis_get_fields(ctx, wl.mesh.n_cells)
        eps = [G.gsis_step(ctx, G.GSIS_MODE_CIS) for _ in range(steps)]
        fg, Ig = G.gsis_get_distributions(ctx, wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0])
        rec1 = G.gsis_get_fields(ctx, wl.mesh.n_cells)
        return rec0, rec1, fg, Ig, eps
    finally:
        G.gsis_destroy(ctx)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_cis_step_matches_oracle_3d(case, precision, order):
    wl = gi.workloads.with_solver(CASES[case](), precision=precision, order=order, relax_block=16)
    f, I = _inputs(wl, 51, precision)
    rec0, rec1, fg, Ig, eps = _run(wl, f, I)
    tol = TOL[precision]
    F0 = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, 3, wl.model)
    fo, Io = K.kinetic_sweep(f, I, wl, relax_block=16, F=F0)
    F1 = K.moments(fo, Io, wl.xi, wl.w, wl.omega, wl.wo, 3, wl.model)
    assert_fields_close(rec0, F0, tol, 3, "moments of f^k")
    assert np.abs(fg[..., 1]).max() == 0.0                      # no hidden components in 3-D
    assert_planes_close(fg, fo, tol, "f^{k+1}")
    assert_planes_close(Ig, Io, tol, "I^{k+1}")
    assert_fields_close(rec1, F1, tol, 3, "moments of f^{k+1}")
    eps_o = OG.epsilon(F1, F0, wl.mesh.cell_volume, wl.model, 3)
    assert abs(eps[0] - eps_o) <= (1e-4 if precision == "fp32" else 1e-9) * eps_o


@pytest.mark.parametrize("block", [1, 5, 64])
def test_3d_block_sizes_and_jacobi(block):
    wl = gi.workloads.with_solver(box162(), precision="fp64", order=2, relax_block=block)
    f, I = _inputs(wl, 52, "fp64")
    _, _, fg, Ig, _ = _run(wl, f, I)
    fo, Io = K.kinetic_sweep(f, I, wl, relax_block=block)
    assert_planes_close(fg, fo, 1e-10, "f block=%d" % block)
    assert_planes_close(Ig, Io, 1e-10, "I block=%d" % block)


@pytest.mark.parametrize("case,order", [("capsule1270", 1), ("box162", 2)])
def test_3d_iterations_follow_the_oracle(case, order):
    """Eight CIS iterations in FP64 (fields, coefficients, wall densities and sweeps
    accumulate): the capsule impulsively started in its Mach-3 free stream at order 1 (at
    order 2 the start from the free stream turns f negative at the body, in the oracle as
    on the GPU), and the closed box from rest with its oblique moving wall at order 2.
    Every eps and the final distributions equal the oracle's."""
    wl = gi.workloads.with_solver(CASES[case](), precision="fp64", order=order, relax_block=16)
    far = wl.mesh.patches[-1]
    if far.kind == gi.mesh.FARFIELD:
        M = gi.fields.uniform_fields(wl.mesh.n_cells, rho=far.rho, u=far.u, T=far.T_t)
    else:
        M = gi.fields.uniform_fields(wl.mesh.n_cells)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 3, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 0,
                                       noise=0.0)
    _, _, fg, Ig, eps_g = _run(wl, f, I, steps=8)
    geo = K.Geometry(wl.mesh)
    eps_o = []
    for _ in range(8):
        f, I, e, _ = OG.cis_step(f, I, wl, geo)
        eps_o.append(e)
    assert np.allclose(eps_g, eps_o, rtol=1e-9, atol=0.0)
    assert_planes_close(fg, f, 1e-9, "f after 8 iterations")
    assert_planes_close(Ig, I, 1e-9, "I after 8 iterations")


def _gsis_inputs(wl, seed, precision):
    M = gi.fields.smooth_random_fields(wl.mesh.cell_centroid, seed, u_scale=0.2)
    if wl.mesh.patches[-1].kind == gi.mesh.FARFIELD:
        M[:, 1] += 0.5 * wl.mesh.patches[-1].u[0]
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 3, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, seed + 1,
                                       noise=0.02)
    if precision == "fp32":
        f, I = f.astype(np.float32).astype(np.float64), I.astype(np.float32).astype(np.float64)
    return f, I


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("case", sorted(CASES))
def test_gsis_step_matches_oracle_3d(case, order, precision):
    """One GSIS iteration (kinetic step, high-order terms, 3-D synthetic equations with a
    fixed number of inner iterations, synchronisation) on tetrahedra: the closed box (walls
    only, mass rescaling) and the capsule (wall and far field)."""
    from oracle import macro as MA
    wl = gi.workloads.with_solver(CASES[case](), precision=precision, order=order, relax_block=16, max_inner=12,
                                  tol_inner=0.0, macro_sweeps=4, cfl_macro=200.0)
    f, I = _gsis_inputs(wl, 71, precision)
    ctx = create(wl)
    try:
        G.gsis_set_distributions(ctx, f, I)
        eps = G.gsis_step(ctx, G.GSIS_MODE_GSIS)
        fg, Ig = G.gsis_get_distributions(ctx, wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0])
        rec = G.gsis_get_fields(ctx, wl.mesh.n_cells)
    finally:
        G.gsis_destroy(ctx)
    geo = K.Geometry(wl.mesh)
    fo, Io, e_o, Fo = OG.gsis_step(f, I, wl, geo, MA.Faces(geo))
    tol = TOL[precision]
    assert_planes_close(fg, fo, tol, "f^{k+1}")
    assert_planes_close(Ig, Io, tol, "I^{k+1}")
    assert_fields_close(rec, Fo, tol, 3, "moments of f^{k+1}")
    assert abs(eps - e_o) <= (1e-4 if precision == "fp32" else 1e-9) * e_o


def test_gsis_3d_iterations_follow_the_oracle():
    """Four GSIS iterations on the closed box in FP64 (order 1): every eps and the final
    distributions equal the oracle's."""
    from oracle import macro as MA
    wl = gi.workloads.with_solver(box162(), precision="fp64", order=1, relax_block=16, max_inner=12, tol_inner=0.0,
                                  macro_sweeps=4, cfl_macro=200.0)
    f, I = _gsis_inputs(wl, 72, "fp64")
    ctx = create(wl)
    try:
        G.gsis_set_distributions(ctx, f, I)
        eps_g = [G.gsis_step(ctx, G.GSIS_MODE_GSIS) for _ in range(4)]
        fg, Ig = G.gsis_get_distributions(ctx, wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0])
    finally:
        G.gsis_destroy(ctx)
    geo = K.Geometry(wl.mesh)
    faces = MA.Faces(geo)
    eps_o, F = [], None
    for _ in range(4):
        f, I, e, F = OG.gsis_step(f, I, wl, geo, faces, F)
        eps_o.append(e)
    assert np.allclose(eps_g, eps_o, rtol=1e-9, atol=0.0)
    assert_planes_close(fg, f, 1e-9, "f after 4 GSIS iterations")
    assert_planes_close(Ig, I, 1e-9, "I after 4 GSIS iterations")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_positivity_bound_matches_oracle(precision):
    """Order 2 from the impulsive Mach-3 free stream around the capsule, with the positivity
    bound theta = 0.1 on the implicit update: one iteration, where the bound is active on
    about a sixth of the values, equals the oracle's; five more follow its eps."""
    wl = gi.workloads.with_solver(CASES["capsule1270"](), precision=precision, order=2, relax_block=16,
                                  venkat_K=0.01, positivity=0.1)
    far = wl.mesh.patches[1]
    M = gi.fields.uniform_fields(wl.mesh.n_cells, rho=far.rho, u=far.u, T=far.T_t)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 3, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 0,
                                       noise=0.0)
    if precision == "fp32":
        f, I = f.astype(np.float32).astype(np.float64), I.astype(np.float32).astype(np.float64)
    _, rec1, fg, Ig, eps_g = _run(wl, f, I, steps=1)
    F0 = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, 3, wl.model)
    fo, Io = K.kinetic_sweep(f, I, wl, relax_block=16, F=F0)
    fu, _ = K.kinetic_sweep(f, I, gi.workloads.with_solver(wl, positivity=0.0), relax_block=16, F=F0)
    assert np.mean(fo != fu) > 0.05                                # the bound is active
    assert np.all(fg >= 0.1 * f * (1 - 1e-6) - 1e-40)              # (FP32 subnormals round coarsely)
    tol = TOL[precision]
    assert_planes_close(fg, fo, tol, "f^{k+1}")
    assert_planes_close(Ig, Io, tol, "I^{k+1}")
    assert_fields_close(rec1, K.moments(fo, Io, wl.xi, wl.w, wl.omega, wl.wo, 3, wl.model), tol, 3, "fields")
    if precision == "fp64":
        _, _, fg6, _, eps6 = _run(wl, f, I, steps=6)
        geo = K.Geometry(wl.mesh)
        eps_o = []
        for _ in range(6):
            f, I, e, _ = OG.cis_step(f, I, wl, geo)
            eps_o.append(e)
        assert np.allclose(eps6, eps_o, rtol=1e-9, atol=0.0)
        assert_planes_close(fg6, f, 1e-9, "f after 6 iterations")


def test_3d_refuses_what_is_built_for_1d_and_2d():
    wl = gi.workloads.with_solver(box162(), precision="fp32", order=2)
    with pytest.raises(G.GsisError) as e:
        create(gi.workloads.with_solver(wl, tc_moments=1))
    assert e.value.code == G.GSIS_ERR_UNSUPPORTED
    ctx = create(wl)
    try:
        for call in (lambda: G.gsis_mlp_samples(ctx, wl.mesh.n_cells),
                     lambda: G.gsis_warm_start(ctx, 1, True),
                     lambda: G.gsis_shard_setup(ctx, wl.xi, wl.w, wl.omega, wl.wo)):
            with pytest.raises(G.GsisError) as e:
                call()
            assert e.value.code == G.GSIS_ERR_UNSUPPORTED
        assert np.isfinite(G.gsis_step(ctx, G.GSIS_MODE_CIS))       # the context stays usable
        assert np.isfinite(G.gsis_step(ctx, G.GSIS_MODE_GSIS))
    finally:
        G.gsis_destroy(ctx)


class _EquilibriumOf:
    """The FP64 multi-temperature equilibrium of per-cell fields, evaluated for the cells
    an oracle call touches (a full-size f would not fit in host memory)."""

    def __init__(self, M, wl):
        self.F = K.fields_from_record(M, wl.model.sigma_R)
        self.wl = wl
        self.cache = {}

    def _cell(self, i):
        i = int(i)
        if i not in self.cache:
            Fi = {k: v[i:i + 1] for k, v in self.F.items()}
            self.cache[i] = K.equilibrium_planes(Fi, self.wl.xi, 3, self.wl.model)[0]
        return self.cache[i]

    def __getitem__(self, idx):
        if isinstance(idx, tuple):
            return self._cell(idx[0])[idx[1:]]
        if np.ndim(idx) == 0:
            return self._cell(idx)
        return np.stack([self._cell(i) for i in idx])


def test_full_size_capsule_sampled_blocks():
    """The 3-D capsule at full size in the benchmark's configuration (FP32, order 2, blocks
    of 16): from a smooth hot state set through gsis_init_fields (equilibrium built on the
    device), one CIS iteration; the fields of whole blocks at the start, on the body, at the
    far field, in the middle and at the end equal the oracle's sweep of the same
    equilibrium."""
    wl = gi.workloads.with_solver(gi.workloads.capsule(), precision="fp32", order=2, relax_block=16)
    m = wl.mesh
    nc = m.n_cells
    assert nc > 190000 and wl.xi.shape[0] == 13824 and wl.omega.shape[0] == 128
    far = m.patches[1]
    M = gi.fields.smooth_random_fields(m.cell_centroid, 53, u_scale=0.3)
    M[:, 1] = (0.5 + M[:, 1]) * far.u[0]
    M[:, 4:8] *= 3.0                                            # post-shock temperatures
    M[:, 8:] = 0.0
    ctx = create(wl)
    try:
        G.gsis_init_fields(ctx, M)
        G.gsis_step(ctx, G.GSIS_MODE_CIS)
        rec1 = G.gsis_get_fields(ctx, nc)
    finally:
        G.gsis_destroy(ctx)
    wall = m.face_owner[m.face_nbr == -1]
    farc = m.face_owner[m.face_nbr == -2]
    blocks = sorted({0, int(wall[len(wall) // 2]) // 16, int(farc[len(farc) // 3]) // 16, nc // 32, (nc - 1) // 16})
    cells = np.concatenate([np.arange(b * 16, min(b * 16 + 16, nc)) for b in blocks])
    f = _EquilibriumOf(M, wl)
    I = K.photon_equilibrium(M[:, 7], wl.omega.shape[0], wl.model.sigma_R)
    F0 = K.moments(f[cells], I[cells], wl.xi, wl.w, wl.omega, wl.wo, 3, wl.model)
    fo, Io = K.kinetic_sweep(f, I, wl, relax_block=16, cells=cells, F=F0)
    F1 = K.moments(fo, Io, wl.xi, wl.w, wl.omega, wl.wo, 3, wl.model)
    assert_fields_close(rec1[cells], F1, 1e-5, 3, "capsule sampled blocks")
