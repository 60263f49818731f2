"""Velocity-space sharding through the C ABI, emulated on one GPU.

Two (and three) shard contexts hold contiguous ranges of the velocity and photon sets of
one workload; their exchange buffers are summed on the device between the phase calls,
as an all-reduce would sum them across GPUs.  After the refresh and after every CIS and
GSIS iteration each shard must hold the fields and eps of an unsharded context, and its
distributions must equal the unsharded ones on its velocity range.  The shards run one
after another on one stream; no kernel waits on another."""
import numpy as np
import pytest

import gsis_inputs as gi
from paper_2601_03935_gb300 import build
from paper_2601_03935_gb300 import gsis as G
from paper_2601_03935_gb300 import shard as SH

from _ctx import create

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-10}


def _close(a, b, rtol, what):
    scale = np.maximum(np.abs(b).max(axis=0), 1e-30)      # per field column
    err = (np.abs(a - b) / scale).max()
    assert err <= rtol, "%s: %.3e > %.1e" % (what, err, rtol)


def _fields_close(a, b, rtol, dim, what):
    cols = [0, 4, 5, 6, 7] + [1 + k for k in range(dim)]
    _close(a[:, cols], b[:, cols], rtol, what + " rho/T/u")
    q = [8 + k for k in range(dim)] + [11 + k for k in range(dim)] + [14 + k for k in range(dim)] + \
        [17 + k for k in range(dim)] + [20, 21, 22, 23]
    scale = b[:, 0] * b[:, 4] ** 1.5
    err = (np.abs(a[:, q] - b[:, q]) / scale[:, None]).max()
    assert err <= rtol, "%s q/sigma: %.3e > %.1e" % (what, err, rtol)


CASES = {
    "cavity200": lambda: gi.workloads.cavity(n_side=10),
    "cylinder288": lambda: gi.workloads.cylinder(n_theta=24, n_radial=6, n_v=24, n_azim=12, Mach=2.0),
}


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_sharded_iterations_equal_the_unsharded_ones(case, precision, world):
    import torch
    build.build()
    wl = gi.workloads.with_solver(CASES[case](), precision=precision, order=2, relax_block=16, max_inner=30)
    n, V, O = wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0]
    if case.startswith("cylinder"):
        far = wl.mesh.patches[1]
        M = gi.fields.smooth_random_fields(wl.mesh.cell_centroid / 6.0, 3, u_scale=0.2)
        M[:, 1] += far.u[0]
        M[:, 4:8] *= far.T_t
    else:
        M = gi.fields.smooth_random_fields(wl.mesh.cell_centroid, 3, u_scale=0.2)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 2, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 4,
                                       noise=0.02)
    stream = torch.cuda.Stream()
    ref = create(wl)
    shards = []
    try:
        shards = [SH.VelocityShard(wl.mesh, wl.xi, wl.w, wl.omega, wl.wo, wl.model, wl.solver, r, world,
                                   stream.cuda_stream) for r in range(world)]
        G.gsis_set_distributions(ref, f, I)
        for s in shards:
            s.set_distributions(f, I)
        SH.refresh(shards, stream=stream)
        tol = TOL[precision]
        F_ref = G.gsis_get_fields(ref, n)
        for s in shards:
            _fields_close(G.gsis_get_fields(s.ctx, n), F_ref, tol, 2, "refresh")
        for mode in (G.GSIS_MODE_CIS, G.GSIS_MODE_CIS, G.GSIS_MODE_GSIS, G.GSIS_MODE_GSIS):
            e_ref = G.gsis_step(ref, mode)
            e = SH.step(shards, mode, stream=stream)
            assert abs(e - e_ref) <= tol * abs(e_ref) + 1e-14, (mode, e, e_ref)
            F_ref = G.gsis_get_fields(ref, n)
            for s in shards:
                _fields_close(G.gsis_get_fields(s.ctx, n), F_ref, tol, 2, "mode %d" % mode)
        fr, Ir = G.gsis_get_distributions(ref, n, V, O)
        for s in shards:
            fs, Is = G.gsis_get_distributions(s.ctx, n, s.hi - s.lo, s.ohi - s.olo)
            for p in range(4):                                 # each plane against its largest value
                ref_p = fr[:, s.lo:s.hi, p]
                err = np.abs(fs[..., p].reshape(n, -1) - ref_p).max() / np.abs(fr[..., p]).max()
                assert err <= tol * 10, "f plane %d: %.3e" % (p, err)
            err = np.abs(Is - Ir[:, s.olo:s.ohi]).max() / np.abs(Ir).max()
            assert err <= tol * 10, "I: %.3e" % err
        # a shard refuses the unsharded iteration
        with pytest.raises(G.GsisError) as err:
            G.gsis_step(shards[0].ctx, G.GSIS_MODE_CIS)
        assert err.value.code == G.GSIS_ERR_UNSUPPORTED
    finally:
        G.gsis_destroy(ref)
        for s in shards:
            s.destroy()
