"""Double-buffered uploads (gsis_stage_distributions / gsis_commit_staged): staging the next
state while a step runs gives exactly the results of plain uploads, and misuse is rejected."""
import numpy as np
import pytest
import torch

import gsis_inputs as gi
from paper_2601_03935_gb300 import build
from paper_2601_03935_gb300 import gsis as G

from _ctx import create

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    G.load()


def _states(wl, n):
    out = []
    for s in range(n):
        M = gi.fields.smooth_random_fields(wl.mesh.cell_centroid, 30 + s, u_scale=0.2)
        f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, wl.dim, wl.model.d_r, wl.model.d_v,
                                           wl.model.sigma_R, 40 + s, noise=0.02)
        out.append((torch.from_numpy(f.astype(np.float32)).pin_memory(),
                    torch.from_numpy(I.astype(np.float32)).pin_memory()))
    return out


def test_staged_pipeline_matches_plain_uploads():
    wl = gi.workloads.with_solver(gi.workloads.cavity(n_side=13), precision="fp32", order=2, relax_block=16)
    nc, V, NO = wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0]
    states = _states(wl, 3)
    stream = torch.cuda.Stream()

    def run(staged):
        ctx = create(wl, stream.cuda_stream)
        res = []
        try:
            if staged:
                G.gsis_stage_distributions(ctx, states[0][0].data_ptr(), states[0][1].data_ptr())
            for k in range(len(states)):
                if staged:
                    G.gsis_commit_staged(ctx)
                    if k + 1 < len(states):      # the next state uploads while this step computes
                        G.gsis_stage_distributions(ctx, states[k + 1][0].data_ptr(), states[k + 1][1].data_ptr())
                else:
                    G.gsis_upload_distributions(ctx, states[k][0].data_ptr(), states[k][1].data_ptr())
                F0 = G.gsis_get_fields(ctx, nc)
                eps = G.gsis_step(ctx, G.GSIS_MODE_CIS)
                f, I = G.gsis_get_distributions(ctx, nc, V, NO)
                res.append((F0, eps, f, I))
        finally:
            G.gsis_destroy(ctx)
        return res

    plain, piped = run(False), run(True)
    for (F0a, ea, fa, Ia), (F0b, eb, fb, Ib) in zip(plain, piped):
        assert np.array_equal(F0a, F0b)
        assert ea == eb
        assert np.array_equal(fa, fb) and np.array_equal(Ia, Ib)


def test_staging_misuse_is_rejected():
    wl = gi.workloads.with_solver(gi.workloads.cavity(n_side=4), precision="fp32", order=1, relax_block=16)
    f, I = _states(wl, 1)[0]
    ctx = create(wl)
    try:
        with pytest.raises(G.GsisError):
            G.gsis_commit_staged(ctx)                                # nothing staged
        G.gsis_stage_distributions(ctx, f.data_ptr(), I.data_ptr())
        with pytest.raises(G.GsisError):
            G.gsis_stage_distributions(ctx, f.data_ptr(), I.data_ptr())   # a second stage before the commit
        G.gsis_commit_staged(ctx)
        assert np.isfinite(G.gsis_step(ctx, G.GSIS_MODE_CIS))
    finally:
        G.gsis_destroy(ctx)


@pytest.mark.parametrize("stream_kind", ["user", "legacy_default"])
def test_side_stream_photon_transport_gives_identical_results(stream_kind):
    """The photon slope pass and sweep run on a stream of the context's own, beside the gas
    kernels.  Asynchronous steps with and without per-kernel profiling, on a user stream or
    the legacy default stream, and synchronous steps give bit-identical distributions,
    fields and eps."""
    wl = gi.workloads.with_solver(gi.workloads.cavity(n_side=40), precision="fp32", order=2, relax_block=16)
    nc, V, NO = wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0]
    M = gi.fields.smooth_random_fields(wl.mesh.cell_centroid, 7, u_scale=0.2)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, wl.dim, wl.model.d_r, wl.model.d_v,
                                       wl.model.sigma_R, 8, noise=0.02)
    user = torch.cuda.Stream()

    def run(prof, sync, stream):
        ctx = create(wl, stream)
        try:
            G.gsis_set_distributions(ctx, f, I)
            G.gsis_profile_enable(ctx, prof)
            for _ in range(4):
                if sync:
                    eps = G.gsis_step(ctx, G.GSIS_MODE_CIS)
                else:
                    G.gsis_step_async(ctx, G.GSIS_MODE_CIS)
            if not sync:
                eps = G.gsis_last_eps(ctx)
            fo, Io = G.gsis_get_distributions(ctx, nc, V, NO)
            F = G.gsis_get_fields(ctx, nc)
        finally:
            G.gsis_destroy(ctx)
        return eps, fo, Io, F

    s = user.cuda_stream if stream_kind == "user" else 0
    ref = run(False, True, user.cuda_stream)
    for prof in (False, True):
        got = run(prof, False, s)
        assert got[0] == ref[0]
        for a, b in zip(got[1:], ref[1:]):
            assert np.array_equal(a, b)


def test_distributions_replaced_between_steps_give_the_results_of_a_fresh_context():
    """A call that replaces the distributions between two steps (upload, set, state
    import) leaves the second step bit-identical to the same step of a fresh context: no
    state of the first step (face values, coefficients, side-stream work) leaks into it."""
    wl = gi.workloads.with_solver(gi.workloads.cavity(n_side=13), precision="fp32", order=2, relax_block=16)
    nc, V, NO = wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0]
    (f1, I1), (f2, I2) = _states(wl, 2)
    stream = torch.cuda.Stream()

    def second_step(replace):
        ctx = create(wl, stream.cuda_stream)
        try:
            G.gsis_upload_distributions(ctx, f1.data_ptr(), I1.data_ptr())
            G.gsis_step(ctx, G.GSIS_MODE_CIS)
            replace(ctx)
            eps = G.gsis_step(ctx, G.GSIS_MODE_CIS)
            return eps, G.gsis_get_distributions(ctx, nc, V, NO)
        finally:
            G.gsis_destroy(ctx)

    ref_ctx = create(wl, stream.cuda_stream)
    try:
        G.gsis_upload_distributions(ref_ctx, f2.data_ptr(), I2.data_ptr())
        state = G.gsis_export_state(ref_ctx)
        eps_ref = G.gsis_step(ref_ctx, G.GSIS_MODE_CIS)
        ref = G.gsis_get_distributions(ref_ctx, nc, V, NO)
    finally:
        G.gsis_destroy(ref_ctx)
    f2d, I2d = f2.numpy().astype(np.float64), I2.numpy().astype(np.float64)
    for name, replace in (("upload", lambda c: G.gsis_upload_distributions(c, f2.data_ptr(), I2.data_ptr())),
                          ("set", lambda c: G.gsis_set_distributions(c, f2d, I2d)),
                          ("import", lambda c: G.gsis_import_state(c, state))):
        eps, got = second_step(replace)
        assert eps == eps_ref, name
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), name
