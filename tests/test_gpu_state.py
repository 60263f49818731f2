"""Checkpoint/resume and failure detection through the C ABI.

* gsis_export_state / gsis_import_state: a run exported after some outer iterations and
  resumed in a fresh context reproduces the uninterrupted run's eps trajectory, fields
  and distributions bit for bit (FP32 and FP64, CIS start then GSIS); images of another
  problem or short buffers are refused.
* gsis_set_wait_limit: a zero poll budget makes the tensor-core completion waits run out
  at once; the sweep's fused epilogue, the synchronisation pass and the standalone moment
  pass then report GSIS_ERR_TIMEOUT (not DIVERGED), and the context keeps working once
  the budget is restored.  No GPU fault is involved: the wait returns, the kernel skips
  the accumulator read and waits for the chain before freeing tensor memory.
"""
import numpy as np
import pytest

import gsis_inputs as gi
from paper_2601_03935_gb300 import build
from paper_2601_03935_gb300 import gsis as G

from _ctx import create

pytestmark = pytest.mark.gpu


def _wl(precision, n_side=8, **kw):
    wl = gi.workloads.cavity(n_side=n_side, Kn=0.05, Kn_p=10.0)
    args = dict(precision=precision, order=2, relax_block=16, max_inner=40, n_cis_precond=2)
    args.update(kw)
    return gi.workloads.with_solver(wl, **args)


def _start(ctx, wl, seed=1):
    M = gi.fields.smooth_random_fields(wl.mesh.cell_centroid, seed, u_scale=0.1)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 2, wl.model.d_r, wl.model.d_v, wl.model.sigma_R,
                                       seed + 3, noise=0.01)
    G.gsis_set_distributions(ctx, f, I)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_resumed_run_reproduces_the_uninterrupted_one_bit_for_bit(precision):
    build.build()
    wl = _wl(precision)
    n, V, O = wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0]
    a = create(wl)
    b = create(wl)
    try:
        _start(a, wl)
        it1, h1 = G.gsis_solve(a, G.GSIS_MODE_GSIS, 4, 1e-30)
        assert it1 == 4
        image = G.gsis_export_state(a)
        it2, h2 = G.gsis_solve(a, G.GSIS_MODE_GSIS, 4, 1e-30)
        Fa = G.gsis_get_fields(a, n)
        fa, Ia = G.gsis_get_distributions(a, n, V, O)
        _start(b, wl, seed=7)                     # a different state, overwritten by the import
        G.gsis_step(b, G.GSIS_MODE_CIS)
        G.gsis_import_state(b, image)
        itb, hb = G.gsis_get_history(b)
        assert itb == 4 and np.array_equal(hb, h1)
        it3, h3 = G.gsis_solve(b, G.GSIS_MODE_GSIS, 4, 1e-30)
        assert it3 == it2 == 4
        assert np.array_equal(h3, h2)                          # eps trajectory, bit for bit
        assert np.array_equal(G.gsis_get_fields(b, n), Fa)
        fb, Ib = G.gsis_get_distributions(b, n, V, O)
        assert np.array_equal(fb, fa) and np.array_equal(Ib, Ia)
        ita, ha = G.gsis_get_history(a)
        assert ita == 8 and np.array_equal(ha, np.concatenate([h1, h2]))
        # refused: a short buffer, a corrupted magic, another problem size
        with pytest.raises(G.GsisError) as e:
            G.gsis_import_state(b, image[:-1])
        assert e.value.code == G.GSIS_ERR_INVALID_ARG
        bad = image.copy()
        bad[0] ^= 0xFF
        with pytest.raises(G.GsisError) as e:
            G.gsis_import_state(b, bad)
        assert e.value.code == G.GSIS_ERR_INVALID_ARG
    finally:
        G.gsis_destroy(a)
        G.gsis_destroy(b)
    other = create(_wl(precision, n_side=6))
    try:
        with pytest.raises(G.GsisError) as e:
            G.gsis_import_state(other, image)
        assert e.value.code == G.GSIS_ERR_INVALID_ARG
    finally:
        G.gsis_destroy(other)


@pytest.mark.parametrize("where", ["sweep_epilogue", "sync_pass", "moment_pass"])
def test_expired_tensor_core_wait_reports_timeout_and_the_context_recovers(where):
    build.build()
    wl = _wl("fp32", tc_moments=2 if where == "sweep_epilogue" else 1, n_cis_precond=0)
    ctx = create(wl)
    ref = create(wl)
    try:
        _start(ctx, wl)
        _start(ref, wl)
        G.gsis_set_wait_limit(ctx, 0)
        with pytest.raises(G.GsisError) as e:
            if where == "sweep_epilogue":
                G.gsis_step(ctx, G.GSIS_MODE_CIS)
            elif where == "sync_pass":
                G.gsis_step(ctx, G.GSIS_MODE_GSIS)
            else:
                G.gsis_refresh_fields(ctx)
        assert e.value.code == G.GSIS_ERR_TIMEOUT
        with pytest.raises(G.GsisError):
            G.gsis_set_wait_limit(ctx, -1)
        # budget restored: the same start gives the same first iteration as a context
        # that never timed out
        G.gsis_set_wait_limit(ctx, 1 << 22)
        _start(ctx, wl)
        mode = G.GSIS_MODE_GSIS if where == "sync_pass" else G.GSIS_MODE_CIS
        e1 = G.gsis_step(ctx, mode)
        e2 = G.gsis_step(ref, mode)
        assert np.isfinite(e1) and e1 == e2
        n = wl.mesh.n_cells
        assert np.array_equal(G.gsis_get_fields(ctx, n), G.gsis_get_fields(ref, n))
    finally:
        G.gsis_destroy(ctx)
        G.gsis_destroy(ref)
