"""The allocation-free moment entry point (gsis_moments_static) against the context
path (gsis_set_distributions + gsis_get_fields), on two calls in a row.

Collected last on purpose: if it fails, a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import gsis_inputs as gi
from paper_2601_03935_gb300 import build
from paper_2601_03935_gb300 import gsis as G

from _ctx import create

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-10}


def _compare(got, ref, rtol, dim):
    rho, T = ref[:, 0], ref[:, 4]
    scale = {0: np.abs(rho), 4: np.abs(ref[:, 4:8]).max(1)}
    cols = [(0, np.abs(rho)), (4, scale[4]), (5, scale[4]), (6, scale[4]), (7, scale[4])]
    cols += [(1 + a, np.sqrt(T)) for a in range(dim)]
    cols += [(b + a, rho * T ** 1.5) for b in (8, 11, 14, 17) for a in range(dim)]
    cols += [(c, rho * T) for c in (20, 21, 22, 23)]
    for c, s in cols:
        err = (np.abs(got[:, c] - ref[:, c]) / s).max()
        assert err <= rtol, "column %d: %.3e > %.1e" % (c, err, rtol)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_static_moments_match_context_fields_twice(precision):
    torch = pytest.importorskip("torch")
    build.build()
    wl = gi.workloads.with_solver(gi.workloads.cavity(n_side=13), precision=precision, order=2, relax_block=16)
    n, nxi, no = wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0]
    dev = torch.device("cuda", 0)
    xi = torch.tensor(wl.xi, dtype=torch.float64, device=dev).contiguous()
    w = torch.tensor(wl.w, dtype=torch.float64, device=dev)
    om = torch.tensor(wl.omega, dtype=torch.float64, device=dev).contiguous()
    wo = torch.tensor(wl.wo, dtype=torch.float64, device=dev)
    out = torch.empty((n, G.GSIS_NF), dtype=torch.float64, device=dev)
    store = torch.float32 if precision == "fp32" else torch.float64
    stream = torch.cuda.current_stream(dev)
    ctx = create(wl)
    try:
        for seed in (3, 4):                                   # two calls in a row, different data
            M = gi.fields.smooth_random_fields(wl.mesh.cell_centroid, seed, u_scale=0.3)
            f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 2, wl.model.d_r, wl.model.d_v,
                                               wl.model.sigma_R, seed + 10)
            if precision == "fp32":
                f, I = f.astype(np.float32).astype(np.float64), I.astype(np.float32).astype(np.float64)
            G.gsis_set_distributions(ctx, f, I)
            ref = G.gsis_get_fields(ctx, n)
            ft = torch.tensor(f, dtype=store, device=dev).contiguous()
            It = torch.tensor(I, dtype=store, device=dev).contiguous()
            out.fill_(np.nan)
            rc = G.gsis_moments_static(2, precision, n, nxi, xi.data_ptr(), w.data_ptr(), no, om.data_ptr(),
                                       wo.data_ptr(), ft.data_ptr(), It.data_ptr(), wl.model.d_r, wl.model.d_v,
                                       wl.model.sigma_R, out.data_ptr(), stream.cuda_stream)
            stream.synchronize()
            assert rc == G.GSIS_OK
            _compare(out.cpu().numpy(), ref, TOL[precision], 2)
    finally:
        G.gsis_destroy(ctx)
    # sizes beyond the static array are refused before any launch
    rc = G.gsis_moments_static(2, precision, 10_000_000, nxi, xi.data_ptr(), w.data_ptr(), no, om.data_ptr(),
                               wo.data_ptr(), ft.data_ptr(), It.data_ptr(), 2.0, 1.16, 0.01, out.data_ptr(),
                               stream.cuda_stream)
    assert rc == G.GSIS_ERR_INVALID_ARG
