"""The allocation-free moment entry point (gsis_moments_static).

It serves callers that cannot allocate device memory (a host framework owning the whole
device heap through its own pool, a plugin limited to the buffers it is handed), so it
keeps its partial sums in a static device array.  Checked here:

* against the context path (gsis_set_distributions + gsis_get_fields) on two calls in a
  row with different data, in 1-D and 2-D, FP32 and FP64;
* against the FP64 oracle at hypersonic speeds (Mach 5 flow velocities), where moments
  summed about zero velocity would cancel in FP32;
* that repeated calls leave the device's free memory unchanged, and that a size beyond
  the static array is refused without touching the output.

Collected last on purpose: if it fails, a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import gsis_inputs as gi
from oracle import kinetic as K
from paper_2601_03935_gb300 import build
from paper_2601_03935_gb300 import gsis as G

from _ctx import assert_fields_close, create

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-10}


def _compare(got, ref, rtol, dim):
    rho, T = ref[:, 0], ref[:, 4]
    cols = [(0, np.abs(rho))] + [(c, np.abs(ref[:, 4:8]).max(1)) for c in (4, 5, 6, 7)]
    cols += [(1 + a, np.sqrt(T)) for a in range(dim)]
    cols += [(b + a, rho * T ** 1.5) for b in (8, 11, 14, 17) for a in range(dim)]
    cols += [(c, rho * T) for c in (20, 21, 22, 23)]
    for c, s in cols:
        err = (np.abs(got[:, c] - ref[:, c]) / s).max()
        assert err <= rtol, "column %d: %.3e > %.1e" % (c, err, rtol)
    # out-of-plane stress components are zero in a reduced velocity space
    assert np.all(got[:, 24] == 0.0) and np.all(got[:, 25] == 0.0)


class _Dev:
    """Device copies of a workload's quadratures and an output buffer."""

    def __init__(self, torch, wl, precision):
        dev = torch.device("cuda", 0)
        self.torch, self.dev, self.wl = torch, dev, wl
        self.n, self.nxi, self.no = wl.mesh.n_cells, wl.xi.shape[0], wl.omega.shape[0]
        self.xi = torch.tensor(wl.xi[:, :wl.dim], dtype=torch.float64, device=dev).contiguous()
        self.w = torch.tensor(wl.w, dtype=torch.float64, device=dev)
        self.om = torch.tensor(wl.omega, dtype=torch.float64, device=dev).contiguous()
        self.wo = torch.tensor(wl.wo, dtype=torch.float64, device=dev)
        self.out = torch.empty((self.n, G.GSIS_NF), dtype=torch.float64, device=dev)
        self.store = torch.float32 if precision == "fp32" else torch.float64
        self.precision = precision
        self.stream = torch.cuda.current_stream(dev)

    def upload(self, f, I):
        self.ft = self.torch.tensor(f, dtype=self.store, device=self.dev).contiguous()
        self.It = self.torch.tensor(I, dtype=self.store, device=self.dev).contiguous()

    def call(self, n_cells=None):
        m = self.wl.model
        return G.gsis_moments_static(self.wl.dim, self.precision, n_cells or self.n, self.nxi, self.xi.data_ptr(),
                                     self.w.data_ptr(), self.no, self.om.data_ptr(), self.wo.data_ptr(),
                                     self.ft.data_ptr(), self.It.data_ptr(), m.d_r, m.d_v, m.sigma_R,
                                     self.out.data_ptr(), self.stream.cuda_stream)


def _workload(dim, precision):
    if dim == 2:
        wl = gi.workloads.cavity(n_side=13)
    else:
        wl = gi.workloads.slab(n_cells=64)
    return gi.workloads.with_solver(wl, precision=precision, order=2, relax_block=16)


def _data(wl, seed, precision, u_scale=0.3):
    M = gi.fields.smooth_random_fields(wl.mesh.cell_centroid, seed, u_scale=u_scale)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, wl.dim, wl.model.d_r, wl.model.d_v,
                                       wl.model.sigma_R, seed + 10)
    if precision == "fp32":
        f, I = f.astype(np.float32).astype(np.float64), I.astype(np.float32).astype(np.float64)
    return f, I


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_static_moments_match_context_fields_twice(precision, dim):
    torch = pytest.importorskip("torch")
    build.build()
    wl = _workload(dim, precision)
    D = _Dev(torch, wl, precision)
    ctx = create(wl)
    try:
        for seed in (3, 4):                                   # two calls in a row, different data
            f, I = _data(wl, seed, precision)
            G.gsis_set_distributions(ctx, f, I)
            ref = G.gsis_get_fields(ctx, D.n)
            D.upload(f, I)
            D.out.fill_(np.nan)
            rc = D.call()
            D.stream.synchronize()
            assert rc == G.GSIS_OK
            _compare(D.out.cpu().numpy(), ref, TOL[precision], dim)
    finally:
        G.gsis_destroy(ctx)


@pytest.mark.parametrize("dim", [1, 2])
def test_static_moments_match_the_oracle_at_mach_5(dim):
    """Flow speeds of a Mach-5 stream (|u| ~ 4-6 thermal speeds) on the wide velocity
    grids of the hypersonic cases: FP32 storage against the FP64 oracle."""
    torch = pytest.importorskip("torch")
    build.build()
    if dim == 2:
        wl = gi.workloads.cylinder(n_theta=16, n_radial=8)            # 48 x 48 velocities
    else:
        wl = gi.workloads.normal_shock(length=16.0)                   # 64 velocities on [-15, 15]
    rng = np.random.default_rng(77)
    n = wl.mesh.n_cells
    M = np.zeros((n, G.GSIS_NF))
    M[:, 0] = rng.uniform(0.5, 2.0, n)
    M[:, 1] = rng.uniform(3.5, 5.8 if dim == 1 else 4.5, n)
    if dim == 2:
        M[:, 2] = rng.uniform(-1.0, 1.0, n)
    M[:, 4:8] = rng.uniform(0.4, 1.2, (n, 4))
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, dim, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 5)
    f, I = f.astype(np.float32).astype(np.float64), I.astype(np.float32).astype(np.float64)
    D = _Dev(torch, wl, "fp32")
    D.upload(f, I)
    assert D.call() == G.GSIS_OK
    D.stream.synchronize()
    got = D.out.cpu().numpy()
    ref = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, dim, wl.model)
    assert np.abs(K.fields_to_record(ref)[:, 8:8 + dim]).max() > 1e-3        # heat fluxes are not zero
    assert_fields_close(got, ref, TOL["fp32"], dim, "static, Mach 5")
    assert np.all(got[:, 24] == 0.0) and np.all(got[:, 25] == 0.0)


def test_static_moments_allocate_nothing_and_refuse_oversize():
    torch = pytest.importorskip("torch")
    build.build()
    wl = _workload(2, "fp32")
    D = _Dev(torch, wl, "fp32")
    D.upload(*_data(wl, 3, "fp32"))
    assert D.call() == G.GSIS_OK                              # the first call looks up the array
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(0)[0]
    for _ in range(5):
        assert D.call() == G.GSIS_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(0)[0] == free0
    # sizes beyond the static array are refused before any launch: the output keeps
    # the sentinel written before the call
    D.out.fill_(-7.0)
    torch.cuda.synchronize()
    assert D.call(n_cells=10_000_000) == G.GSIS_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert bool((D.out == -7.0).all())
