"""Host side of velocity-space sharding on CPU: the partition of the velocity and photon
sets, and the sum of per-shard partial moments across two gloo ranks.

Each rank sums the raw velocity moments of its range of a seeded distribution (per cell:
mass, momentum, second and third moments of F0 about a shift velocity, the internal
planes' first moments, the photon moments, and the outgoing wall flux) and the product's
allreduce_ adds them over the ranks.  The result must equal the single-process sums over
the full sets element by element, and the fields formed from it must equal the oracle's
moments of the full distribution."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import gsis_inputs as gi  # noqa: E402
from oracle import kinetic as K  # noqa: E402
from paper_2601_03935_gb300 import shard as SH  # noqa: E402


def test_split_range_partitions_contiguously_and_evenly():
    for n in (1, 2, 7, 64, 784, 2304):
        for world in range(1, 9):
            if world > n:
                with pytest.raises(ValueError):
                    SH.split_range(n, 0, world)
                continue
            parts = [SH.split_range(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
            sizes = [hi - lo for lo, hi in parts]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1


def _problem():
    wl = gi.workloads.cavity(n_side=4, n_v=20)
    M = gi.fields.smooth_random_fields(wl.mesh.cell_centroid, 9, u_scale=0.3)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 2, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 10)
    return wl, f, I


def _sums(wl, f, I, lo, hi, olo, ohi, u0):
    """Raw moments of the velocity range [lo, hi) and direction range [olo, ohi), per cell,
    about u0; and the outgoing mass flux of every boundary face over [lo, hi)."""
    xi, w = wl.xi[lo:hi, :2], wl.w[lo:hi]
    fs = f[:, lo:hi]
    c = xi[None] - u0[:, None, :]
    c2 = np.sum(c * c, axis=-1)
    f0 = fs[..., 0] * w
    cols = [f0.sum(1)] + [(f0 * c[..., a]).sum(1) for a in range(2)]
    cols += [(f0 * c[..., a] * c[..., b]).sum(1) for a in range(2) for b in range(a, 2)]
    cols += [(f0 * c[..., a] * c2).sum(1) for a in range(2)]
    for p in (1, 2, 3):
        fp = fs[..., p] * w
        cols += [fp.sum(1)] + [(fp * c[..., a]).sum(1) for a in range(2)]
    wo, om = wl.wo[olo:ohi], wl.omega[olo:ohi]
    Iw = I[:, olo:ohi] * wo
    cols += [Iw.sum(1)] + [(Iw * om[:, a]).sum(1) for a in range(2)]
    m = wl.mesh
    bnd = np.nonzero(m.face_nbr < 0)[0]
    xn = m.face_normal[bnd, :2] @ xi.T                       # [nbf, V]
    out = np.sum(np.where(xn > 0, xn * w * f[m.face_owner[bnd]][:, lo:hi, 0], 0.0), axis=1)
    return np.concatenate([np.stack(cols, 1).ravel(), out])


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl, f, I = _problem()
        u0 = np.full((wl.mesh.n_cells, 2), 0.1)
        lo, hi = SH.split_range(wl.xi.shape[0], rank, world)
        olo, ohi = SH.split_range(wl.wo.shape[0], rank, world)
        t = torch.from_numpy(_sums(wl, f, I, lo, hi, olo, ohi, u0))
        SH.allreduce_([t])
        q.put((rank, t.numpy().copy()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_to_the_unsharded_moments():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl, f, I = _problem()
    n = wl.mesh.n_cells
    u0 = np.full((n, 2), 0.1)
    full = _sums(wl, f, I, 0, wl.xi.shape[0], 0, wl.wo.shape[0], u0)
    for r in (0, 1):
        assert np.allclose(got[r], full, rtol=1e-13, atol=1e-15 * np.abs(full).max())
    # fields from the summed moments equal the oracle's moments of the full distribution
    S = got[0][:n * 20].reshape(n, 20)        # F0: 1, c (2), cc (3), c|c|^2 (2); H0, f1, f2: 1, c; I: 1, Omega
    F = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, 2, wl.model)
    rho = S[:, 0]
    u = u0 + S[:, 1:3] / rho[:, None]
    assert np.allclose(rho, F["rho"], rtol=1e-13) and np.allclose(u, F["u"][:, :2], rtol=1e-12, atol=1e-14)
    d = u - u0
    Pxx = S[:, 3] - rho * d[:, 0] ** 2
    Pyy = S[:, 5] - rho * d[:, 1] ** 2
    T_t = (Pxx + Pyy + S[:, 8]) / (3 * rho)
    assert np.allclose(T_t, F["T_t"], rtol=1e-12)
    assert np.allclose(2 * S[:, 11] / (wl.model.d_r * rho), F["T_r"], rtol=1e-12)
    assert np.allclose(2 * S[:, 14] / (wl.model.d_v * rho), F["T_v"], rtol=1e-12)
    assert np.allclose(S[:, 17], F["e_R"], rtol=1e-12)
