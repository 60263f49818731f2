"""Test helpers: create library contexts from seeded workloads and compare with the oracle."""
import numpy as np

from paper_2601_03935_gb300 import gsis as G


def create(wl, stream=0):
    m = wl.mesh
    return G.gsis_create(m.dim, m.face_owner, m.face_nbr, m.face_normal, m.face_area, m.face_centroid,
                         m.cell_volume, m.cell_centroid, m.patches, wl.xi[:, :m.dim], wl.w, wl.omega, wl.wo,
                         wl.model, wl.solver, stream, period=getattr(m, "period", 0.0))


def assert_planes_close(got, ref, rtol, what=""):
    """Elementwise comparison of [n, V, P] (or [n, V]) arrays, each plane against its own scale."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    if ref.ndim == 2:
        got, ref = got[..., None], ref[..., None]
    for p in range(ref.shape[-1]):
        scale = np.abs(ref[..., p]).max()
        err = np.abs(got[..., p] - ref[..., p]).max()
        assert err <= rtol * scale, "%s plane %d: max err %.3e > %.1e * %.3e" % (what, p, err, rtol, scale)


def assert_fields_close(rec_got, F_ref, rtol, dim, what=""):
    """Library field records vs oracle field dicts: rho, u, temperatures relative to
    their magnitude; heat fluxes and stresses absolute against rho T^1.5."""
    from oracle import kinetic as K
    ref = K.fields_to_record(F_ref)
    g = np.asarray(rec_got)
    rho, T = ref[:, 0], ref[:, 4]
    s = rho * T ** 1.5
    checks = [("rho", [0], np.abs(ref[:, 0])), ("T", [4, 5, 6, 7], np.abs(ref[:, 4:8]).max(axis=1))]
    checks.append(("u", list(range(1, 1 + dim)), np.sqrt(T)))
    qs = [8 + a for a in range(dim)] + [11 + a for a in range(dim)] + [14 + a for a in range(dim)] \
        + [17 + a for a in range(dim)]
    checks.append(("q", qs, s))
    checks.append(("sigma", [20, 21, 22, 23] + ([24, 25] if dim == 3 else []), rho * T))
    for name, cols, scale in checks:
        for c in cols:
            err = np.abs(g[:, c] - ref[:, c]) / np.maximum(scale, 1e-300)
            assert err.max() <= rtol, "%s %s[col %d]: max rel err %.3e > %.1e" % (what, name, c, err.max(), rtol)
