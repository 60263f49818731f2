"""Thin ctypes binding of the GSIS C ABI (include/gsis.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  All computation
happens in libgsis.so; if the library cannot be loaded, :func:`load` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

GSIS_OK = 0
GSIS_ERR_INVALID_ARG = -1
GSIS_ERR_OUT_OF_MEMORY = -2
GSIS_ERR_CUDA = -3
GSIS_ERR_DIVERGED = -4
GSIS_ERR_NOT_CONVERGED = -5
GSIS_ERR_TIMEOUT = -6
GSIS_ERR_BAD_MESH = -7
GSIS_ERR_UNSUPPORTED = -8
GSIS_NF = 26
GSIS_PATCH_WALL = 0
GSIS_PATCH_FARFIELD = 1
GSIS_PATCH_SYMMETRY = 2
GSIS_FP32 = 0
GSIS_FP64 = 1
GSIS_MODE_CIS = 0
GSIS_MODE_GSIS = 1

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_fp = C.POINTER(C.c_float)


class gsis_patch(C.Structure):
    _fields_ = [("kind", C.c_int32), ("rho", C.c_double), ("u", C.c_double * 3), ("T_t", C.c_double),
                ("T_r", C.c_double), ("T_v", C.c_double), ("T_R", C.c_double)]


class gsis_mesh(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_cells", C.c_int64), ("n_faces", C.c_int64),
                ("face_owner", _ip), ("face_nbr", _ip), ("face_normal", _dp), ("face_area", _dp),
                ("face_centroid", _dp), ("cell_volume", _dp), ("cell_centroid", _dp),
                ("n_patches", C.c_int32), ("patches", C.POINTER(gsis_patch)), ("period", _dp)]


class gsis_velocity_quad(C.Structure):
    _fields_ = [("n", C.c_int32), ("xi", _dp), ("w", _dp)]


class gsis_photon_quad(C.Structure):
    _fields_ = [("n", C.c_int32), ("omega", _dp), ("w", _dp)]


class gsis_model_params(C.Structure):
    _fields_ = [("d_r", C.c_double), ("d_v", C.c_double), ("Z_r", C.c_double), ("Z_v", C.c_double),
                ("omega", C.c_double), ("Sc", C.c_double), ("Kn", C.c_double), ("Kn_p", C.c_double),
                ("sigma_R", C.c_double), ("k_eff_density_scaled", C.c_int32), ("A", _dp),
                ("Tv_ref", C.c_double), ("dv_temperature_dependent", C.c_int32)]


class gsis_solver_params(C.Structure):
    _fields_ = [("precision", C.c_int32), ("order", C.c_int32), ("relax_block", C.c_int32),
                ("cfl_meso", C.c_double), ("cfl_macro", C.c_double), ("venkat_K", C.c_double),
                ("n_cis_precond", C.c_int32), ("max_outer", C.c_int32), ("max_inner", C.c_int32),
                ("macro_sweeps", C.c_int32), ("tol_outer", C.c_double), ("tol_inner", C.c_double),
                ("sync_relax", C.c_double), ("macro_fp32", C.c_int32), ("tc_moments", C.c_int32),
                ("positivity", C.c_double), ("defect_correction", C.c_int32)]


_LIB = None


def load():
    """Load libgsis.so from the package directory (build it first with build.build())."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libgsis.so")
    if not os.path.exists(path):
        raise RuntimeError("libgsis.so is missing: run paper_2601_03935_gb300.build.build() first")
    lib = C.CDLL(path)
    vp = C.c_void_p
    sig = {
        "gsis_create": (C.c_int, [C.POINTER(gsis_mesh), C.POINTER(gsis_velocity_quad), C.POINTER(gsis_photon_quad),
                                  C.POINTER(gsis_model_params), C.POINTER(gsis_solver_params), vp,
                                  C.POINTER(vp)]),
        "gsis_destroy": (None, [vp]),
        "gsis_strerror": (C.c_char_p, [C.c_int]),
        "gsis_last_error": (C.c_char_p, [vp]),
        "gsis_init_fields": (C.c_int, [vp, _dp, C.c_int64]),
        "gsis_set_distributions": (C.c_int, [vp, _dp, C.c_int64, _dp, C.c_int64]),
        "gsis_get_distributions": (C.c_int, [vp, _dp, C.c_int64, _dp, C.c_int64]),
        "gsis_upload_distributions": (C.c_int, [vp, vp, vp]),
        "gsis_refresh_fields": (C.c_int, [vp]),
        "gsis_stage_distributions": (C.c_int, [vp, vp, vp]),
        "gsis_commit_staged": (C.c_int, [vp]),
        "gsis_get_fields": (C.c_int, [vp, _dp, C.c_int64]),
        "gsis_download_fields_async": (C.c_int, [vp, _dp, C.c_int64]),
        "gsis_step": (C.c_int, [vp, C.c_int32, _dp]),
        "gsis_step_async": (C.c_int, [vp, C.c_int32]),
        "gsis_solve": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_double, _ip, _dp]),
        "gsis_macro_stats": (C.c_int, [vp, _ip, _dp, _dp]),
        "gsis_state_size": (C.c_int, [vp, C.POINTER(C.c_int64)]),
        "gsis_export_state": (C.c_int, [vp, vp, C.c_int64]),
        "gsis_import_state": (C.c_int, [vp, vp, C.c_int64]),
        "gsis_get_history": (C.c_int, [vp, C.POINTER(C.c_int64), _dp, C.c_int64, C.POINTER(C.c_int64)]),
        "gsis_set_wait_limit": (C.c_int, [vp, C.c_int32]),
        "gsis_shard_setup": (C.c_int, [vp, C.c_int32, _dp, _dp, C.c_int32, _dp, _dp]),
        "gsis_shard_buffer": (C.c_int, [vp, C.POINTER(C.c_void_p), C.POINTER(C.c_int64)]),
        "gsis_shard_refresh": (C.c_int, [vp, C.c_int32]),
        "gsis_shard_begin": (C.c_int, [vp, C.c_int32]),
        "gsis_shard_mid": (C.c_int, [vp]),
        "gsis_shard_end": (C.c_int, [vp, _dp]),
        "gsis_mlp_init": (C.c_int, [vp, C.c_uint64]),
        "gsis_mlp_set_params": (C.c_int, [vp, _fp, C.c_int64]),
        "gsis_mlp_get_params": (C.c_int, [vp, _fp, C.c_int64]),
        "gsis_mlp_samples": (C.c_int, [vp, _fp, _fp, C.c_int64]),
        "gsis_mlp_train": (C.c_int, [vp, _fp, _fp, C.c_int64, C.c_int32, C.c_int32, C.c_double, C.c_uint64, _dp]),
        "gsis_mlp_predict": (C.c_int, [vp, _fp, C.c_int64, _fp]),
        "gsis_mlp_loss_grad": (C.c_int, [vp, _fp, _fp, C.c_int64, _dp, _fp]),
        "gsis_warm_start": (C.c_int, [vp, C.c_int32, C.c_int32]),
        "gsis_last_eps": (C.c_int, [vp, _dp]),
        "gsis_profile_enable": (C.c_int, [vp, C.c_int32]),
        "gsis_profile_reset": (C.c_int, [vp]),
        "gsis_profile_read": (C.c_int, [vp, C.c_int32, C.POINTER(C.c_char_p), _dp, C.POINTER(C.c_int64),
                                        C.POINTER(C.c_int32)]),
        "gsis_launch_count": (C.c_int64, [vp]),
        "gsis_get_layout": (C.c_int, [vp, _ip, _ip, _ip, _ip]),
        "gsis_moments_static": (C.c_int, [C.c_int32, C.c_int32, C.c_int64, C.c_int32, vp, vp, C.c_int32, vp, vp,
                                          vp, vp, C.c_double, C.c_double, C.c_double, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class GsisError(RuntimeError):
    def __init__(self, code, detail=""):
        self.code = code
        super().__init__("%s (%d)%s" % (load().gsis_strerror(code).decode(), code, (": " + detail) if detail else ""))


def _check(rc, ctx=None):
    if rc != GSIS_OK:
        detail = load().gsis_last_error(ctx).decode() if ctx else ""
        raise GsisError(rc, detail)


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


class _Keep:
    """Holds the numpy arrays a C struct points into."""


def gsis_create(dim, face_owner, face_nbr, face_normal, face_area, face_centroid, cell_volume, cell_centroid,
                patches, xi, w, omega, wo, model, solver, stream=0, period=None):
    """Create a context.  ``patches`` is a list of dicts/objects with kind, rho, u, T_t, T_r, T_v, T_R;
    ``model`` and ``solver`` are objects with the fields of gsis_model_params/gsis_solver_params
    (precision as "fp32"/"fp64").  ``stream`` is a cudaStream_t as an int (0 = default).
    ``period``: None, a number (the period of x) or dim numbers (0: not periodic)."""
    lib = load()
    k = _Keep()
    k.owner = np.ascontiguousarray(face_owner, np.int32)
    k.nbr = np.ascontiguousarray(face_nbr, np.int32)
    k.normal, k.area, k.fc = _d(face_normal), _d(face_area), _d(face_centroid)
    k.vol, k.cc = _d(cell_volume), _d(cell_centroid)
    pa = (gsis_patch * max(len(patches), 1))()
    for i, p in enumerate(patches):
        g = (lambda n, d=0.0: getattr(p, n, d)) if not isinstance(p, dict) else (lambda n, d=0.0: p.get(n, d))
        pa[i].kind = int(g("kind", 0))
        pa[i].rho = float(g("rho", 1.0))
        u = list(g("u", (0.0, 0.0, 0.0)))
        for a in range(3):
            pa[i].u[a] = float(u[a]) if a < len(u) else 0.0
        pa[i].T_t, pa[i].T_r = float(g("T_t", 1.0)), float(g("T_r", 1.0))
        pa[i].T_v, pa[i].T_R = float(g("T_v", 1.0)), float(g("T_R", 1.0))
    k.pa = pa
    k.per = None
    if period is not None and np.any(np.asarray(period, np.float64) != 0.0):
        k.per = np.zeros(dim)
        p_ = np.atleast_1d(np.asarray(period, np.float64))
        k.per[:p_.shape[0]] = p_[:dim]
    mesh = gsis_mesh(dim, cell_volume.shape[0], k.owner.shape[0], _ptr(k.owner, C.c_int32), _ptr(k.nbr, C.c_int32),
                     _ptr(k.normal), _ptr(k.area), _ptr(k.fc), _ptr(k.vol), _ptr(k.cc), len(patches), pa,
                     None if k.per is None else _ptr(k.per))
    k.xi, k.w = _d(xi), _d(w)
    k.om, k.wo = _d(omega), _d(wo)
    vq = gsis_velocity_quad(k.w.shape[0], _ptr(k.xi), _ptr(k.w))
    pq = gsis_photon_quad(k.wo.shape[0], _ptr(k.om), _ptr(k.wo))
    k.A = None if getattr(model, "A", None) is None else _d(model.A).reshape(9)
    mp = gsis_model_params(model.d_r, model.d_v, model.Z_r, model.Z_v, model.omega, model.Sc, model.Kn, model.Kn_p,
                           model.sigma_R, int(bool(model.k_eff_density_scaled)),
                           None if k.A is None else _ptr(k.A), float(getattr(model, "Tv_ref", 0.0)),
                           int(bool(getattr(model, "dv_temperature_dependent", False))))
    prec = {"fp32": GSIS_FP32, "fp64": GSIS_FP64}.get(solver.precision, solver.precision)
    sp = gsis_solver_params(prec, solver.order, getattr(solver, "relax_block", 16), solver.cfl_meso,
                            solver.cfl_macro, solver.venkat_K, solver.n_cis_precond, solver.max_outer,
                            solver.max_inner, solver.macro_sweeps, solver.tol_outer, solver.tol_inner,
                            getattr(solver, "sync_relax", 1.0), int(getattr(solver, "macro_fp32", 0)),
                            int(getattr(solver, "tc_moments", 1)), float(getattr(solver, "positivity", 0.0)),
                            int(getattr(solver, "defect_correction", 0)))
    out = C.c_void_p()
    rc = lib.gsis_create(C.byref(mesh), C.byref(vq), C.byref(pq), C.byref(mp), C.byref(sp), C.c_void_p(stream),
                         C.byref(out))
    _check(rc)
    return out


def gsis_destroy(ctx):
    load().gsis_destroy(ctx)


def gsis_init_fields(ctx, M):
    M = _d(M)
    _check(load().gsis_init_fields(ctx, _ptr(M), M.size), ctx)


def gsis_set_distributions(ctx, f, I):
    f, I = _d(f), _d(I)
    _check(load().gsis_set_distributions(ctx, _ptr(f), f.size, _ptr(I), I.size), ctx)


def gsis_get_distributions(ctx, n_cells, n_xi, n_omega):
    f = np.empty((n_cells, n_xi, 4))
    I = np.empty((n_cells, n_omega))
    _check(load().gsis_get_distributions(ctx, _ptr(f), f.size, _ptr(I), I.size), ctx)
    return f, I


def gsis_upload_distributions(ctx, f_ptr, I_ptr):
    """Host pointers (ints) to buffers in the storage precision."""
    _check(load().gsis_upload_distributions(ctx, C.c_void_p(f_ptr), C.c_void_p(I_ptr)), ctx)


def gsis_stage_distributions(ctx, f_ptr, I_ptr):
    """Start the asynchronous upload of the next state (host pointers, storage precision)."""
    _check(load().gsis_stage_distributions(ctx, C.c_void_p(f_ptr), C.c_void_p(I_ptr)), ctx)


def gsis_commit_staged(ctx):
    """Make the staged state current and take its fields (asynchronous on the context stream)."""
    _check(load().gsis_commit_staged(ctx), ctx)


def gsis_refresh_fields(ctx):
    """Recompute the fields from the distributions on the device (asynchronous)."""
    _check(load().gsis_refresh_fields(ctx), ctx)


def gsis_get_fields(ctx, n_cells):
    out = np.empty((n_cells, GSIS_NF))
    _check(load().gsis_get_fields(ctx, _ptr(out), out.size), ctx)
    return out


def gsis_download_fields_async(ctx, out_ptr, n_cells):
    _check(load().gsis_download_fields_async(ctx, C.cast(C.c_void_p(out_ptr), _dp), n_cells * GSIS_NF), ctx)


def gsis_step(ctx, mode=GSIS_MODE_CIS):
    eps = C.c_double(0.0)
    _check(load().gsis_step(ctx, mode, C.byref(eps)), ctx)
    return eps.value


def gsis_solve(ctx, mode=GSIS_MODE_GSIS, max_outer=0, tol=0.0, raise_on_max=False):
    """Iterate to eps < tol; returns (iterations, eps history).  Reaching max_outer is
    reported by the history (and raises only with raise_on_max)."""
    n = max_outer if max_outer > 0 else 100000
    hist = np.zeros(n)
    it = C.c_int32(0)
    rc = load().gsis_solve(ctx, mode, max_outer, tol, C.byref(it), _ptr(hist))
    if rc != GSIS_OK and not (rc == GSIS_ERR_NOT_CONVERGED and not raise_on_max):
        _check(rc, ctx)
    return it.value, hist[:it.value].copy()


def gsis_state_size(ctx):
    n = C.c_int64(0)
    _check(load().gsis_state_size(ctx, C.byref(n)), ctx)
    return n.value


def gsis_export_state(ctx):
    """The context's iteration state as a bytes-like uint8 array."""
    buf = np.zeros(gsis_state_size(ctx), np.uint8)
    _check(load().gsis_export_state(ctx, buf.ctypes.data_as(C.c_void_p), buf.size), ctx)
    return buf


def gsis_import_state(ctx, buf):
    b = np.ascontiguousarray(np.frombuffer(bytes(buf), np.uint8) if not isinstance(buf, np.ndarray) else buf,
                             dtype=np.uint8)
    _check(load().gsis_import_state(ctx, b.ctypes.data_as(C.c_void_p), b.size), ctx)


def gsis_get_history(ctx):
    """(iterations since the distributions were set, eps history)."""
    it, n = C.c_int64(0), C.c_int64(0)
    _check(load().gsis_get_history(ctx, C.byref(it), None, 0, C.byref(n)), ctx)
    h = np.zeros(max(n.value, 1))
    _check(load().gsis_get_history(ctx, C.byref(it), _ptr(h), n.value, C.byref(n)), ctx)
    return it.value, h[:n.value].copy()


def gsis_set_wait_limit(ctx, polls):
    _check(load().gsis_set_wait_limit(ctx, polls), ctx)


def gsis_shard_setup(ctx, xi_all, w_all, omega_all, wo_all):
    xi, w = _d(xi_all), _d(w_all)
    om, wo = _d(omega_all), _d(wo_all)
    _check(load().gsis_shard_setup(ctx, w.shape[0], _ptr(xi), _ptr(w), wo.shape[0], _ptr(om), _ptr(wo)), ctx)


def gsis_shard_buffer(ctx):
    """(device pointer, number of doubles) of the context's exchange buffer."""
    p, n = C.c_void_p(0), C.c_int64(0)
    _check(load().gsis_shard_buffer(ctx, C.byref(p), C.byref(n)), ctx)
    return p.value, n.value


def gsis_shard_refresh(ctx, pass_):
    _check(load().gsis_shard_refresh(ctx, pass_), ctx)


def gsis_shard_begin(ctx, mode):
    _check(load().gsis_shard_begin(ctx, mode), ctx)


def gsis_shard_mid(ctx):
    _check(load().gsis_shard_mid(ctx), ctx)


def gsis_shard_end(ctx):
    eps = C.c_double(float("nan"))
    _check(load().gsis_shard_end(ctx, C.byref(eps)), ctx)
    return eps.value


GSIS_MLP_NPARAM = 36804
GSIS_MLP_NW = 36748


def _f(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def gsis_mlp_init(ctx, seed=0):
    _check(load().gsis_mlp_init(ctx, seed), ctx)


def gsis_mlp_set_params(ctx, params):
    p = _f(params)
    _check(load().gsis_mlp_set_params(ctx, p.ctypes.data_as(_fp), p.size), ctx)


def gsis_mlp_get_params(ctx):
    p = np.zeros(GSIS_MLP_NPARAM, np.float32)
    _check(load().gsis_mlp_get_params(ctx, p.ctypes.data_as(_fp), p.size), ctx)
    return p


def gsis_mlp_samples(ctx, n_cells, targets=True):
    X = np.zeros((n_cells, 16), np.float32)
    Y = np.zeros((n_cells, 12), np.float32) if targets else None
    _check(load().gsis_mlp_samples(ctx, X.ctypes.data_as(_fp), Y.ctypes.data_as(_fp) if targets else None,
                                   n_cells), ctx)
    return (X, Y) if targets else X


def gsis_mlp_train(ctx, X, Y, epochs=10, batch=1024, lr=1e-3, seed=0):
    X, Y = _f(X), _f(Y)
    loss = C.c_double(0.0)
    _check(load().gsis_mlp_train(ctx, X.ctypes.data_as(_fp), Y.ctypes.data_as(_fp), X.shape[0], epochs, batch, lr,
                                 seed, C.byref(loss)), ctx)
    return loss.value


def gsis_mlp_predict(ctx, X):
    X = _f(X)
    Y = np.zeros((X.shape[0], 12), np.float32)
    _check(load().gsis_mlp_predict(ctx, X.ctypes.data_as(_fp), X.shape[0], Y.ctypes.data_as(_fp)), ctx)
    return Y


def gsis_mlp_loss_grad(ctx, X, Y):
    X, Y = _f(X), _f(Y)
    loss = C.c_double(0.0)
    g = np.zeros(GSIS_MLP_NW, np.float32)
    _check(load().gsis_mlp_loss_grad(ctx, X.ctypes.data_as(_fp), Y.ctypes.data_as(_fp), X.shape[0], C.byref(loss),
                                     g.ctypes.data_as(_fp)), ctx)
    return loss.value, g


def gsis_warm_start(ctx, n_presolve=1, use_mlp=False):
    _check(load().gsis_warm_start(ctx, n_presolve, int(use_mlp)), ctx)


def gsis_macro_stats(ctx):
    """(inner iterations, first residual norm, last residual norm) of the last synthetic solve."""
    it, r0, rn = C.c_int32(0), C.c_double(0.0), C.c_double(0.0)
    _check(load().gsis_macro_stats(ctx, C.byref(it), C.byref(r0), C.byref(rn)), ctx)
    return it.value, r0.value, rn.value


def gsis_step_async(ctx, mode=GSIS_MODE_CIS):
    _check(load().gsis_step_async(ctx, mode), ctx)


def gsis_last_eps(ctx):
    eps = C.c_double(0.0)
    _check(load().gsis_last_eps(ctx, C.byref(eps)), ctx)
    return eps.value


def gsis_profile_enable(ctx, on=True):
    _check(load().gsis_profile_enable(ctx, int(on)), ctx)


def gsis_profile_reset(ctx):
    _check(load().gsis_profile_reset(ctx), ctx)


def gsis_profile_read(ctx):
    n = 64
    names = (C.c_char_p * n)()
    ms = (C.c_double * n)()
    cnt = (C.c_int64 * n)()
    nout = C.c_int32(0)
    _check(load().gsis_profile_read(ctx, n, names, ms, cnt, C.byref(nout)), ctx)
    return {names[i].decode(): (ms[i], cnt[i]) for i in range(min(n, nout.value))}


def gsis_launch_count(ctx):
    return int(load().gsis_launch_count(ctx))


def gsis_get_layout(ctx):
    v = [C.c_int32() for _ in range(4)]
    _check(load().gsis_get_layout(ctx, *[C.byref(x) for x in v]), ctx)
    return dict(v_pad=v[0].value, o_pad=v[1].value, n_chunks=v[2].value, block=v[3].value)


def gsis_moments_static(dim, precision, n_cells, n_xi, xi_ptr, w_ptr, n_omega, omega_ptr, wo_ptr, f_ptr, I_ptr,
                        d_r, d_v, sigma_R, fields_ptr, stream=0):
    """Allocation-free moments of device-resident distributions (all pointers are device
    addresses as ints); returns the status code."""
    prec = {"fp32": GSIS_FP32, "fp64": GSIS_FP64}.get(precision, precision)
    return load().gsis_moments_static(dim, prec, n_cells, n_xi, xi_ptr, w_ptr, n_omega, omega_ptr, wo_ptr, f_ptr,
                                      I_ptr, d_r, d_v, sigma_R, fields_ptr, stream)
