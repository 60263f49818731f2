"""CPU-side checks of the C ABI: the library builds, loads and exports every entry
point that include/gsis.h declares; argument validation runs before any device call."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import gsis_inputs as gi
from paper_2601_03935_gb300 import build
from paper_2601_03935_gb300 import gsis as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return G.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "gsis.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gsis_[a-z_]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = declared_functions()
    assert "gsis_create" in names and "gsis_step" in names and len(names) >= 15


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_strerror_names_codes(lib):
    assert lib.gsis_strerror(0) == b"ok"
    assert b"unsupported" in lib.gsis_strerror(G.GSIS_ERR_UNSUPPORTED)
    assert lib.gsis_strerror(12345) == b"unknown status"


def _args(wl):
    m = wl.mesh
    return (m.dim, m.face_owner, m.face_nbr, m.face_normal, m.face_area, m.face_centroid, m.cell_volume,
            m.cell_centroid, m.patches, wl.xi[:, :m.dim], wl.w, wl.omega, wl.wo, wl.model, wl.solver)


def test_validation_rejects_before_touching_the_device(lib):
    wl = gi.workloads.slab(n_cells=8)
    bad = gi.workloads.with_solver(wl, order=3)
    with pytest.raises(G.GsisError) as e:
        G.gsis_create(*_args(bad))
    assert e.value.code == G.GSIS_ERR_INVALID_ARG
    bad = gi.workloads.with_solver(wl, relax_block=65)
    with pytest.raises(G.GsisError) as e:
        G.gsis_create(*_args(bad))
    assert e.value.code == G.GSIS_ERR_INVALID_ARG
    bad = gi.workloads.with_model(wl, Kn=-1.0)
    with pytest.raises(G.GsisError) as e:
        G.gsis_create(*_args(bad))
    assert e.value.code == G.GSIS_ERR_INVALID_ARG
    args = list(_args(wl))
    args[0] = 4
    with pytest.raises(G.GsisError) as e:
        G.gsis_create(*args)
    assert e.value.code == G.GSIS_ERR_INVALID_ARG
    # 3-D meshes run the kinetic path on CUDA cores: tensor-core moments are refused
    box = gi.workloads.Workload("box", gi.mesh.box_tetrahedra(1), *gi.quadrature.trapezoid_nd(4, 4.0, 3),
                                *gi.quadrature.photon_product(2, 2), gi.workloads.ModelParams(),
                                gi.workloads.SolverParams(tc_moments=1))
    with pytest.raises(G.GsisError) as e:
        G.gsis_create(*_args(box))
    assert e.value.code == G.GSIS_ERR_UNSUPPORTED
    out = C.c_void_p()
    assert lib.gsis_create(None, None, None, None, None, None, C.byref(out)) == G.GSIS_ERR_INVALID_ARG


def test_null_context_calls_are_rejected(lib):
    assert lib.gsis_step(None, 0, None) == G.GSIS_ERR_INVALID_ARG
    assert lib.gsis_get_fields(None, None, 0) == G.GSIS_ERR_INVALID_ARG
    assert lib.gsis_launch_count(None) == 0
    lib.gsis_destroy(None)


def _mesh_args(wl, **change):
    m = wl.mesh
    a = dict(dim=m.dim, face_owner=m.face_owner.copy(), face_nbr=m.face_nbr.copy(), face_normal=m.face_normal.copy(),
             face_area=m.face_area.copy(), face_centroid=m.face_centroid.copy(), cell_volume=m.cell_volume.copy(),
             cell_centroid=m.cell_centroid.copy())
    for k, fn in change.items():
        a[k] = fn(a[k])
    return (a["dim"], a["face_owner"], a["face_nbr"], a["face_normal"], a["face_area"], a["face_centroid"],
            a["cell_volume"], a["cell_centroid"], m.patches, wl.xi[:, :m.dim], wl.w, wl.omega, wl.wo, wl.model,
            wl.solver, 0)


def _code(args):
    with pytest.raises(G.GsisError) as e:
        G.gsis_create(*args)
    return e.value.code


def _set(i, v):
    def fn(x):
        x = x.copy()
        x[i] = v
        return x
    return fn


def test_bad_meshes_and_parameters_are_refused_on_the_host(lib):
    """Malformed meshes return BAD_MESH, cells with more faces than the layout holds
    UNSUPPORTED, and out-of-range sizes and solver parameters INVALID_ARG, all before a
    kernel is launched (this runs without a GPU)."""
    wl = gi.workloads.slab(n_cells=8)
    nf = wl.mesh.n_faces
    assert _code(_mesh_args(wl, face_owner=_set(0, 8))) == G.GSIS_ERR_BAD_MESH           # owner past the last cell
    assert _code(_mesh_args(wl, face_owner=_set(0, -1))) == G.GSIS_ERR_BAD_MESH
    assert _code(_mesh_args(wl, face_nbr=_set(0, 0))) == G.GSIS_ERR_BAD_MESH             # a face from a cell to itself
    assert _code(_mesh_args(wl, face_nbr=_set(nf - 1, -1 - 7))) == G.GSIS_ERR_BAD_MESH   # a patch id with no patch
    assert _code(_mesh_args(wl, face_area=_set(0, 0.0))) == G.GSIS_ERR_BAD_MESH
    assert _code(_mesh_args(wl, face_normal=_set(0, 0.5))) == G.GSIS_ERR_BAD_MESH        # not a unit normal
    assert _code(_mesh_args(wl, cell_volume=_set(3, 0.0))) == G.GSIS_ERR_BAD_MESH
    # every face owned by cell 0 (its neighbours stay distinct): more faces than a 1-D cell holds
    many = _mesh_args(wl, face_owner=lambda x: np.zeros_like(x),
                      face_nbr=lambda x: np.where(x >= 0, np.arange(1, x.shape[0] + 1) % 8, x))
    assert _code(many) in (G.GSIS_ERR_UNSUPPORTED, G.GSIS_ERR_BAD_MESH)
    for kw in (dict(positivity=1.0), dict(positivity=-0.1), dict(sync_relax=0.0), dict(macro_fp32=3),
               dict(tc_moments=3), dict(max_inner=0), dict(venkat_K=0.0), dict(defect_correction=2)):
        assert _code(_args(gi.workloads.with_solver(wl, **kw))) == G.GSIS_ERR_INVALID_ARG, kw
    empty_v = list(_args(wl))
    empty_v[9], empty_v[10] = wl.xi[:0, :1], wl.w[:0]
    assert _code(empty_v) == G.GSIS_ERR_INVALID_ARG
    with pytest.raises(G.GsisError) as e:
        G.gsis_create(*_args(wl), 0, period=-1.0)
    assert e.value.code == G.GSIS_ERR_INVALID_ARG
    empty_o = list(_args(wl))
    empty_o[11], empty_o[12] = wl.omega[:0], wl.wo[:0]
    assert _code(empty_o) == G.GSIS_ERR_INVALID_ARG
