"""Seeded mesh generators (inputs only).

A mesh is described the way a finite-volume code consumes it (Section 5): a
list of faces, each with an owner cell, a neighbour cell (or a boundary patch),
a unit normal pointing from owner to neighbour (outward at the boundary), an
area and a centroid, plus cell volumes and centroids.  ``face_nbr < 0`` marks a
boundary face of patch ``-1 - face_nbr``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

WALL = 0        # diffuse wall for the gas, black wall for photons
FARFIELD = 1    # incoming characteristics carry a prescribed equilibrium state
SYMMETRY = 2    # specular reflection of molecules and photons (a mirror plane)


@dataclass
class Patch:
    kind: int
    rho: float = 1.0
    u: tuple = (0.0, 0.0, 0.0)
    T_t: float = 1.0
    T_r: float = 1.0
    T_v: float = 1.0
    T_R: float = 1.0


@dataclass
class Mesh:
    dim: int
    n_cells: int
    face_owner: np.ndarray
    face_nbr: np.ndarray
    face_normal: np.ndarray
    face_area: np.ndarray
    face_centroid: np.ndarray
    cell_volume: np.ndarray
    cell_centroid: np.ndarray
    patches: list = field(default_factory=list)

    @property
    def n_faces(self) -> int:
        return int(self.face_owner.shape[0])


def slab_1d(n_cells: int, length: float = 1.0, patches=None) -> Mesh:
    """Uniform 1-D slab on [0, L]; patch 0 is the left wall, patch 1 the right wall."""
    x = np.linspace(0.0, length, n_cells + 1)
    dx = np.diff(x)
    owner = list(range(n_cells - 1)) + [0, n_cells - 1]
    nbr = list(range(1, n_cells)) + [-1, -2]
    normal = [1.0] * (n_cells - 1) + [-1.0, 1.0]
    fc = list(x[1:-1]) + [x[0], x[-1]]
    return Mesh(
        dim=1, n_cells=n_cells,
        face_owner=np.asarray(owner, np.int32), face_nbr=np.asarray(nbr, np.int32),
        face_normal=np.asarray(normal, np.float64).reshape(-1, 1),
        face_area=np.ones(len(owner)),
        face_centroid=np.asarray(fc, np.float64).reshape(-1, 1),
        cell_volume=dx.copy(), cell_centroid=(0.5 * (x[1:] + x[:-1])).reshape(-1, 1),
        patches=list(patches) if patches is not None else [Patch(WALL), Patch(WALL)])


def _faces_from_triangles(verts, tris, side_of_edge):
    """Build the face list of a triangle mesh.

    ``side_of_edge(p, q)`` returns the boundary patch id of a boundary edge.
    """
    edge_map = {}
    owner, nbr, e_vert = [], [], []
    for c, t in enumerate(tris):
        for k in range(3):
            a, b = int(t[k]), int(t[(k + 1) % 3])
            key = (a, b) if a < b else (b, a)
            if key in edge_map:
                nbr[edge_map[key]] = c
            else:
                edge_map[key] = len(owner)
                owner.append(c)
                nbr.append(None)
                e_vert.append(key)
    owner = np.asarray(owner, np.int32)
    e_vert = np.asarray(e_vert, np.int64)
    cc = verts[tris].mean(axis=1)
    p, q = verts[e_vert[:, 0]], verts[e_vert[:, 1]]
    d = q - p
    area = np.hypot(d[:, 0], d[:, 1])
    n = np.stack([d[:, 1], -d[:, 0]], axis=1) / area[:, None]
    fc = 0.5 * (p + q)
    flip = np.einsum("ij,ij->i", n, fc - cc[owner]) < 0
    n[flip] *= -1.0
    nb = np.empty(len(owner), np.int32)
    for f, v in enumerate(nbr):
        nb[f] = v if v is not None else -1 - side_of_edge(p[f], q[f])
    x0, y0 = verts[tris[:, 0]].T
    x1, y1 = verts[tris[:, 1]].T
    x2, y2 = verts[tris[:, 2]].T
    vol = 0.5 * np.abs((x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0))
    return owner, nb, n, area, fc, vol, cc


def cavity_triangles(n_side: int, seed: int = 0, jitter: float = 0.2, flip_p: float = 0.5,
                     patches=None) -> Mesh:
    """Jittered, randomly split triangulation of the unit square: 2*n_side^2 cells.

    Interior vertices move by up to ``jitter*h`` in each direction, each square
    is cut along a randomly chosen diagonal.  Cells are numbered square by square
    along a Z-order (Morton) curve, so that any run of consecutive cells is a
    compact patch.  Patches: 0 bottom, 1 right, 2 top (lid), 3 left.
    """
    rng = np.random.default_rng(seed)
    h = 1.0 / n_side
    g = np.linspace(0.0, 1.0, n_side + 1)
    X, Y = np.meshgrid(g, g, indexing="xy")
    verts = np.stack([X.ravel(), Y.ravel()], axis=1)
    inner = (verts[:, 0] > 0) & (verts[:, 0] < 1) & (verts[:, 1] > 0) & (verts[:, 1] < 1)
    verts[inner] += rng.uniform(-jitter * h, jitter * h, size=(int(inner.sum()), 2))
    diag = rng.random(n_side * n_side) < flip_p

    def morton(i, j):
        code = 0
        for b in range(16):
            code |= ((i >> b) & 1) << (2 * b) | ((j >> b) & 1) << (2 * b + 1)
        return code

    squares = sorted(((i, j) for j in range(n_side) for i in range(n_side)), key=lambda t: morton(*t))
    tris = []
    for i, j in squares:
        a = j * (n_side + 1) + i
        b, c, d = a + 1, a + n_side + 2, a + n_side + 1
        if diag[j * n_side + i]:
            tris += [(a, b, c), (a, c, d)]
        else:
            tris += [(a, b, d), (b, c, d)]
    tris = np.asarray(tris, np.int64)

    def side(p, q):
        m = 0.5 * (p + q)
        if abs(m[1]) < 1e-12:
            return 0
        if abs(m[0] - 1.0) < 1e-12:
            return 1
        if abs(m[1] - 1.0) < 1e-12:
            return 2
        return 3

    owner, nb, n, area, fc, vol, cc = _faces_from_triangles(verts, tris, side)
    if patches is None:
        patches = [Patch(WALL, T_t=1.0), Patch(WALL, T_t=1.0),
                   Patch(WALL, u=(0.18, 0.0, 0.0), T_t=3.0), Patch(WALL, T_t=1.0)]
    return Mesh(dim=2, n_cells=len(tris), face_owner=owner, face_nbr=nb, face_normal=n,
                face_area=area, face_centroid=fc, cell_volume=vol, cell_centroid=cc,
                patches=list(patches))


def cylinder_ogrid(n_theta: int, n_radial: int, seed: int = 1, r_body: float = 0.5,
                   r_outer: float = 3.0, stretch: float = 3.0, patches=None) -> Mesh:
    """Triangulated O-grid around a circular cylinder (diameter 1, outer diameter 6).

    Radial spacing clusters geometrically at the wall; each quad is split along a
    seeded random diagonal.  Patches: 0 the cylinder wall, 1 the far field.
    """
    rng = np.random.default_rng(seed)
    s = np.linspace(0.0, 1.0, n_radial + 1)
    r = r_body + (r_outer - r_body) * (np.expm1(stretch * s) / np.expm1(stretch))
    th = np.linspace(0.0, 2.0 * np.pi, n_theta, endpoint=False)
    R, TH = np.meshgrid(r, th, indexing="ij")             # [n_radial+1, n_theta]
    verts = np.stack([(R * np.cos(TH)).ravel(), (R * np.sin(TH)).ravel()], axis=1)
    diag = rng.random(n_radial * n_theta) < 0.5
    tris = []
    for j in range(n_radial):
        for i in range(n_theta):
            i1 = (i + 1) % n_theta
            a, b = j * n_theta + i, j * n_theta + i1
            c, d = (j + 1) * n_theta + i1, (j + 1) * n_theta + i
            if diag[j * n_theta + i]:
                tris += [(a, b, c), (a, c, d)]
            else:
                tris += [(a, b, d), (b, c, d)]
    tris = np.asarray(tris, np.int64)

    def side(p, q):
        m = 0.5 * (p + q)
        return 0 if np.hypot(*m) < 0.5 * (r_body + r_outer) else 1

    owner, nb, n, area, fc, vol, cc = _faces_from_triangles(verts, tris, side)
    if patches is None:
        patches = [Patch(WALL, T_t=0.5), Patch(FARFIELD)]
    return Mesh(dim=2, n_cells=len(tris), face_owner=owner, face_nbr=nb, face_normal=n,
                face_area=area, face_centroid=fc, cell_volume=vol, cell_centroid=cc,
                patches=list(patches))
