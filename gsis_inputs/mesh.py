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
    # > 0: the domain is periodic in x with this period (centroid differences wrap)
    period: float = 0.0

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


def ring_1d(n_cells: int, length: float = 1.0) -> Mesh:
    """Uniform periodic 1-D row of cells on [0, L): the slab's interior faces plus one face
    from the last cell to the first (normal +x), so every cell has an upstream and a
    downstream neighbour.  No boundary patches.  The mesh carries period = L, so that a
    consumer that honours it takes centroid differences across that face as those of a
    periodic domain (the minimal image); one that does not is periodic only where no
    centroid difference enters (first-order transport)."""
    x = np.linspace(0.0, length, n_cells + 1)
    owner = list(range(n_cells - 1)) + [n_cells - 1]
    nbr = list(range(1, n_cells)) + [0]
    fc = list(x[1:-1]) + [x[-1]]
    return Mesh(
        dim=1, n_cells=n_cells,
        face_owner=np.asarray(owner, np.int32), face_nbr=np.asarray(nbr, np.int32),
        face_normal=np.ones((n_cells, 1)), face_area=np.ones(n_cells),
        face_centroid=np.asarray(fc, np.float64).reshape(-1, 1),
        cell_volume=np.diff(x), cell_centroid=(0.5 * (x[1:] + x[:-1])).reshape(-1, 1), patches=[],
        period=float(length))


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


def channel_triangles(n_side: int, seed: int = 0, jitter: float = 0.2, flip_p: float = 0.5,
                      patches=None) -> Mesh:
    """The unit square of ``cavity_triangles`` made periodic in x (period 1): its left and
    right boundary edges (whose vertices are not jittered, so they pair by height) become
    interior faces from the cell at x = 1 to the cell at x = 0, with the right edge's
    normal (+x) and centroid.  Patches: 0 bottom, 1 top."""
    m = cavity_triangles(n_side, seed=seed, jitter=jitter, flip_p=flip_p,
                         patches=[Patch(WALL), Patch(WALL), Patch(WALL), Patch(WALL)])
    right = np.where(m.face_nbr == -1 - 1)[0]
    left = np.where(m.face_nbr == -1 - 3)[0]
    by_y = {round(float(m.face_centroid[f, 1]), 9): f for f in left}
    owner, nbr = m.face_owner.copy(), m.face_nbr.copy()
    keep = np.ones(m.n_faces, bool)
    for f in right:
        g = by_y[round(float(m.face_centroid[f, 1]), 9)]
        nbr[f] = owner[g]               # right cell -> left cell across the seam
        keep[g] = False
    nbr[nbr == -1 - 2] = -1 - 1         # top wall becomes patch 1
    if patches is None:
        patches = [Patch(WALL, T_t=1.0), Patch(WALL, u=(0.2, 0.0, 0.0), T_t=1.0)]
    return Mesh(dim=2, n_cells=m.n_cells, face_owner=owner[keep], face_nbr=nbr[keep],
                face_normal=m.face_normal[keep], face_area=m.face_area[keep],
                face_centroid=m.face_centroid[keep], cell_volume=m.cell_volume,
                cell_centroid=m.cell_centroid, patches=list(patches), period=1.0)


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


def box_tetrahedra(n: int, seed: int = 2, jitter: float = 0.15, size=(1.0, 1.0, 1.0), patches=None) -> Mesh:
    """Jittered tetrahedral mesh of a box: n^3 hexahedra, each cut into 6 tetrahedra along
    its main diagonal (every hexahedron cut the same way, so neighbouring cuts match):
    6 n^3 cells.  Interior vertices move by up to ``jitter*h`` per direction.  Hexahedra
    are numbered along a 3-D Morton curve and each one's tetrahedra are consecutive, so
    runs of consecutive cells are compact.  Patches: 0 x = 0, 1 x = L_x, 2 y = 0,
    3 y = L_y, 4 z = 0, 5 z = L_z (walls by default)."""
    rng = np.random.default_rng(seed)
    L = np.asarray(size, np.float64)
    g = np.linspace(0.0, 1.0, n + 1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    inner = np.all((verts > 0) & (verts < 1), axis=1)
    verts[inner] += rng.uniform(-jitter / n, jitter / n, size=(int(inner.sum()), 3))
    verts *= L[None]
    vid = lambda i, j, k: (i * (n + 1) + j) * (n + 1) + k

    def morton3(i, j, k):
        code = np.zeros_like(i)
        for b in range(11):
            code |= (((i >> b) & 1) << (3 * b)) | (((j >> b) & 1) << (3 * b + 1)) | (((k >> b) & 1) << (3 * b + 2))
        return code

    I, J, Kk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    I, J, Kk = I.ravel(), J.ravel(), Kk.ravel()
    order = np.argsort(morton3(I, J, Kk), kind="stable")
    I, J, Kk = I[order], J[order], Kk[order]
    perms = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))
    tets = []
    for p in perms:
        path = [np.zeros(3, int)]
        for a in p:
            step = path[-1].copy()
            step[a] = 1
            path.append(step)
        tets.append(np.stack([vid(I + c[0], J + c[1], Kk + c[2]) for c in path], axis=1))
    tets = np.stack(tets, axis=1).reshape(-1, 4)                 # [hex * 6 + t, 4]
    P = verts[tets]                                             # [nc, 4, 3]
    vol6 = np.einsum("nd,nd->n", np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), P[:, 3] - P[:, 0])
    vol = np.abs(vol6) / 6.0
    cc = P.mean(axis=1)
    # faces: the triple opposite each vertex; shared triples pair owner and neighbour
    tri = np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]], tets[:, [0, 1, 3]], tets[:, [0, 1, 2]]])
    cell = np.concatenate([np.arange(tets.shape[0])] * 4)
    key = np.sort(tri, axis=1)
    o = np.lexsort((key[:, 2], key[:, 1], key[:, 0]))
    key, tri, cell = key[o], tri[o], cell[o]
    same = np.all(key[1:] == key[:-1], axis=1)
    first = np.ones(key.shape[0], bool)
    first[1:] = ~same
    owner = cell[first]
    ftri = tri[first]
    nb = np.full(owner.shape[0], -1, np.int64)
    idx_first = np.nonzero(first)[0]
    pair = np.zeros(key.shape[0], bool)
    pair[:-1] = same
    nb[np.searchsorted(idx_first, np.nonzero(pair)[0])] = cell[np.nonzero(pair)[0] + 1]
    A, B, C = verts[ftri[:, 0]], verts[ftri[:, 1]], verts[ftri[:, 2]]
    cr = np.cross(B - A, C - A)
    area = 0.5 * np.linalg.norm(cr, axis=1)
    nrm = cr / (2.0 * area[:, None])
    fc = (A + B + C) / 3.0
    flip = np.einsum("fd,fd->f", nrm, fc - cc[owner]) < 0.0     # outward from the owner
    nrm[flip] = -nrm[flip]
    bnd = nb < 0
    side = np.zeros(owner.shape[0], np.int64)
    for a in range(3):
        side[bnd & (np.abs(fc[:, a]) < 1e-9 * L[a])] = 2 * a
        side[bnd & (np.abs(fc[:, a] - L[a]) < 1e-9 * L[a])] = 2 * a + 1
    nb[bnd] = -1 - side[bnd]
    if patches is None:
        patches = [Patch(WALL, T_t=1.0) for _ in range(6)]
    return Mesh(dim=3, n_cells=int(tets.shape[0]), face_owner=owner.astype(np.int32), face_nbr=nb.astype(np.int32),
                face_normal=nrm, face_area=area, face_centroid=fc, cell_volume=vol, cell_centroid=cc,
                patches=list(patches))


def drop_cells(m: Mesh, keep, patch: int) -> Mesh:
    """The mesh without the cells where ``keep`` is False, numbered in their old order.
    Faces between a kept and a dropped cell become boundary faces of ``patch`` (normal
    outward from the kept cell); faces of dropped cells only are removed."""
    keep = np.asarray(keep, bool)
    new = np.full(m.n_cells, -1, np.int64)
    new[keep] = np.arange(int(keep.sum()))
    o, nb = m.face_owner.astype(np.int64), m.face_nbr.astype(np.int64)
    ko = keep[o]
    kn = np.where(nb >= 0, keep[np.maximum(nb, 0)], False)
    inner = nb >= 0
    owner = np.where(ko, o, np.maximum(nb, 0))
    nbr = np.where(ko & kn, nb, np.where(inner, -1 - patch, nb))
    flip = ~ko & kn
    use = ko | kn
    normal = np.where(flip[:, None], -m.face_normal, m.face_normal)
    owner, nbr = new[owner[use]], nbr[use]
    nbr = np.where(nbr >= 0, new[np.maximum(nbr, 0)], nbr)
    return Mesh(dim=m.dim, n_cells=int(keep.sum()), face_owner=owner.astype(np.int32), face_nbr=nbr.astype(np.int32),
                face_normal=normal[use], face_area=m.face_area[use], face_centroid=m.face_centroid[use],
                cell_volume=m.cell_volume[keep], cell_centroid=m.cell_centroid[keep], patches=list(m.patches))


def sphere_cone_radius(x, x_nose=0.3, D=0.4, half_angle=60.0, nose=0.25, shoulder=0.1, aft_angle=40.0,
                       back=0.5):
    """Body radius r(x) (0 outside the body) of an axisymmetric sphere-cone entry capsule
    facing -x: a spherical nose of radius nose*D at x_nose, tangent to a cone of the given
    half-angle, rounded at the base diameter D by a torus of radius shoulder*D, then a
    conical afterbody narrowing at aft_angle to a flat back of radius back*D/2."""
    x = np.asarray(x, np.float64)
    R, Rn, Rs = 0.5 * D, nose * D, shoulder * D
    th, ta = np.radians(half_angle), np.radians(aft_angle)
    xc = x_nose + Rn                                    # nose centre
    xt, rt = xc - Rn * np.sin(th), Rn * np.cos(th)      # nose-cone tangency
    rp = R - Rs + Rs * np.cos(th)                       # cone-shoulder tangency
    xp = xt + (rp - rt) / np.tan(th)
    cx, cr = xp + Rs * np.sin(th), R - Rs               # shoulder centre
    x2, r2 = cx + Rs * np.sin(ta), cr + Rs * np.cos(ta) # shoulder-afterbody tangency
    rb = back * R
    xb = x2 + (r2 - rb) / np.tan(ta)
    r = np.zeros_like(x)
    m = (x >= x_nose) & (x < xt)
    r[m] = np.sqrt(np.maximum(Rn * Rn - (xc - x[m]) ** 2, 0.0))
    m = (x >= xt) & (x < xp)
    r[m] = rt + (x[m] - xt) * np.tan(th)
    m = (x >= xp) & (x < x2)
    r[m] = cr + np.sqrt(np.maximum(Rs * Rs - (x[m] - cx) ** 2, 0.0))
    m = (x >= x2) & (x <= xb)
    r[m] = r2 - (x[m] - x2) * np.tan(ta)
    return r


def capsule_tetrahedra(n: int, seed: int = 2, jitter: float = 0.15, patches=None) -> Mesh:
    """Sphere-cone re-entry capsule in the unit cube, tetrahedral: box_tetrahedra(n)
    without the cells whose centroids lie inside the body (sphere_cone_radius: axis
    y = z = 0.5, stagnation point x = 0.3, base diameter D = 0.4, 60-degree forebody
    cone with nose radius 0.25 D, shoulder radius 0.1 D, 40-degree afterbody to a flat
    back of diameter D / 2).  The exposed faces form patch 0 (the body), the six sides
    of the cube patch 1 (far field); ``patches`` gives those two."""
    box = box_tetrahedra(n, seed=seed, jitter=jitter)
    x, y, z = box.cell_centroid.T
    inside = np.hypot(y - 0.5, z - 0.5) <= sphere_cone_radius(x)
    box.face_nbr = np.where(box.face_nbr < 0, -2, box.face_nbr).astype(np.int32)   # cube sides: patch 1
    if patches is None:
        patches = [Patch(WALL, T_t=1.0), Patch(FARFIELD)]
    box.patches = list(patches)
    return drop_cells(box, ~inside, 0)
