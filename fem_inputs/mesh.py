"""Structured tetrahedral box meshes with hierarchical-P2 node numbering.

The paper's test meshes (Sec. 4.1, Table 1) are the unit cube cut into n^3
cubes.  Each cube is split into the 6 Kuhn (Freudenthal) tetrahedra that share
the cube's main diagonal; with that split the vertex and mid-side node counts
of Table 1 are reproduced exactly (the "#Tet" column of Table 1 lists the cube
count, the tetrahedron count is six times it).

Node numbering (Sec. 2.4, Eq. (ellipticeqn) orders the unknowns [u_l; u_q]):
vertices first, id = i + (nx+1)*(j + (ny+1)*k); then edges, numbered in
increasing (min vertex id, max vertex id).  Each tetrahedron lists its 4
vertices and its 6 edges in the paper's local edge order (12),(23),(34),
(13),(14),(24) of Sec. 2.3.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

# local vertex pairs of the paper's bubbles phi_5..phi_10 (Sec. 2.3), 0-based
LOCAL_EDGES = np.array([(0, 1), (1, 2), (2, 3), (0, 2), (0, 3), (1, 3)], dtype=np.int64)

# the six axis permutations, each giving one Kuhn tetrahedron of a cube
KUHN_PERMS = list(itertools.permutations(range(3)))


@dataclass
class BoxMesh:
    nx: int
    ny: int
    nz: int
    lengths: tuple
    coords: np.ndarray      # (NV, 3) float64 vertex coordinates
    tets: np.ndarray        # (NT, 4) int64 vertex ids
    edges: np.ndarray       # (NE, 2) int64 (min, max) vertex ids, sorted
    tet_edges: np.ndarray   # (NT, 6) int64 edge ids in LOCAL_EDGES order
    grid: np.ndarray        # (NV, 3) int64 lattice index (i, j, k) of each vertex

    @property
    def n_vertices(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_edges(self) -> int:
        return int(self.edges.shape[0])

    @property
    def n_nodes(self) -> int:
        """P2 nodes: vertices then edge midpoints."""
        return self.n_vertices + self.n_edges

    def tet_nodes(self) -> np.ndarray:
        """(NT, 10) global node ids: 4 vertices, then 6 edges (offset by NV)."""
        return np.concatenate([self.tets, self.tet_edges + self.n_vertices], axis=1)

    def node_coords(self) -> np.ndarray:
        """(NV+NE, 3) coordinates of vertices then edge midpoints."""
        mid = 0.5 * (self.coords[self.edges[:, 0]] + self.coords[self.edges[:, 1]])
        return np.concatenate([self.coords, mid], axis=0)


def box_mesh(nx: int, ny: int | None = None, nz: int | None = None,
             lengths=(1.0, 1.0, 1.0), jitter: float = 0.0,
             rng: np.random.Generator | None = None) -> BoxMesh:
    """Kuhn-split box mesh of nx*ny*nz bricks over [0,Lx]x[0,Ly]x[0,Lz].

    jitter > 0 moves every interior vertex by a seeded uniform offset in
    [-jitter*h, jitter*h] per coordinate (h = brick size along that axis);
    boundary vertices stay on their faces.  Every tetrahedron must keep a
    positive volume, which is asserted.
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    Lx, Ly, Lz = (float(v) for v in lengths)
    n1 = np.array([nx + 1, ny + 1, nz + 1], dtype=np.int64)
    kk, jj, ii = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    grid = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1).astype(np.int64)
    h = np.array([Lx / nx, Ly / ny, Lz / nz])
    coords = grid.astype(np.float64) * h
    if jitter > 0.0:
        assert rng is not None, "jittered meshes need a seeded generator"
        off = rng.uniform(-jitter, jitter, size=coords.shape) * h
        interior = np.ones(len(coords), dtype=bool)
        for ax in range(3):
            # keep each vertex on every face it lies on (coordinate clamp per axis)
            on = (grid[:, ax] == 0) | (grid[:, ax] == n1[ax] - 1)
            off[on, ax] = 0.0
            interior &= ~on
        coords = coords + off

    def vid(g):
        return g[..., 0] + n1[0] * (g[..., 1] + n1[1] * g[..., 2])

    bk, bj, bi = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    base = np.stack([bi.ravel(), bj.ravel(), bk.ravel()], axis=1).astype(np.int64)
    eye = np.eye(3, dtype=np.int64)
    tets = []
    # brick-major ordering: the 6 tetrahedra of a brick are consecutive
    for b in range(6):
        a0, a1, a2 = KUHN_PERMS[b]
        v0 = base
        v1 = v0 + eye[a0]
        v2 = v1 + eye[a1]
        v3 = v2 + eye[a2]
        tets.append(np.stack([vid(v0), vid(v1), vid(v2), vid(v3)], axis=1))
    tets = np.stack(tets, axis=1).reshape(-1, 4)

    pairs = tets[:, LOCAL_EDGES]                     # (NT, 6, 2)
    lo = pairs.min(axis=2)
    hi = pairs.max(axis=2)
    nv = len(coords)
    key = lo * nv + hi
    ukey, inv = np.unique(key.ravel(), return_inverse=True)
    edges = np.stack([ukey // nv, ukey % nv], axis=1)
    tet_edges = inv.reshape(-1, 6)

    mesh = BoxMesh(nx, ny, nz, (Lx, Ly, Lz), coords, tets, edges, tet_edges, grid)
    vol = tet_volumes(mesh.coords, mesh.tets)
    assert np.all(np.abs(vol) > 0.0), "degenerate tetrahedron"
    if jitter > 0.0:
        # the jitter must not flip any element relative to the unjittered mesh
        ref = tet_volumes(grid.astype(np.float64) * h, tets)
        assert np.all(np.sign(vol) == np.sign(ref)), "jitter inverted a tetrahedron"
    return mesh


def tet_volumes(coords: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Signed volumes det[X1-X0, X2-X0, X3-X0]/6."""
    X = coords[tets]
    J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)
    return np.linalg.det(J) / 6.0


def boundary_faces(mesh: BoxMesh, axis: int, side: int) -> np.ndarray:
    """Boundary triangles on the face {x_axis = 0} (side 0) or {x_axis = L} (side 1).

    Returns (NF, 3) vertex ids, each row sorted ascending, rows sorted
    lexicographically, so the "triangle order" of seeded loads is well defined.
    """
    target = 0 if side == 0 else (mesh.nx, mesh.ny, mesh.nz)[axis]
    on = mesh.grid[:, axis] == target
    faces = []
    for drop in range(4):
        keep = [c for c in range(4) if c != drop]
        tri = mesh.tets[:, keep]
        m = on[tri].all(axis=1)
        faces.append(tri[m])
    faces = np.sort(np.concatenate(faces, axis=0), axis=1)
    faces = np.unique(faces, axis=0)
    return faces


def face_edges(mesh: BoxMesh, faces: np.ndarray) -> np.ndarray:
    """(NF, 3) edge ids of each triangle, for local edges (01), (12), (02)."""
    nv = mesh.n_vertices
    ekey = mesh.edges[:, 0] * nv + mesh.edges[:, 1]
    out = np.empty((len(faces), 3), dtype=np.int64)
    for c, (a, b) in enumerate([(0, 1), (1, 2), (0, 2)]):
        lo = np.minimum(faces[:, a], faces[:, b])
        hi = np.maximum(faces[:, a], faces[:, b])
        idx = np.searchsorted(ekey, lo * nv + hi)
        assert np.all(ekey[idx] == lo * nv + hi)
        out[:, c] = idx
    return out
