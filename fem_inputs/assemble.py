"""Exact assembly of the hierarchical-P2 (and Taylor-Hood P2/P1) systems of Sec. 2.

Basis on a tetrahedron (Sec. 2.3): the hats lambda_1..lambda_4 and the bubbles
4*lambda_a*lambda_b over the local edges (12),(23),(34),(13),(14),(24).
Every basis gradient is linear, so it is written as
    grad phi_i = sum_p lambda_p * c[i, p]          (c[i, p] in R^3)
with c[i, p] = grad lambda_i for a hat and
c[e, p] = 4 (delta_pa grad lambda_b + delta_pb grad lambda_a) for the bubble of
edge (a, b).  Products of two gradients then integrate exactly with
    int_T lambda_p lambda_q = |T| (1 + delta_pq) / 20.

Bilinear forms (Sec. 2.2, Eqs. (weakveclapform), (weakelasmixform)):
    vector Laplacian   a(u,v) = int grad u : grad v
    elasticity         a(u,v) = int 2 mu eps(u):eps(v) + lam div u div v
    mixed / Stokes     a(u,v) = 2 mu int eps(u):eps(v),
                       b(v,q) = -int q div v,   c(p,q) = (1/lam) int p q  (0 for Stokes)
With G_ij[al, be] = int d_al phi_i d_be phi_j and S_ij = trace G_ij, the 3x3
block coupling test function i with trial function j is
    Laplacian:   S_ij I
    elasticity:  mu S_ij I + mu G_ij^T + lam G_ij
    mixed:       mu S_ij I + mu G_ij^T
B_kj[be] = -int lambda_k d_be phi_j and C_kl = (1/lam) int lambda_k lambda_l.
Element matrices are symmetrised as (K + K^T)/2 before summation, so the
assembled A is exactly symmetric in floating point.
"""
from __future__ import annotations

import numpy as np

from .mesh import LOCAL_EDGES, BoxMesh


def barycentric_gradients(X: np.ndarray):
    """X: (T, 4, 3) vertex coordinates -> (grads (T,4,3), volumes (T,))."""
    J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)          # row k = grad lambda_{k+1}
    g = np.empty((len(X), 4, 3))
    g[:, 1:] = Jinv
    g[:, 0] = -Jinv.sum(axis=1)
    return g, np.abs(det) / 6.0


def gradient_coefficients(g: np.ndarray) -> np.ndarray:
    """c[t, i, p, :] with grad phi_i = sum_p lambda_p c[t, i, p] (i over 10 basis functions)."""
    T = len(g)
    c = np.zeros((T, 10, 4, 3))
    for i in range(4):
        c[:, i, :, :] = g[:, i, None, :]          # sum_p lambda_p = 1
    for e, (a, b) in enumerate(LOCAL_EDGES):
        c[:, 4 + e, a, :] += 4.0 * g[:, b]
        c[:, 4 + e, b, :] += 4.0 * g[:, a]
    return c


def lambda_mass(vol: np.ndarray) -> np.ndarray:
    """M[t,p,q] = int_T lambda_p lambda_q = |T| (1+delta_pq)/20."""
    M = np.full((len(vol), 4, 4), 1.0) + np.eye(4)
    return M * (vol / 20.0)[:, None, None]


def element_blocks(X: np.ndarray, kind: str, mu: float = 1.0, lam: float = 1.0):
    """Velocity element matrix as (T, 10, 10, 3, 3) blocks, symmetrised."""
    g, vol = barycentric_gradients(X)
    c = gradient_coefficients(g)
    M = lambda_mass(vol)
    # G[t,i,j,al,be] = sum_pq c[t,i,p,al] M[t,p,q] c[t,j,q,be], as batched products of
    # the (30 x 4) coefficient matrix with M
    T = len(X)
    C30 = np.ascontiguousarray(np.transpose(c, (0, 1, 3, 2))).reshape(T, 30, 4)
    G30 = C30 @ M @ np.transpose(C30, (0, 2, 1))
    G = np.transpose(G30.reshape(T, 10, 3, 10, 3), (0, 1, 3, 2, 4))
    S = np.trace(G, axis1=3, axis2=4)
    I3 = np.eye(3)
    if kind == "laplace":
        K = S[..., None, None] * I3
    elif kind == "elasticity":
        K = mu * S[..., None, None] * I3 + mu * np.swapaxes(G, 3, 4) + lam * G
    elif kind in ("mixed", "stokes"):
        K = mu * S[..., None, None] * I3 + mu * np.swapaxes(G, 3, 4)
    else:
        raise ValueError(kind)
    # symmetrise the 30x30 element matrix: K_ij[a,b] <-> K_ji[b,a]
    K = 0.5 * (K + np.transpose(K, (0, 2, 1, 4, 3)))
    return K


def element_divergence(X: np.ndarray):
    """B_e[t,k,j,be] = -int lambda_k d_be phi_j  (k over 4 pressure hats)."""
    g, vol = barycentric_gradients(X)
    c = gradient_coefficients(g)
    M = lambda_mass(vol)
    return -np.einsum("tkp,tjpb->tkjb", M, c)


def element_pressure_mass(X: np.ndarray):
    """int lambda_k lambda_l, (T, 4, 4)."""
    _, vol = barycentric_gradients(X)
    return lambda_mass(vol)


def _csr_from_keys(rows: np.ndarray, cols: np.ndarray, n_rows: int, n_cols: int):
    """Sorted unique (row, col) pattern -> rowptr, col, and the inverse map."""
    key = rows.astype(np.int64) * n_cols + cols
    ukey, inv = np.unique(key, return_inverse=True)
    r = ukey // n_cols
    col = (ukey % n_cols).astype(np.int32)
    rowptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    return rowptr, col, inv


def _uniform(mesh: BoxMesh) -> bool:
    """True when every brick is a translate of the first (an unjittered box mesh):
    the 6 element matrices of the first brick then serve all bricks."""
    h = np.array(mesh.lengths) / np.array([mesh.nx, mesh.ny, mesh.nz])
    return bool(np.array_equal(mesh.coords, mesh.grid.astype(np.float64) * h))


def _element_stream(mesh: BoxMesh, fn, chunk: int):
    """Yields (start, element arrays) over chunks of tetrahedra; on uniform meshes
    the first brick's 6 element arrays are tiled (tetrahedra are brick-major)."""
    X = mesh.coords[mesh.tets]
    T = len(X)
    if _uniform(mesh):
        ref = fn(X[:6])
        for s in range(0, T, chunk):
            cnt = min(chunk, T - s)
            reps = -(-cnt // 6) + 1
            tiled = np.concatenate([ref] * reps, axis=0)
            off = s % 6
            yield s, tiled[off:off + cnt]
        return
    for s in range(0, T, chunk):
        yield s, fn(X[s:s + chunk])


def assemble_velocity(mesh: BoxMesh, kind: str, mu: float = 1.0, lam: float = 1.0,
                      chunk: int = 16386):
    """Global 3x3-block CSR of A over all P2 nodes, structural pattern = node pairs
    sharing a tetrahedron.  Returns rowptr (N+1,), col (nnzb,), val (nnzb, 3, 3)."""
    tn = mesh.tet_nodes()                                # (T, 10)
    N = mesh.n_nodes
    rows = np.repeat(tn, 10, axis=1).ravel()
    cols = np.tile(tn, (1, 10)).ravel()
    rowptr, col, inv = _csr_from_keys(rows, cols, N, N)
    inv = inv.reshape(len(tn), 100)
    nnzb = len(col)
    val = np.zeros((nnzb, 9))
    for s, Ke in _element_stream(mesh, lambda X: element_blocks(X, kind, mu, lam), chunk):
        Ke = Ke.reshape(-1, 9)
        idx = inv[s:s + len(Ke) // 100].ravel()
        for comp in range(9):
            val[:, comp] += np.bincount(idx, weights=Ke[:, comp], minlength=nnzb)
    return rowptr, col, val.reshape(nnzb, 3, 3)


def assemble_divergence(mesh: BoxMesh, chunk: int = 16386):
    """B as 1x3-block CSR: rows = pressure nodes (vertices), cols = velocity nodes."""
    tn = mesh.tet_nodes()
    rows = np.repeat(mesh.tets, 10, axis=1).ravel()
    cols = np.tile(tn, (1, 4)).ravel()
    rowptr, col, inv = _csr_from_keys(rows, cols, mesh.n_vertices, mesh.n_nodes)
    inv = inv.reshape(len(tn), 40)
    nnz = len(col)
    val = np.zeros((nnz, 3))
    for s, Be in _element_stream(mesh, element_divergence, chunk):
        Be = Be.reshape(-1, 3)
        idx = inv[s:s + len(Be) // 40].ravel()
        for comp in range(3):
            val[:, comp] += np.bincount(idx, weights=Be[:, comp], minlength=nnz)
    return rowptr, col, val


def assemble_pressure_mass(mesh: BoxMesh, scale: float, chunk: int = 65538):
    """scale * int lambda_k lambda_l as scalar CSR over vertices (the P1 pattern)."""
    rows = np.repeat(mesh.tets, 4, axis=1).ravel()
    cols = np.tile(mesh.tets, (1, 4)).ravel()
    nv = mesh.n_vertices
    rowptr, col, inv = _csr_from_keys(rows, cols, nv, nv)
    inv = inv.reshape(len(mesh.tets), 16)
    val = np.zeros(len(col))
    for s, Me in _element_stream(mesh, element_pressure_mass, chunk):
        Me = Me.reshape(-1) * scale
        val += np.bincount(inv[s:s + len(Me) // 16].ravel(), weights=Me, minlength=len(col))
    return rowptr, col, val


def face_load(mesh: BoxMesh, faces: np.ndarray, fedges: np.ndarray, gvals: np.ndarray):
    """Exact int_F g . phi_i for P2 traces on boundary triangles.

    gvals: (NF, 3, 3) traction at the triangle's 3 vertices (row = vertex,
    col = component); g is linear on the face (a constant traction repeats the
    value).  Moments: int_F mu^alpha = 2|F| alpha! / (|alpha| + 2)!.
    Returns a (NV+NE, 3) nodal load.
    """
    X = mesh.coords[faces]
    area = 0.5 * np.linalg.norm(np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), axis=1)
    out = np.zeros((mesh.n_nodes, 3))
    # hat m: sum_k g_k |F| (1 + delta_km) / 12
    for m in range(3):
        w = np.full(3, 1.0 / 12.0)
        w[m] = 2.0 / 12.0
        contrib = area[:, None] * np.einsum("k,fkc->fc", w, gvals)
        np.add.at(out, faces[:, m], contrib)
    # bubble 4 mu_a mu_b: sum_k g_k 4 * (|F|/30 if k in {a,b} else |F|/60)
    for e, (a, b) in enumerate([(0, 1), (1, 2), (0, 2)]):
        w = np.full(3, 4.0 / 60.0)
        w[a] = 4.0 / 30.0
        w[b] = 4.0 / 30.0
        contrib = area[:, None] * np.einsum("k,fkc->fc", w, gvals)
        np.add.at(out, mesh.n_vertices + fedges[:, e], contrib)
    return out


def hierarchical_interpolant(mesh: BoxMesh, fun) -> np.ndarray:
    """P2 hierarchical coefficients of a vector function: value at each vertex, and
    g(mid) - (g(a) + g(b))/2 at each edge.  fun maps (K,3) points to (K,d)."""
    gv = fun(mesh.coords)
    a, b = mesh.edges[:, 0], mesh.edges[:, 1]
    mid = 0.5 * (mesh.coords[a] + mesh.coords[b])
    ge = fun(mid) - 0.5 * (gv[a] + gv[b])
    return np.concatenate([gv, ge], axis=0)
