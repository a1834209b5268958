"""Seeded synthetic systems in the form of Sec. 2.4 (Eqs. (ellipticeqn), (mixedeqn)).

Each builder returns a `Problem`: the homogenised block system with Dirichlet
nodes kept as identity rows (zero off-diagonal blocks in row and column, zero
right-hand side), node tags, and the Dirichlet lift so that the full finite
element solution is  u = u_0 + lift.

Dirichlet elimination is symmetric: the known coefficients are moved to the
right-hand side (f <- f - A[:, D] x_D, g <- g - B[:, D] x_D), then the
couplings of Dirichlet nodes are zeroed but kept in the sparsity pattern, so
the pattern stays the topological one (node pairs sharing a tetrahedron).

Generators are numpy's PCG64 (`np.random.default_rng(seed)`), portable across
platforms; every random draw of a problem comes from its own seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .assemble import (assemble_divergence, assemble_pressure_mass, assemble_velocity,
                       face_load, hierarchical_interpolant)
from .mesh import BoxMesh, box_mesh, boundary_faces, face_edges

TAG_VERTEX = 0
TAG_EDGE = 1
TAG_DIRICHLET = 0x10

KIND_CODES = {"laplace": 0, "elasticity": 1, "mixed": 2, "stokes": 3}


@dataclass
class Problem:
    name: str
    kind: str                       # laplace | elasticity | mixed | stokes
    mesh: BoxMesh
    a_rowptr: np.ndarray            # int32 (N+1,)
    a_col: np.ndarray               # int32 (nnzb,)
    a_val: np.ndarray               # float64 (nnzb, 3, 3), row-major blocks
    tags: np.ndarray                # int32 (N,)
    f: np.ndarray                   # float64 (N, 3) homogenised load
    lift: np.ndarray                # float64 (N, 3) Dirichlet coefficients
    b_rowptr: np.ndarray | None = None   # int32 (NP+1,)
    b_col: np.ndarray | None = None      # int32
    b_val: np.ndarray | None = None      # float64 (nnz, 3)
    c_rowptr: np.ndarray | None = None
    c_col: np.ndarray | None = None
    c_val: np.ndarray | None = None      # float64, zeros for Stokes (pattern = P1 graph)
    g: np.ndarray | None = None          # float64 (NP,)
    exact_u: np.ndarray | None = None    # (N, 3) exact hierarchical coefficients, if known
    exact_p: np.ndarray | None = None
    p_weights: np.ndarray | None = None  # int phi_i of the P1 pressure basis (Stokes)
    params: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return len(self.tags)

    @property
    def n_pres(self) -> int:
        return 0 if self.g is None else len(self.g)

    @property
    def n_dof(self) -> int:
        return 3 * self.n_nodes + self.n_pres

    @property
    def saddle(self) -> bool:
        return self.kind in ("mixed", "stokes")

    def rhs(self) -> np.ndarray:
        """Full right-hand side [f; g] as one float64 vector."""
        if self.saddle:
            return np.concatenate([self.f.ravel(), self.g])
        return self.f.ravel().copy()

    def a_scipy(self) -> sp.bsr_matrix:
        N = self.n_nodes
        return sp.bsr_matrix((self.a_val, self.a_col, self.a_rowptr), shape=(3 * N, 3 * N))


def lame(E: float, nu: float):
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    return lam, mu


def node_tags(mesh: BoxMesh, dirichlet_vertices: np.ndarray) -> np.ndarray:
    """Vertex / edge tags; an edge is Dirichlet when both its end vertices are
    (it then lies on the Dirichlet part of the boundary of a box)."""
    tags = np.concatenate([np.full(mesh.n_vertices, TAG_VERTEX, np.int32),
                           np.full(mesh.n_edges, TAG_EDGE, np.int32)])
    dv = np.zeros(mesh.n_vertices, dtype=bool)
    dv[dirichlet_vertices] = True
    de = dv[mesh.edges[:, 0]] & dv[mesh.edges[:, 1]]
    tags[:mesh.n_vertices][dv] |= TAG_DIRICHLET
    tags[mesh.n_vertices:][de] |= TAG_DIRICHLET
    return tags


def _bsr_matvec(rowptr, col, val, x):
    N = len(rowptr) - 1
    A = sp.bsr_matrix((val, col, rowptr), shape=(3 * N, 3 * x.shape[0]))
    return (A @ x.ravel()).reshape(-1, 3)


def eliminate_dirichlet(prob: Problem) -> Problem:
    """Symmetric elimination of the Dirichlet nodes (see module docstring)."""
    dmask = (prob.tags & TAG_DIRICHLET) != 0
    lift = np.where(dmask[:, None], prob.lift, 0.0)
    prob.lift = lift
    prob.f = prob.f - _bsr_matvec(prob.a_rowptr, prob.a_col, prob.a_val, lift)
    prob.f[dmask] = 0.0
    rows = np.repeat(np.arange(prob.n_nodes), np.diff(prob.a_rowptr))
    cols = prob.a_col
    touch = dmask[rows] | dmask[cols]
    prob.a_val[touch] = 0.0
    diag = touch & (rows == cols)
    prob.a_val[diag] = np.eye(3)
    if prob.saddle:
        brows = np.repeat(np.arange(prob.n_pres), np.diff(prob.b_rowptr))
        bl = np.einsum("kc,kc->k", prob.b_val, lift[prob.b_col])
        prob.g = prob.g - np.bincount(brows, weights=bl, minlength=prob.n_pres)
        prob.b_val[dmask[prob.b_col]] = 0.0
        # a pressure test function whose support holds no free velocity node gives
        # an equation between boundary data only; its data mismatch is dropped
        free_rows = np.bincount(brows, weights=np.abs(prob.b_val).sum(axis=1),
                                minlength=prob.n_pres) > 0.0
        cdiag = np.zeros(prob.n_pres)
        crows = np.repeat(np.arange(prob.n_pres), np.diff(prob.c_rowptr))
        on_diag = crows == prob.c_col
        cdiag[crows[on_diag]] = prob.c_val[on_diag]
        prob.g[~free_rows & (cdiag == 0.0)] = 0.0
    return prob


def _face_normal(axis: int, side: int) -> np.ndarray:
    n = np.zeros(3)
    n[axis] = -1.0 if side == 0 else 1.0
    return n


def _all_faces():
    return [(ax, s) for ax in range(3) for s in (0, 1)]


# ----------------------------------------------------------------------------------------
# vector Laplacian (Eq. (veclap)) with a harmonic quadratic solution
# ----------------------------------------------------------------------------------------

def harmonic_quadratic(rng: np.random.Generator):
    """u_c(x) = a_c + b_c.x + x^T H_c x with trace(H_c) = 0, for c = 0..2."""
    a = rng.standard_normal(3)
    b = rng.standard_normal((3, 3))
    H = rng.standard_normal((3, 3, 3))
    H = 0.5 * (H + np.transpose(H, (0, 2, 1)))
    for c in range(3):
        H[c] -= np.trace(H[c]) / 3.0 * np.eye(3)

    def u(x):
        return a[None, :] + x @ b.T + np.einsum("ki,cij,kj->kc", x, H, x)

    def grad(x):   # (K, 3 components, 3 derivatives)
        return b[None, :, :] + 2.0 * np.einsum("cij,kj->kci", H, x)

    return u, grad


def vector_laplace_problem(n: int, seed: int = 0, dirichlet_faces=((2, 0),)) -> Problem:
    """-Delta u = 0 on the unit cube, u = harmonic quadratic: Dirichlet data on
    `dirichlet_faces`, Neumann data du/dn on the other faces; the exact FE solution
    is the hierarchical interpolant of u."""
    rng = np.random.default_rng(seed)
    mesh = box_mesh(n)
    u, grad = harmonic_quadratic(rng)
    rowptr, col, val = assemble_velocity(mesh, "laplace")
    f = np.zeros((mesh.n_nodes, 3))
    dverts = []
    for ax, side in _all_faces():
        faces = boundary_faces(mesh, ax, side)
        if (ax, side) in dirichlet_faces:
            dverts.append(np.unique(faces))
            continue
        nrm = _face_normal(ax, side)
        gv = np.einsum("kci,i->kc", grad(mesh.coords[faces.ravel()]), nrm).reshape(-1, 3, 3)
        f += face_load(mesh, faces, face_edges(mesh, faces), gv)
    tags = node_tags(mesh, np.concatenate(dverts) if dverts else np.zeros(0, np.int64))
    exact = hierarchical_interpolant(mesh, u)
    prob = Problem(f"vector_laplace_n{n}_s{seed}", "laplace", mesh, rowptr, col, val, tags,
                   f, exact.copy(), exact_u=exact, params={"n": n, "seed": seed})
    return eliminate_dirichlet(prob)


def paper_setting_problem(kind: str, n: int) -> Problem:
    """The test problem of the paper's Sec. 4.1 for the vector Laplacian,
    pure-displacement elasticity and (Sec. 4.4) mixed elasticity: unit cube of n^3
    cubes, u = (0, 0, 0) on z = 0, u = (0, 0, 1) on z = 1, zero Neumann data on the
    other faces, no body force; elasticity with mu = 1.15e6, lambda = 1.73e6 (mixed
    form: c(p, q) = (1/lambda) int p q, Taylor-Hood P2/P1).  For the vector
    Laplacian the exact solution (0, 0, z) lies in the P2 space."""
    mesh = box_mesh(n)
    mu, lam = 1.15e6, 1.73e6
    saddle = None
    if kind == "laplace":
        rowptr, col, val = assemble_velocity(mesh, "laplace")
    elif kind == "elasticity":
        rowptr, col, val = assemble_velocity(mesh, "elasticity", mu=mu, lam=lam)
    elif kind == "mixed":
        (rowptr, col, val), bpart, cpart = _saddle_parts(mesh, "mixed", mu, lam)
        saddle = (*bpart, *cpart, np.zeros(mesh.n_vertices))
    else:
        raise ValueError(kind)
    bottom = boundary_faces(mesh, 2, 0)
    top = boundary_faces(mesh, 2, 1)
    tags = node_tags(mesh, np.unique(np.concatenate([bottom.ravel(), top.ravel()])))
    lift = np.zeros((mesh.n_nodes, 3))
    top_v = np.unique(top.ravel())
    lift[top_v, 2] = 1.0          # vertex coefficients; edge coefficients of linear data are 0
    exact = hierarchical_interpolant(mesh, lambda x: np.stack(
        [np.zeros(len(x)), np.zeros(len(x)), x[:, 2]], axis=1)) if kind == "laplace" else None
    f = np.zeros((mesh.n_nodes, 3))
    params = {"n": n, "setting": "Sec. 4.1"}
    if saddle is None:
        prob = Problem(f"paper_{kind}_n{n}", kind, mesh, rowptr, col, val, tags, f, lift,
                       exact_u=exact, params=params)
    else:
        prob = Problem(f"paper_{kind}_n{n}", kind, mesh, rowptr, col, val, tags, f, lift,
                       *saddle, params={**params, "lam": lam, "mu": mu})
    return eliminate_dirichlet(prob)


# ----------------------------------------------------------------------------------------
# linear elasticity, pure displacement (Eq. (elasdis))
# ----------------------------------------------------------------------------------------

def elasticity_problem(n, seed: int = 0, E: float = 1.0, nu: float = 0.3,
                       lengths=(1.0, 1.0, 1.0), n_rhs: int = 1, traction: str = "uniform",
                       jitter: float = 0.0) -> Problem:
    """Clamped at z=0, seeded traction on z=1, zero traction elsewhere.

    traction='uniform': one constant vector per top triangle from U[-1,1]^3;
    traction='gaussian': N(0,1) per top triangle.  n_rhs > 1 draws that many
    independent loads in sequence (f then has shape (n_rhs, N, 3)).
    `n` may be an int or an (nx, ny, nz) triple.
    """
    rng = np.random.default_rng(seed)
    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    mesh = box_mesh(nx, ny, nz, lengths=lengths, jitter=jitter, rng=rng if jitter else None)
    lam, mu = lame(E, nu)
    rowptr, col, val = assemble_velocity(mesh, "elasticity", mu=mu, lam=lam)
    bottom = boundary_faces(mesh, 2, 0)
    top = boundary_faces(mesh, 2, 1)
    tedges = face_edges(mesh, top)
    loads = []
    for _ in range(n_rhs):
        if traction == "uniform":
            t = rng.uniform(-1.0, 1.0, size=(len(top), 3))
        else:
            t = rng.standard_normal((len(top), 3))
        loads.append(face_load(mesh, top, tedges, np.repeat(t[:, None, :], 3, axis=1)))
    tags = node_tags(mesh, np.unique(bottom))
    zero = np.zeros((mesh.n_nodes, 3))
    prob = Problem(f"elasticity_n{nx}x{ny}x{nz}_s{seed}", "elasticity", mesh, rowptr, col, val,
                   tags, loads[0], zero,
                   params={"n": (nx, ny, nz), "seed": seed, "E": E, "nu": nu, "lam": lam,
                           "mu": mu, "lengths": tuple(lengths)})
    prob = eliminate_dirichlet(prob)
    if n_rhs > 1:
        dmask = (prob.tags & TAG_DIRICHLET) != 0
        F = np.stack(loads)
        F[:, dmask] = 0.0
        prob.f = F
    return prob


def elasticity_quadratic(rng: np.random.Generator, lam: float, mu: float):
    """A random quadratic displacement with div sigma(u) = 0 (no body force).

    u_c = a_c + b_c.x + x^T H_c x / 2.  For quadratic u, div sigma =
    mu Lap u + (lam+mu) grad div u is the constant vector with entries
    mu tr(H_d) + (lam+mu) sum_c (H_c)_{cd}; (H_d)_{dd} is solved so it vanishes.
    """
    a = rng.standard_normal(3)
    b = rng.standard_normal((3, 3))
    H = rng.standard_normal((3, 3, 3))
    H = 0.5 * (H + np.transpose(H, (0, 2, 1)))
    for d in range(3):
        rest = mu * (np.trace(H[d]) - H[d, d, d]) + (lam + mu) * (
            sum(H[c, c, d] for c in range(3) if c != d))
        H[d, d, d] = -rest / (lam + 2 * mu)

    def u(x):
        return a[None, :] + x @ b.T + 0.5 * np.einsum("ki,cij,kj->kc", x, H, x)

    def grad(x):    # (K, c, i) = d u_c / d x_i
        return b[None, :, :] + np.einsum("cij,kj->kci", H, x)

    def stress(x):
        Gr = grad(x)
        eps = 0.5 * (Gr + np.transpose(Gr, (0, 2, 1)))
        div = np.trace(Gr, axis1=1, axis2=2)
        return 2 * mu * eps + lam * div[:, None, None] * np.eye(3)

    return u, stress


def elasticity_quadratic_problem(n: int, seed: int = 0, E: float = 1.0, nu: float = 0.3,
                                 jitter: float = 0.0) -> Problem:
    """Elasticity with a body-force-free quadratic exact solution: Dirichlet data
    on z=0, traction sigma(u) n on the other faces."""
    rng = np.random.default_rng(seed)
    mesh = box_mesh(n, jitter=jitter, rng=rng if jitter else None)
    lam, mu = lame(E, nu)
    u, stress = elasticity_quadratic(rng, lam, mu)
    rowptr, col, val = assemble_velocity(mesh, "elasticity", mu=mu, lam=lam)
    f = np.zeros((mesh.n_nodes, 3))
    for ax, side in _all_faces():
        faces = boundary_faces(mesh, ax, side)
        if (ax, side) == (2, 0):
            dverts = np.unique(faces)
            continue
        nrm = _face_normal(ax, side)
        gv = np.einsum("kij,j->ki", stress(mesh.coords[faces.ravel()]), nrm).reshape(-1, 3, 3)
        f += face_load(mesh, faces, face_edges(mesh, faces), gv)
    tags = node_tags(mesh, dverts)
    exact = hierarchical_interpolant(mesh, u)
    prob = Problem(f"elasticity_quadratic_n{n}_s{seed}", "elasticity", mesh, rowptr, col, val,
                   tags, f, exact.copy(), exact_u=exact,
                   params={"n": n, "seed": seed, "lam": lam, "mu": mu})
    return eliminate_dirichlet(prob)


def unconstrained_elasticity(n: int, E: float = 1.0, nu: float = 0.3, jitter: float = 0.0,
                             seed: int = 0):
    """The elasticity stiffness matrix with no boundary condition (for null-space checks)."""
    rng = np.random.default_rng(seed)
    mesh = box_mesh(n, jitter=jitter, rng=rng if jitter else None)
    lam, mu = lame(E, nu)
    return mesh, assemble_velocity(mesh, "elasticity", mu=mu, lam=lam)


def rigid_body_modes(mesh: BoxMesh) -> np.ndarray:
    """(6, NV+NE, 3): 3 translations and 3 rotations w x x as hierarchical P2
    coefficients (linear fields have zero edge coefficients)."""
    modes = np.zeros((6, mesh.n_nodes, 3))
    for d in range(3):
        modes[d, :mesh.n_vertices, d] = 1.0
    x = mesh.coords
    for r in range(3):
        w = np.zeros(3)
        w[r] = 1.0
        modes[3 + r, :mesh.n_vertices] = np.cross(w[None, :], x)
    return modes


# ----------------------------------------------------------------------------------------
# mixed forms (Eqs. (elasmix), (stokesmix)) with Taylor-Hood P2/P1
# ----------------------------------------------------------------------------------------

def _saddle_parts(mesh: BoxMesh, kind: str, mu: float, lam: float | None):
    rowptr, col, val = assemble_velocity(mesh, kind, mu=mu)
    brp, bc, bv = assemble_divergence(mesh)
    scale = 0.0 if kind == "stokes" else 1.0 / lam
    crp, cc, cv = assemble_pressure_mass(mesh, scale)
    return (rowptr, col, val), (brp, bc, bv), (crp, cc, cv)


def pressure_weights(mesh: BoxMesh) -> np.ndarray:
    """w_i = int phi_i dx of the P1 hats: row sums of the P1 mass matrix."""
    rp, _, cv = assemble_pressure_mass(mesh, 1.0)
    return np.bincount(np.repeat(np.arange(mesh.n_vertices), np.diff(rp)), weights=cv,
                       minlength=mesh.n_vertices)


def stokes_lid_problem(n: int, mu: float = 1.0) -> Problem:
    """Lid-driven cavity: u = (1,0,0) on every node with z = 1, u = 0 on the rest of
    the boundary, c = 0; the pressure is fixed up to a constant (mean zero)."""
    mesh = box_mesh(n)
    (rp, c, v), (brp, bc, bv), (crp, cc, cv) = _saddle_parts(mesh, "stokes", mu, None)
    bnd = np.unique(np.concatenate([boundary_faces(mesh, ax, s) for ax, s in _all_faces()]))
    tags = node_tags(mesh, bnd)

    def lid(x):
        out = np.zeros((len(x), 3))
        out[np.isclose(x[:, 2], 1.0), 0] = 1.0
        return out

    liftv = hierarchical_interpolant(mesh, lid)
    prob = Problem(f"stokes_lid_n{n}", "stokes", mesh, rp, c, v, tags,
                   np.zeros((mesh.n_nodes, 3)), liftv, brp, bc, bv, crp, cc, cv,
                   np.zeros(mesh.n_vertices), p_weights=pressure_weights(mesh),
                   params={"n": n, "mu": mu})
    return eliminate_dirichlet(prob)


def mixed_elasticity_family(n: int, nus, seed: int = 0, E: float = 1.0, jitter: float = 0.2):
    """mixed_elasticity_problem for several nu on one mesh: a(u,v) scales with mu and
    c(p,q) with 1/lam, so the mesh, A (for mu = 1), B, the mass and the loads are
    assembled once and scaled."""
    rng = np.random.default_rng(seed)
    mesh = box_mesh(n, jitter=jitter, rng=rng if jitter else None)
    rp, c, v1 = assemble_velocity(mesh, "mixed", mu=1.0)
    brp, bc, bv = assemble_divergence(mesh)
    crp, cc, m1 = assemble_pressure_mass(mesh, 1.0)
    top = boundary_faces(mesh, 2, 1)
    t = rng.uniform(-1.0, 1.0, size=(len(top), 3))
    f = face_load(mesh, top, face_edges(mesh, top), np.repeat(t[:, None, :], 3, axis=1))
    tags = node_tags(mesh, np.unique(boundary_faces(mesh, 2, 0)))
    out = []
    for nu in nus:
        lam, mu = lame(E, nu)
        prob = Problem(f"mixed_elasticity_n{n}_nu{nu}_s{seed}", "mixed", mesh, rp, c, v1 * mu,
                       tags.copy(), f.copy(), np.zeros((mesh.n_nodes, 3)), brp, bc, bv.copy(),
                       crp, cc, m1 / lam, np.zeros(mesh.n_vertices),
                       params={"n": n, "nu": nu, "seed": seed, "lam": lam, "mu": mu})
        out.append(eliminate_dirichlet(prob))
    return out


def mixed_elasticity_problem(n: int, nu: float = 0.49, seed: int = 0, E: float = 1.0,
                             jitter: float = 0.2) -> Problem:
    """Mixed displacement-pressure elasticity, c = (1/lam) int p q: clamped z=0,
    seeded uniform traction on z=1, vertices jittered by U[-jitter h, jitter h]."""
    rng = np.random.default_rng(seed)
    mesh = box_mesh(n, jitter=jitter, rng=rng if jitter else None)
    lam, mu = lame(E, nu)
    (rp, c, v), (brp, bc, bv), (crp, cc, cv) = _saddle_parts(mesh, "mixed", mu, lam)
    top = boundary_faces(mesh, 2, 1)
    t = rng.uniform(-1.0, 1.0, size=(len(top), 3))
    f = face_load(mesh, top, face_edges(mesh, top), np.repeat(t[:, None, :], 3, axis=1))
    tags = node_tags(mesh, np.unique(boundary_faces(mesh, 2, 0)))
    prob = Problem(f"mixed_elasticity_n{n}_nu{nu}_s{seed}", "mixed", mesh, rp, c, v, tags, f,
                   np.zeros((mesh.n_nodes, 3)), brp, bc, bv, crp, cc, cv,
                   np.zeros(mesh.n_vertices),
                   params={"n": n, "nu": nu, "seed": seed, "lam": lam, "mu": mu})
    return eliminate_dirichlet(prob)


def stokes_quadratic(rng: np.random.Generator, mu: float):
    """Divergence-free quadratic u = a + b x + x^T H x / 2 with the linear pressure
    p = mu sum_c tr(H_c) x_c that solves -mu Lap u + grad p = 0, div u = 0.

    div u = tr(b) + sum_c (H_c)_{c,:} . x, so tr(b) = 0 and sum_c (H_c)_{cj} = 0 for
    every j; each of the latter is solved for the entry (H_j)_{jj}.
    """
    a = rng.standard_normal(3)
    b = rng.standard_normal((3, 3))
    b[2, 2] = -(b[0, 0] + b[1, 1])
    H = rng.standard_normal((3, 3, 3))
    H = 0.5 * (H + np.transpose(H, (0, 2, 1)))
    # enforce sum_c H[c, c, j] = 0 for j = 0, 1, 2 by adjusting H[j, j, j]
    for j in range(3):
        H[j, j, j] = -sum(H[c, c, j] for c in range(3) if c != j)

    def u(x):
        return a[None, :] + x @ b.T + 0.5 * np.einsum("ki,cij,kj->kc", x, H, x)

    lap = np.array([np.trace(H[c]) for c in range(3)])

    def p(x):
        return mu * x @ lap

    return u, p


def stokes_quadratic_problem(n: int, seed: int = 0, mu: float = 1.0) -> Problem:
    """Stokes with an exact P2/P1 solution: Dirichlet data from a divergence-free
    quadratic u on the whole boundary; the pressure is linear (up to a constant)."""
    rng = np.random.default_rng(seed)
    mesh = box_mesh(n)
    u, pfun = stokes_quadratic(rng, mu)
    (rp, c, v), (brp, bc, bv), (crp, cc, cv) = _saddle_parts(mesh, "stokes", mu, None)
    bnd = np.unique(np.concatenate([boundary_faces(mesh, ax, s) for ax, s in _all_faces()]))
    tags = node_tags(mesh, bnd)
    exact = hierarchical_interpolant(mesh, u)
    prob = Problem(f"stokes_quadratic_n{n}_s{seed}", "stokes", mesh, rp, c, v, tags,
                   np.zeros((mesh.n_nodes, 3)), exact.copy(), brp, bc, bv, crp, cc, cv,
                   np.zeros(mesh.n_vertices), exact_u=exact, exact_p=pfun(mesh.coords),
                   p_weights=pressure_weights(mesh), params={"n": n, "seed": seed, "mu": mu})
    return eliminate_dirichlet(prob)


def mixed_quadratic_problem(n: int, seed: int = 0, E: float = 1.0, nu: float = 0.3,
                            jitter: float = 0.0) -> Problem:
    """Mixed elasticity with the body-force-free quadratic of `elasticity_quadratic`:
    p = -lam div u is linear, the traction (2 mu eps(u) - p I) n equals sigma(u) n."""
    rng = np.random.default_rng(seed)
    mesh = box_mesh(n, jitter=jitter, rng=rng if jitter else None)
    lam, mu = lame(E, nu)
    u, stress = elasticity_quadratic(rng, lam, mu)
    (rp, c, v), (brp, bc, bv), (crp, cc, cv) = _saddle_parts(mesh, "mixed", mu, lam)
    f = np.zeros((mesh.n_nodes, 3))
    for ax, side in _all_faces():
        faces = boundary_faces(mesh, ax, side)
        if (ax, side) == (2, 0):
            dverts = np.unique(faces)
            continue
        nrm = _face_normal(ax, side)
        gv = np.einsum("kij,j->ki", stress(mesh.coords[faces.ravel()]), nrm).reshape(-1, 3, 3)
        f += face_load(mesh, faces, face_edges(mesh, faces), gv)
    tags = node_tags(mesh, dverts)
    exact = hierarchical_interpolant(mesh, u)
    # p = -lam div u, and trace sigma = (2 mu + 3 lam) div u
    pe = -lam * np.trace(stress(mesh.coords), axis1=1, axis2=2) / (2 * mu + 3 * lam)
    prob = Problem(f"mixed_quadratic_n{n}_s{seed}", "mixed", mesh, rp, c, v, tags, f,
                   exact.copy(), brp, bc, bv, crp, cc, cv, np.zeros(mesh.n_vertices),
                   exact_u=exact, exact_p=pe, params={"n": n, "seed": seed, "lam": lam, "mu": mu})
    return eliminate_dirichlet(prob)
