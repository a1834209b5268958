"""Plain FP64 CPU oracle of the graph-based AMG of Sec. 3 (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use
this module.  It shares no code with the CUDA library and is written to be read
against the paper, not to be fast:

  coarsening graphs   Sec. 3.2.1: separate graphs of K_ll (vertex nodes) and
                      K_qq (edge nodes); K_ql ignored.  Sec. 3.2.2: the pressure
                      graph is the P1 pattern.  Optional "non-separating" mode
                      uses the graph of the whole matrix (Table 2, row 3).
  C/F selection       the greedy maximal independent set in increasing node
                      index (the reading of the FK98 selection cited in Sec. 3.2.1).
  prolongation        Eqs. (disprolongmat), (mixprolongmat): per node, C -> 1 on
                      itself, F -> 1/k on each of its k C-neighbours, the same
                      weight on all 3 components; R = P^T.
  Galerkin            A_{l+1} = P^T A_l P (Sec. 3.2.1/3.2.2), pattern kept
                      structurally (entries that cancel numerically stay).
  smoothers           Sec. 3.3: damped 3x3-block Jacobi, multicolour 3x3-block
                      Gauss-Seidel (first-fit colouring in index order).  The
                      post-smoothing sweeps run the colours in reverse order
                      inside a Krylov method (a symmetric preconditioner for CG)
                      and in the pre-smoothing order for the stand-alone AMG
                      iteration (Options.post_order).
  cycle               Algorithm 1 (nu = 1: V-cycle, nu = 2: W-cycle).
  Krylov              PCG, flexible CG, right-preconditioned FGMRES(m).

Dirichlet nodes (identity rows) are handled as follows: a coarse node inherits
the Dirichlet tag of its C node; P entries in rows of Dirichlet fine nodes and
in columns of Dirichlet coarse nodes are zero (the structure is kept); the
diagonal block of a Dirichlet coarse node is the identity.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

TAG_TYPE_MASK = 0x0F
TAG_VERTEX = 0
TAG_EDGE = 1
TAG_DIRICHLET = 0x10

STATE_UNDECIDED, STATE_C, STATE_F = 0, 1, 2


# ----------------------------------------------------------------------------------------
# graphs, C/F splitting, colouring
# ----------------------------------------------------------------------------------------

def block_pattern(rowptr: np.ndarray, col: np.ndarray, n: int) -> sp.csr_matrix:
    """0/1 node graph (with self loops) of a block-sparse matrix's structure."""
    data = np.ones(len(col), dtype=np.float64)
    return sp.csr_matrix((data, np.asarray(col), np.asarray(rowptr)), shape=(n, n))


def coarsening_graph(pattern: sp.csr_matrix, node_type: np.ndarray, separate: bool = True):
    """Adjacency lists used for the C/F split (self loops removed).

    separate=True keeps only edges between nodes of the same type (vertex-vertex:
    graph of K_ll; edge-edge: graph of K_qq); separate=False keeps the whole graph.
    """
    coo = pattern.tocoo()
    keep = coo.row != coo.col
    if separate:
        keep &= node_type[coo.row] == node_type[coo.col]
    g = sp.csr_matrix((np.ones(int(keep.sum())), (coo.row[keep], coo.col[keep])),
                      shape=pattern.shape)
    g.sort_indices()
    return g


def greedy_mis(graph: sp.csr_matrix) -> np.ndarray:
    """Sequential greedy maximal independent set, visiting nodes in increasing index:
    an undecided node becomes C and its undecided neighbours become F."""
    n = graph.shape[0]
    state = np.zeros(n, dtype=np.int8)
    indptr, indices = graph.indptr, graph.indices
    for i in range(n):
        if state[i] != STATE_UNDECIDED:
            continue
        state[i] = STATE_C
        nb = indices[indptr[i]:indptr[i + 1]]
        und = nb[state[nb] == STATE_UNDECIDED]
        state[und] = STATE_F
    return state


def greedy_colouring(pattern: sp.csr_matrix) -> np.ndarray:
    """First-fit colouring in increasing node index: each node takes the smallest
    colour not used by an already coloured (lower-index) neighbour."""
    n = pattern.shape[0]
    colour = np.full(n, -1, dtype=np.int32)
    indptr, indices = pattern.indptr, pattern.indices
    for i in range(n):
        nb = indices[indptr[i]:indptr[i + 1]]
        used = set(colour[nb].tolist())
        c = 0
        while c in used:
            c += 1
        colour[i] = c
    return colour


def build_prolongation(graph: sp.csr_matrix, state: np.ndarray, dirichlet: np.ndarray):
    """Per-node prolongation of Eq. (disprolongmat).

    Returns (P_structure, P_values, coarse_of_fine): P_structure is the 0/1 pattern
    (n_fine x n_coarse), P_values the weights with Dirichlet rows/columns zeroed.
    Coarse ids are the C nodes in increasing fine index.
    """
    n = graph.shape[0]
    is_c = state == STATE_C
    cid = np.full(n, -1, dtype=np.int64)
    cid[is_c] = np.arange(int(is_c.sum()))
    nc = int(is_c.sum())
    rows, cols, vals = [], [], []
    indptr, indices = graph.indptr, graph.indices
    for i in range(n):
        if is_c[i]:
            rows.append(i)
            cols.append(cid[i])
            vals.append(1.0)
            continue
        nb = indices[indptr[i]:indptr[i + 1]]
        cn = nb[is_c[nb]]
        k = len(cn)
        assert k >= 1, "F node without a C neighbour (the independent set is not maximal)"
        w = 1.0 / k
        for j in cn:
            rows.append(i)
            cols.append(cid[j])
            vals.append(w)
    rows = np.array(rows)
    cols = np.array(cols)
    vals = np.array(vals)
    structure = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, nc))
    cdir = np.zeros(nc, dtype=bool)
    cdir[cid[is_c]] = dirichlet[is_c]
    zero = dirichlet[rows] | cdir[cols]
    vals = np.where(zero, 0.0, vals)
    values = sp.csr_matrix((vals, (rows, cols)), shape=(n, nc))
    return structure, values, cid


# ----------------------------------------------------------------------------------------
# levels
# ----------------------------------------------------------------------------------------

@dataclass
class Level:
    n: int                          # number of 3-component nodes
    rowptr: np.ndarray              # block structure of A_l
    col: np.ndarray
    val: np.ndarray                 # (nnzb, 3, 3)
    tags: np.ndarray                # int32 node tags (type | Dirichlet bit)
    A: sp.csr_matrix = None         # scalar CSR view of A_l (3n x 3n)
    dinv: np.ndarray = None         # (n, 3, 3) inverses of the diagonal blocks
    colour: np.ndarray = None
    colour_rows: list = None        # per colour: node ids
    colour_A: list = None           # per colour: rows of A (scalar CSR)
    state: np.ndarray = None        # C/F state used to build the next level
    P: sp.csr_matrix = None         # node-level weights (n x n_coarse)
    P_structure: sp.csr_matrix = None
    Pk: sp.csr_matrix = None        # kron(P, I3)
    coarse_of_fine: np.ndarray = None
    # saddle parts (pressure block)
    npres: int = 0
    B: sp.csr_matrix = None         # (npres x 3n)
    C: sp.csr_matrix = None         # (npres x npres)
    c_pattern: sp.csr_matrix = None
    H: sp.csr_matrix = None
    H_structure: sp.csr_matrix = None
    p_state: np.ndarray = None
    extra: dict = field(default_factory=dict)


def scalar_view(rowptr, col, val, n):
    return sp.bsr_matrix((val, col, rowptr), shape=(3 * n, 3 * n)).tocsr()


def diag_block_inverses(rowptr, col, val, n):
    out = np.empty((n, 3, 3))
    for i in range(n):
        seg = slice(rowptr[i], rowptr[i + 1])
        k = np.nonzero(col[seg] == i)[0]
        assert len(k) == 1, "missing diagonal block"
        out[i] = np.linalg.inv(val[rowptr[i] + k[0]])
    return out


def galerkin_blocks(level: Level, P_val: sp.csr_matrix, P_struct: sp.csr_matrix):
    """K_{l+1} = P^T K_l P on the structural pattern P_s^T pattern(K_l) P_s."""
    nc = P_val.shape[1]
    pat = block_pattern(level.rowptr, level.col, level.n)
    cpat = (P_struct.T @ pat @ P_struct).tocsr()
    cpat.sort_indices()
    Pk = sp.kron(P_val, sp.identity(3), format="csr")
    Ac = (Pk.T @ level.A @ Pk).tocoo()
    crow = np.asarray(cpat.indptr, dtype=np.int64)
    ccol = np.asarray(cpat.indices, dtype=np.int64)
    val = np.zeros((len(ccol), 3, 3))
    bi, bj = Ac.row // 3, Ac.col // 3
    keys = np.repeat(np.arange(nc), np.diff(crow)) * nc + ccol
    pos = np.searchsorted(keys, bi * nc + bj)
    assert np.all(keys[pos] == bi * nc + bj), "numeric entry outside the symbolic pattern"
    val[pos, Ac.row % 3, Ac.col % 3] = Ac.data
    return crow.astype(np.int32), ccol.astype(np.int32), val, Pk


@dataclass
class Options:
    smoother: str = "gs"            # gs | jacobi (SPD); sgs | bs (saddle)
    m_pre: int = 1
    m_post: int = 1
    omega: float = 0.5              # block Jacobi damping
    nu: int = 1                     # 1: V-cycle, 2: W-cycle
    cycles: int = 1                 # cycles per preconditioner application
    max_levels: int = 5
    coarse_dofs: int = 300
    separate: bool = True           # separated (new) vs non-separating graph
    omega_p: float = 0.125          # sGS pressure step
    # learned multipliers (1: the plain method): relaxation, coarse-grid
    # correction scale, sGS pressure step; level_weights, if given, holds one
    # (ws, wc, wp) per level and overrides the three
    ws: float = 1.0
    wc: float = 1.0
    wp: float = 1.0
    level_weights: list = None
    # colour order of the post-smoothing sweeps (Gauss-Seidel, Vanka): "reverse"
    # (descending: with the ascending pre-smoothing the cycle is a symmetric
    # preconditioner, as CG needs) or "same" (ascending, as pre-smoothing: the
    # stand-alone AMG iteration of Sec. 4.2, Tables 4 and 8)
    post_order: str = "reverse"


@dataclass
class Hierarchy:
    levels: list
    opts: Options
    coarse_factor: object = None
    saddle: bool = False
    kind: str = "elasticity"

    @property
    def L(self) -> int:
        return len(self.levels) - 1


def _finish_level(lv: Level, colour_needed: bool = True):
    lv.dinv = diag_block_inverses(lv.rowptr, lv.col, lv.val, lv.n)
    if colour_needed:
        lv.colour = greedy_colouring(block_pattern(lv.rowptr, lv.col, lv.n))
        lv.colour_rows = [np.nonzero(lv.colour == c)[0] for c in range(lv.colour.max() + 1)]
        lv.colour_A = []
        for rows in lv.colour_rows:
            sidx = (3 * rows[:, None] + np.arange(3)).ravel()
            lv.colour_A.append(lv.A[sidx])


def coarsen_level(lv: Level, opts: Options) -> Level:
    """Graph -> C/F split -> P -> Galerkin for one SPD (velocity) level."""
    pat = block_pattern(lv.rowptr, lv.col, lv.n)
    ntype = lv.tags & TAG_TYPE_MASK
    dirichlet = (lv.tags & TAG_DIRICHLET) != 0
    g = coarsening_graph(pat, ntype, opts.separate)
    lv.state = greedy_mis(g)
    lv.P_structure, lv.P, lv.coarse_of_fine = build_prolongation(g, lv.state, dirichlet)
    crow, ccol, cval, lv.Pk = galerkin_blocks(lv, lv.P, lv.P_structure)
    is_c = lv.state == STATE_C
    ctags = lv.tags[is_c].astype(np.int32)
    nc = int(is_c.sum())
    cdir = (ctags & TAG_DIRICHLET) != 0
    rows = np.repeat(np.arange(nc), np.diff(crow))
    diag = (rows == ccol) & cdir[rows]
    cval[diag] = np.eye(3)
    nxt = Level(nc, crow, ccol, cval, ctags)
    nxt.A = scalar_view(crow, ccol, cval, nc)
    return nxt


def level_dofs(lv: Level) -> int:
    return 3 * lv.n + lv.npres


def build_hierarchy(prob, opts: Options | None = None) -> Hierarchy:
    """AMG setup for an SPD problem (Sec. 3.2.1) or a saddle problem (Sec. 3.2.2)."""
    saddle = prob.kind in ("mixed", "stokes")
    opts = opts or Options(smoother="sgs" if saddle else "gs")
    lv = Level(prob.n_nodes, np.asarray(prob.a_rowptr), np.asarray(prob.a_col),
               np.array(prob.a_val, dtype=np.float64), np.asarray(prob.tags, dtype=np.int32))
    lv.A = scalar_view(lv.rowptr, lv.col, lv.val, lv.n)
    if saddle:
        from . import saddle as sd
        sd.attach_pressure(lv, prob)
    levels = [lv]
    while (level_dofs(levels[-1]) > opts.coarse_dofs and len(levels) < opts.max_levels):
        cur = levels[-1]
        nxt = coarsen_level(cur, opts)
        if saddle:
            sd.coarsen_pressure(cur, nxt)
        if nxt.n == cur.n:
            break
        levels.append(nxt)
    h = Hierarchy(levels, opts, saddle=saddle, kind=prob.kind)
    for i, lv in enumerate(levels):
        last = i == len(levels) - 1
        _finish_level(lv, colour_needed=not last and not saddle)
        if saddle:
            sd.finish_saddle_level(lv, h, last)
    if saddle:
        h.coarse_factor = sd.factor_coarsest(h)
        if opts.smoother == "bs":
            sd.bs_setup(h)
        if opts.smoother == "vanka":
            sd.vanka_setup(h)
    else:
        h.coarse_factor = ("cplu", complete_pivot_lu(levels[-1].A.toarray()))
    return h


# ----------------------------------------------------------------------------------------
# coarsest level (Algorithm 1, step 6: "any direct solver")
# ----------------------------------------------------------------------------------------

PIVOT_RTOL = 1e-13
PIVOT_TIE = 1e-9


def complete_pivot_lu(K: np.ndarray, rtol: float = PIVOT_RTOL, tie: float = PIVOT_TIE):
    """Gaussian elimination with complete pivoting, stopped at the numerical rank.

    Step k takes the largest magnitude M of the remaining block; the pivot is the
    first entry in row-major order of that block whose magnitude is >= (1 - tie) M
    (entries within a relative `tie` of the largest count as equal, so that
    rounding differences in the matrix do not change the pivot sequence of
    matrices with exactly tied entries, such as the Galerkin coarse matrices of a
    structured mesh); it is swapped to (k, k) and eliminated below.  Elimination
    stops when M <= rtol * max|K|; the unknowns of the remaining columns are then
    set to zero, which gives one solution of a consistent singular system (e.g. a
    Stokes matrix with its constant-pressure mode) and the exact solution of a
    nonsingular one.
    Returns (LU, row_perm, col_perm, rank).
    """
    A = np.array(K, dtype=np.float64)
    n = A.shape[0]
    rp = np.arange(n)
    cp = np.arange(n)
    scale = np.abs(A).max() if n else 0.0
    rank = 0
    for k in range(n):
        sub = np.abs(A[k:, k:])
        big = sub.max()
        if big <= rtol * scale:
            break
        flat = int(np.argmax(sub.ravel() >= (1.0 - tie) * big))
        i, j = divmod(flat, n - k)
        i += k
        j += k
        A[[k, i], :] = A[[i, k], :]
        rp[[k, i]] = rp[[i, k]]
        A[:, [k, j]] = A[:, [j, k]]
        cp[[k, j]] = cp[[j, k]]
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
        rank = k + 1
    return A, rp, cp, rank


def complete_pivot_solve(fac, b):
    LU, rp, cp, r = fac
    y = b[rp].astype(np.float64)
    for k in range(r):                       # forward substitution with unit L
        y[k + 1:] -= LU[k + 1:, k] * y[k]
    z = np.zeros_like(y)
    for k in range(r - 1, -1, -1):           # back substitution on the leading r x r U
        z[k] = (y[k] - LU[k, k + 1:r] @ z[k + 1:r]) / LU[k, k]
    x = np.zeros_like(z)
    x[cp] = z
    return x


# ----------------------------------------------------------------------------------------
# smoothers (Sec. 3.3) and the cycle (Algorithm 1)
# ----------------------------------------------------------------------------------------

def apply_dinv(dinv: np.ndarray, r: np.ndarray) -> np.ndarray:
    return np.einsum("nij,nj->ni", dinv, r.reshape(-1, 3)).ravel()


def jacobi_sweep(lv: Level, x, b, omega):
    """x <- x + omega D^{-1} (b - A x), D = 3x3 nodal diagonal blocks."""
    return x + omega * apply_dinv(lv.dinv, b - lv.A @ x)


def gs_sweep(lv: Level, x, b, reverse: bool = False, ws: float = 1.0):
    """Multicolour block Gauss-Seidel: per colour, every row of that colour is
    updated from the values at the start of the colour,
    x_i <- x_i + ws D_i^{-1} (b_i - sum_j A_ij x_j)  (ws = 1: Gauss-Seidel; other
    values: symmetric over-/under-relaxation with the same colour order)."""
    x = x.copy()
    order = range(len(lv.colour_rows))
    if reverse:
        order = reversed(order)
    for c in order:
        rows = lv.colour_rows[c]
        sidx = (3 * rows[:, None] + np.arange(3)).ravel()
        r = b[sidx] - lv.colour_A[c] @ x
        x[sidx] += ws * apply_dinv(lv.dinv[rows], r)
    return x


def level_multipliers(o: Options, l: int):
    """(ws, wc, wp) of level l: the per-level row if given, else the three globals."""
    if o.level_weights is not None and l < len(o.level_weights):
        ws, wc, wp = o.level_weights[l]
        return float(ws), float(wc), float(wp)
    return o.ws, o.wc, o.wp


def smooth(h: Hierarchy, l: int, x, b, post: bool):
    lv = h.levels[l]
    o = h.opts
    if h.saddle:
        from . import saddle as sd
        return sd.smooth(h, l, x, b, post)
    ws = level_multipliers(o, l)[0]
    if o.smoother == "jacobi":
        return jacobi_sweep(lv, x, b, o.omega * ws)
    return gs_sweep(lv, x, b, reverse=post and o.post_order == "reverse", ws=ws)


def operator(h: Hierarchy, l: int):
    if h.saddle:
        from . import saddle as sd
        return lambda v: sd.apply_K(h.levels[l], v)
    return lambda v: h.levels[l].A @ v


def restrict(h: Hierarchy, l: int, r):
    lv = h.levels[l]
    if h.saddle:
        from . import saddle as sd
        return sd.restrict(lv, r)
    return lv.Pk.T @ r


def prolong(h: Hierarchy, l: int, xc):
    lv = h.levels[l]
    if h.saddle:
        from . import saddle as sd
        return sd.prolong(lv, xc)
    return lv.Pk @ xc


def coarse_solve(h: Hierarchy, b):
    return complete_pivot_solve(h.coarse_factor[1], b)


def amg_cycle(h: Hierarchy, l: int, x, b):
    """Algorithm 1, AMG(K_l, x_l, b_l), with nu recursive calls."""
    o = h.opts
    if l == h.L:
        return coarse_solve(h, b)
    K = operator(h, l)
    for _ in range(o.m_pre):
        x = smooth(h, l, x, b, post=False)
    bc = restrict(h, l, b - K(x))
    if l + 1 == h.L:
        xc = coarse_solve(h, bc)
    else:
        xc = np.zeros_like(bc)
        for _ in range(o.nu):
            xc = amg_cycle(h, l + 1, xc, bc)
    x = x + level_multipliers(o, l)[1] * prolong(h, l, xc)
    for _ in range(o.m_post):
        x = smooth(h, l, x, b, post=True)
    return x


def precondition(h: Hierarchy, r):
    """M^{-1} r: `cycles` applications of Algorithm 1 from a zero initial guess."""
    z = np.zeros_like(r)
    for _ in range(h.opts.cycles):
        z = amg_cycle(h, 0, z, r)
    return z


# ----------------------------------------------------------------------------------------
# Krylov methods
# ----------------------------------------------------------------------------------------

@dataclass
class SolveResult:
    x: np.ndarray
    iterations: int
    converged: bool
    history: list
    true_rel_residual: float


def pcg(apply_A, apply_M, b, tol, maxit=1000, flexible=False):
    """Preconditioned CG from x0 = 0, stopping when ||b - A x_k|| / ||b|| <= tol.

    flexible=True uses the Polak-Ribiere form beta_k = <z_k, r_k - r_{k-1}> /
    <z_{k-1}, r_{k-1}> (flexible CG for a varying preconditioner)."""
    x = np.zeros_like(b)
    r = b.copy()
    nb = np.linalg.norm(b)
    hist = [1.0]
    if nb == 0.0:
        return SolveResult(x, 0, True, hist, 0.0)
    z = apply_M(r)
    p = z.copy()
    rz = r @ z
    it = 0
    conv = False
    while it < maxit:
        q = apply_A(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r_old = r
        r = r - alpha * q
        it += 1
        rel = np.linalg.norm(r) / nb
        hist.append(rel)
        if rel <= tol:
            conv = True
            break
        z_new = apply_M(r)
        if flexible:
            beta = (z_new @ (r - r_old)) / rz
        else:
            beta = (z_new @ r) / rz
        rz = z_new @ r
        p = z_new + beta * p
    true = np.linalg.norm(b - apply_A(x)) / nb
    return SolveResult(x, it, conv, hist, true)


def fgmres(apply_A, apply_M, b, tol, restart=50, maxit=1000, project=None):
    """Right-preconditioned flexible GMRES(m) (Saad 1993), modified Gram-Schmidt,
    x0 = 0, stopping when ||b - A x_k|| / ||b|| <= tol.  `project`, if given, is
    applied to every preconditioned vector (e.g. a pressure-mean projection)."""
    n = len(b)
    x = np.zeros(n)
    nb = np.linalg.norm(b)
    hist = [1.0]
    if nb == 0.0:
        return SolveResult(x, 0, True, hist, 0.0)
    it = 0
    conv = False
    while it < maxit and not conv:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        Hm = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        j_used = 0
        for j in range(restart):
            z = apply_M(V[j])
            if project is not None:
                z = project(z)
            Z[j] = z
            w = apply_A(z)
            for i in range(j + 1):
                Hm[i, j] = w @ V[i]
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            if Hm[j + 1, j] != 0.0:
                V[j + 1] = w / Hm[j + 1, j]
            for i in range(j):
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            den = np.hypot(Hm[j, j], Hm[j + 1, j])
            cs[j] = Hm[j, j] / den
            sn[j] = Hm[j + 1, j] / den
            Hm[j, j] = den
            Hm[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_used = j + 1
            rel = abs(g[j + 1]) / nb
            hist.append(rel)
            if rel <= tol or it >= maxit:
                conv = rel <= tol
                break
        y = sla.solve_triangular(Hm[:j_used, :j_used], g[:j_used])
        x = x + Z[:j_used].T @ y
    true = np.linalg.norm(b - apply_A(x)) / nb
    return SolveResult(x, it, conv and true <= tol * 10, hist, true)


def solve(prob, opts: Options | None = None, tol: float = 1e-8, h: Hierarchy | None = None,
          method: str | None = None, maxit: int = 1000):
    """AMG-preconditioned Krylov solve of the homogenised system, x0 = 0."""
    h = h or build_hierarchy(prob, opts)
    b = prob.rhs()
    if h.saddle:
        from . import saddle as sd
        return sd.solve(h, prob, b, tol, maxit, method), h
    K = operator(h, 0)
    M = lambda r: precondition(h, r)   # noqa: E731
    if method == "amg":
        return amg_iteration(K, M, b, tol, maxit=maxit), h
    flexible = method == "fcg"
    return pcg(K, M, b, tol, maxit=maxit, flexible=flexible), h


def amg_iteration(apply_A, apply_M, b, tol, maxit=1000):
    """The stand-alone AMG solver (Sec. 4.2): x_{k+1} = x_k + M^{-1}(b - A x_k) from
    x_0 = 0, one preconditioner application (`cycles` cycles of Algorithm 1) per
    iteration, stopping when ||b - A x_k|| / ||b|| <= tol."""
    x = np.zeros_like(b)
    nb = np.linalg.norm(b)
    hist = [1.0]
    if nb == 0.0:
        return SolveResult(x, 0, True, hist, 0.0)
    r = b.copy()
    it = 0
    while it < maxit:
        x = x + apply_M(r)
        r = b - apply_A(x)
        it += 1
        hist.append(np.linalg.norm(r) / nb)
        if hist[-1] <= tol:
            return SolveResult(x, it, True, hist, hist[-1])
    return SolveResult(x, it, False, hist, hist[-1])
