"""Saddle-point parts of the CPU oracle (TEST INFRASTRUCTURE ONLY).

System of Eq. (mixedeqn): K = [A B^T; B -C], unknowns [u; p].
  coarsening   Sec. 3.2.2: velocity as in the SPD case, pressure on the
               conventional P1 graph; P = diag(I, J, H) (Eq. (mixprolongmat)),
               K_{l+1} = P^T K_l P, i.e. A_{l+1} = Pu^T A Pu,
               B_{l+1} = H^T B Pu, C_{l+1} = H^T C H.
  smoother     segregated Gauss-Seidel, Eq. (uzsm) with K^ = [M_A 0; B -1/omega S_D]
               and M_A = damped block Jacobi (0.5), omega = 0.125 (Sec. 4.4):
                   u <- u + M_A^{-1} (f - A u - B^T p)
                   p <- p + omega S_D^{-1} (B u - C p - g)
               The identity of Eq. (uzsm) is read as S_D = diag(C + B M_A^{-1} B^T)
               (M_A = 2 D, D the 3x3-block diagonal of A) so that omega is
               independent of the scaling of the equations.
  smoother     Braess-Sarazin type, Eqs. (bssm) / (bssmpre) (Options.smoother = "bs"):
               one step is x += K^{-1} (b - K x) with
                   K^ = [A^  B^T; B  B A^{-1} B^T - S^],  A^ = 2 diag(A) (scalar diagonal)
               and S^{-1} one V(1,1)-cycle of the graph AMG on the scalar matrix
               S = C + B A^{-1} B^T (the "C + B A^{-1} B" of Sec. 3.3.2 read with the
               transpose): coarsened on the P1 graph, i.e. through the same pressure
               prolongations H as the saddle hierarchy, S_{k+1} = H^T S_k H, damped
               scalar Jacobi (0.5) as its smoother and a direct solve on the coarsest
               pressure level.  Solving K^ [du; dp] = [r_u; r_p] gives
                   w = A^{-1} r_u,  dp = S^{-1} (B w - r_p),  du = w - A^{-1} B^T dp.
  coarsest     the same rank-revealing complete-pivoting LU as the SPD case
               (see amg.complete_pivot_lu); it also covers the singular Galerkin
               Stokes matrices (constant pressure and other coarse null modes).
  Krylov       right-preconditioned FGMRES; for Stokes every preconditioned vector
               and the result are projected to int p dx = 0 (weights int phi_i).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import amg


def attach_pressure(lv, prob):
    n = prob.n_nodes
    npres = prob.n_pres
    b = sp.bsr_matrix((prob.b_val.reshape(-1, 1, 3), prob.b_col, prob.b_rowptr),
                      shape=(npres, 3 * n)).tocsr()
    c = sp.csr_matrix((prob.c_val, prob.c_col, prob.c_rowptr), shape=(npres, npres))
    lv.npres = npres
    lv.B = b
    lv.C = c
    lv.c_pattern = amg.block_pattern(prob.c_rowptr, prob.c_col, npres)
    # structural node pattern of B (pressure rows x velocity nodes)
    lv.extra["b_pattern"] = sp.csr_matrix(
        (np.ones(len(prob.b_col)), prob.b_col, prob.b_rowptr), shape=(npres, n))
    lv.extra["stokes"] = prob.kind == "stokes"
    # Stokes: pressure normalisation weights w_i = int phi_i (problem data)
    lv.extra["pmass"] = prob.p_weights if prob.kind == "stokes" else None


def coarsen_pressure(cur, nxt):
    """C/F split of the pressure P1 graph and Galerkin of B, C through H."""
    g = amg.coarsening_graph(cur.c_pattern, np.zeros(cur.npres, dtype=np.int32), True)
    cur.p_state = amg.greedy_mis(g)
    cur.H_structure, cur.H, _ = amg.build_prolongation(
        g, cur.p_state, np.zeros(cur.npres, dtype=bool))
    nxt.npres = cur.H.shape[1]
    nxt.B = (cur.H.T @ cur.B @ cur.Pk).tocsr()
    nxt.C = (cur.H.T @ cur.C @ cur.H).tocsr()
    cp = (cur.H_structure.T @ cur.c_pattern @ cur.H_structure).tocsr()
    cp.data[:] = 1.0
    cp.sort_indices()
    nxt.c_pattern = cp
    bp = (cur.H_structure.T @ cur.extra["b_pattern"] @ cur.P_structure).tocsr()
    bp.data[:] = 1.0
    bp.sort_indices()
    nxt.extra["b_pattern"] = bp
    nxt.extra["stokes"] = cur.extra["stokes"]
    nxt.extra["pmass"] = None


def level_dofs(lv) -> int:
    return 3 * lv.n + lv.npres


def schur_diagonal(lv, omega):
    """S_D[k] = C_kk + sum_j B_kj (D_j / omega)^{-1} B_kj^T over the velocity nodes j of
    pressure row k (M_A = D / omega is the damped block Jacobi matrix)."""
    B = lv.B.tocsr()
    out = np.array(lv.C.diagonal(), dtype=np.float64)
    for k in range(lv.npres):
        cols = B.indices[B.indptr[k]:B.indptr[k + 1]]
        vals = B.data[B.indptr[k]:B.indptr[k + 1]]
        blocks = {}
        for c, v in zip(cols, vals):
            blocks.setdefault(c // 3, np.zeros(3))[c % 3] += v
        for node, bv in blocks.items():
            out[k] += omega * (bv @ lv.dinv[node] @ bv)
    return out


def finish_saddle_level(lv, h, last):
    if not last:
        lv.extra["schur_diag"] = schur_diagonal(lv, h.opts.omega)


BS_JACOBI = 0.5     # damping of the scalar Jacobi smoother of the S-cycle


def bs_setup(h):
    """Per non-coarsest level l: A^{-1} = 1 / (2 diag A) and the S hierarchy
    S_l, H_l^T S_l H_l, ... down to the coarsest pressure level (its last matrix
    factorised by the complete-pivoting LU)."""
    L = len(h.levels) - 1
    for l in range(L):
        lv = h.levels[l]
        ahat_inv = 0.5 / lv.A.diagonal()
        S = (lv.C + lv.B @ sp.diags(ahat_inv) @ lv.B.T).tocsr()
        mats = [S]
        for k in range(l, L):
            Hk = h.levels[k].H
            mats.append((Hk.T @ mats[-1] @ Hk).tocsr())
        lv.extra["bs"] = {"ahat_inv": ahat_inv, "S": mats,
                          "S_dinv": [np.divide(1.0, m.diagonal(),
                                               out=np.zeros(m.shape[0]),
                                               where=m.diagonal() != 0.0) for m in mats],
                          "coarse": amg.complete_pivot_lu(mats[-1].toarray())}


def s_cycle(h, l, rhs):
    """One V(1,1)-cycle of the S hierarchy of level l from a zero initial guess."""
    bs = h.levels[l].extra["bs"]
    mats, dinv = bs["S"], bs["S_dinv"]

    def rec(k, b):
        if k == len(mats) - 1:
            return amg.complete_pivot_solve(bs["coarse"], b)
        S = mats[k]
        x = BS_JACOBI * dinv[k] * b
        Hk = h.levels[l + k].H
        xc = rec(k + 1, Hk.T @ (b - S @ x))
        x = x + Hk @ xc
        return x + BS_JACOBI * dinv[k] * (b - S @ x)
    return rec(0, rhs)


VANKA_OMEGA = 0.7    # damping of the Vanka correction (not stated in the paper; see the pins)


def vanka_setup(h):
    """Per non-coarsest level: the patches (pressure unknown k and the velocity
    nodes of the structural pattern of row k of B) and their local matrices
    K_k = [A_k B_k^T; B_k -C_kk], kept as the pieces of its block elimination:
    A_k^{-1} (A_k a principal submatrix of the SPD A: Cholesky), w_k = A_k^{-1} B_k^T
    and the scalar Schur complement s_k = B_k w_k + C_kk; and the first-fit greedy
    colouring, in patch order, of the patches' overlap graph (two patches conflict
    when they share a velocity node)."""
    L = len(h.levels) - 1
    for l in range(L):
        lv = h.levels[l]
        bp = lv.extra["b_pattern"]
        A = lv.A.tocsr()
        B = lv.B.tocsr()
        C = lv.C.tocsr()
        patches, ainv, w, sk = [], [], [], []
        for k in range(lv.npres):
            nodes = np.sort(bp.indices[bp.indptr[k]:bp.indptr[k + 1]])
            dofs = (3 * nodes[:, None] + np.arange(3)).ravel()
            Ak = A[dofs][:, dofs].toarray()
            Bk = B[k, dofs].toarray().ravel()
            fac = sla.cho_factor(Ak)
            Ai = sla.cho_solve(fac, np.eye(len(dofs)))
            wk = Ai @ Bk
            patches.append(dofs)
            ainv.append(Ai)
            w.append(wk)
            sk.append(float(Bk @ wk + C[k, k]))
        overlap = (bp @ bp.T).tocsr()
        colour = amg.greedy_colouring(overlap)
        lv.extra["vanka"] = {"dofs": patches, "ainv": ainv, "w": w, "s": np.array(sk),
                             "B": B, "colour": colour,
                             "ncolours": int(colour.max()) + 1 if len(colour) else 0}


def vanka_local_solve(vk, k, ru, rp):
    """[du; dp] = K_k^{-1} [ru; rp] by block elimination: y = A_k^{-1} ru,
    dp = (B_k y - rp) / s_k (0 when s_k = 0: the patch's pressure couples to no
    free velocity and has no C entry), du = y - w_k dp."""
    y = vk["ainv"][k] @ ru
    dofs = vk["dofs"][k]
    bk = vk["B"][k, dofs].toarray().ravel()
    s_k = vk["s"][k]
    dp = (bk @ y - rp) / s_k if s_k != 0.0 else 0.0
    return y - vk["w"][k] * dp, dp


def smooth_vanka(h, l, x, b, post):
    """Multiplicative Vanka, Eq. (locpatchsm), over the patch colours (ascending
    before the coarse correction, descending after it): per colour the residual of
    the whole level is updated, then every patch of the colour adds
    omega K_k^{-1} r_k to its unknowns (patches of one colour do not overlap)."""
    lv = h.levels[l]
    vk = lv.extra["vanka"]
    nu = 3 * lv.n
    x = x.copy()
    order = range(vk["ncolours"])
    if post and h.opts.post_order == "reverse":
        order = reversed(list(order))
    for c in order:
        r = b - apply_K(lv, x)
        for k in np.nonzero(vk["colour"] == c)[0]:
            dofs = vk["dofs"][k]
            du, dp = vanka_local_solve(vk, k, r[dofs], r[nu + k])
            x[dofs] += VANKA_OMEGA * du
            x[nu + k] += VANKA_OMEGA * dp
    return x


def smooth_bs(h, l, x, b):
    """One Braess-Sarazin step, Eq. (bssm) with K^ of Eq. (bssmpre)."""
    lv = h.levels[l]
    bs = lv.extra["bs"]
    nu = 3 * lv.n
    r = b - apply_K(lv, x)
    ru, rp = r[:nu], r[nu:]
    w = bs["ahat_inv"] * ru
    dp = s_cycle(h, l, lv.B @ w - rp)
    du = w - bs["ahat_inv"] * (lv.B.T @ dp)
    return x + np.concatenate([du, dp])


def apply_K(lv, v):
    nu = 3 * lv.n
    u, p = v[:nu], v[nu:]
    return np.concatenate([lv.A @ u + lv.B.T @ p, lv.B @ u - lv.C @ p])


def restrict(lv, r):
    nu = 3 * lv.n
    return np.concatenate([lv.Pk.T @ r[:nu], lv.H.T @ r[nu:]])


def prolong(lv, xc):
    ncu = lv.Pk.shape[1]
    return np.concatenate([lv.Pk @ xc[:ncu], lv.H @ xc[ncu:]])


def smooth(h, l, x, b, post):
    """Segregated Gauss-Seidel, Eq. (uzsm) with M_A = damped block Jacobi, or the
    Braess-Sarazin step (Options.smoother = "bs")."""
    lv = h.levels[l]
    o = h.opts
    if o.smoother == "bs":
        return smooth_bs(h, l, x, b)
    if o.smoother == "vanka":
        return smooth_vanka(h, l, x, b, post)
    nu = 3 * lv.n
    u, p = x[:nu].copy(), x[nu:].copy()
    f, g = b[:nu], b[nu:]
    ru = f - lv.A @ u - lv.B.T @ p
    ws, _, wp = amg.level_multipliers(o, l)
    u = u + o.omega * ws * amg.apply_dinv(lv.dinv, ru)
    sdg = lv.extra["schur_diag"]
    rp = lv.B @ u - lv.C @ p - g
    p = p + o.omega_p * wp * np.divide(rp, sdg, out=np.zeros_like(rp), where=sdg != 0.0)
    return np.concatenate([u, p])


def coarse_matrix(lv):
    return np.block([[lv.A.toarray(), lv.B.T.toarray()], [lv.B.toarray(), -lv.C.toarray()]])


def factor_coarsest(h):
    return ("cplu", amg.complete_pivot_lu(coarse_matrix(h.levels[-1])))


def pressure_projector(h):
    lv = h.levels[0]
    if not lv.extra["stokes"]:
        return None
    w = lv.extra["pmass"]
    nu = 3 * lv.n

    def project(v):
        v = v.copy()
        v[nu:] -= (w @ v[nu:]) / w.sum()
        return v
    return project


def solve(h, prob, b, tol, maxit, method=None):
    """FGMRES(50) (Sec. 4.4), or with method = "amg" the stand-alone AMG iteration."""
    lv0 = h.levels[0]
    project = pressure_projector(h)
    K = lambda v: apply_K(lv0, v)                            # noqa: E731
    if method == "amg":
        M = lambda r: (project or (lambda v: v))(amg.precondition(h, r))   # noqa: E731
        res = amg.amg_iteration(K, M, b, tol, maxit=maxit)
    else:
        res = amg.fgmres(K, lambda r: amg.precondition(h, r), b, tol,
                         restart=50, maxit=maxit, project=project)
    if project is not None:
        res.x = project(res.x)
    return res
