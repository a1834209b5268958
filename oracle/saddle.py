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
    """Segregated Gauss-Seidel, Eq. (uzsm) with M_A = damped block Jacobi."""
    lv = h.levels[l]
    o = h.opts
    nu = 3 * lv.n
    u, p = x[:nu].copy(), x[nu:].copy()
    f, g = b[:nu], b[nu:]
    ru = f - lv.A @ u - lv.B.T @ p
    u = u + o.omega * o.ws * amg.apply_dinv(lv.dinv, ru)
    sdg = lv.extra["schur_diag"]
    rp = lv.B @ u - lv.C @ p - g
    p = p + o.omega_p * o.wp * np.divide(rp, sdg, out=np.zeros_like(rp), where=sdg != 0.0)
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


def solve(h, prob, b, tol, maxit):
    lv0 = h.levels[0]
    project = pressure_projector(h)
    res = amg.fgmres(lambda v: apply_K(lv0, v), lambda r: amg.precondition(h, r), b, tol,
                     restart=50, maxit=maxit, project=project)
    if project is not None:
        res.x = project(res.x)
    return res
