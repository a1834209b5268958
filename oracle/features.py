"""Plain FP64 statistics of a hierarchy that the learned-weights network reads
(TEST INFRASTRUCTURE ONLY: used by tests/ to check the CUDA statistics kernel).

For a level with blocks A_ij (3x3), diagonal blocks D_i = A_ii and Frobenius
norms |.|, over its nodes i that are not Dirichlet nodes:
  mean of log10(|D_i| |D_i^-1|)          block conditioning of the diagonal
  standard deviation of log10 |D_i|       spread of the diagonal scale
  mean of sum_{j != i} |A_ij| / |D_i|     off-diagonal weight of a block row
and over its F nodes (C/F state F) with an interpolation row, the interpolation
set S_i being the C nodes in the pattern of row i of P (the C-neighbours of i in
the coarsening graph, Dirichlet-zeroed weights included):
  mean of sum_{j in S_i} |A_ij| / sum_{j != i} |A_ij|
  mean of |S_i| / 8
The network sees [log10(unknowns) / 7, the five numbers of level 0, the five
of level 1, the mean over pressure rows of C_kk / S_D,kk (saddle kinds, S_D the
sGS scaling diag(C + B (D / omega)^-1 B^T)), 1 for saddle kinds].

The per-level inputs (level_features) describe one non-coarsest level l and the
level below it: [log10(unknowns of level l) / 7, the five numbers of level l,
the first four of level l + 1, l / 4, the pressure mean of level l (saddle
kinds with an sGS scaling), 1 for saddle kinds].

These are definitions (there is no published formula: the learned part has no
basis in the paper), written out node by node so that each can be read off.
"""
from __future__ import annotations

import numpy as np

from . import amg

N_FEATURES = 13


def _level_stats(lv: amg.Level, has_next: bool):
    tags = np.asarray(lv.tags)
    vals_cond, vals_ld, vals_off = [], [], []
    vals_share, vals_k = [], []
    P = lv.P_structure.tocsr() if has_next else None
    for i in range(lv.n):
        if tags[i] & amg.TAG_DIRICHLET:
            continue
        dn, off, offc = 0.0, 0.0, 0.0
        fnode = has_next and lv.state[i] == amg.STATE_F and P.indptr[i + 1] > P.indptr[i]
        interp = set()
        if fnode:
            interp = set(P.indices[P.indptr[i]:P.indptr[i + 1]].tolist())
        for k in range(lv.rowptr[i], lv.rowptr[i + 1]):
            j = int(lv.col[k])
            f = float(np.linalg.norm(lv.val[k]))
            if j == i:
                dn = f
                continue
            off += f
            if fnode and lv.state[j] == amg.STATE_C and int(lv.coarse_of_fine[j]) in interp:
                offc += f
        di = float(np.linalg.norm(lv.dinv[i]))
        vals_cond.append(np.log10(dn * di))
        vals_ld.append(np.log10(dn))
        vals_off.append(off / dn)
        if fnode:
            vals_share.append(offc / off if off > 0.0 else 0.0)
            vals_k.append(P.indptr[i + 1] - P.indptr[i])
    if not vals_cond:
        return [0.0] * 5
    out = [float(np.mean(vals_cond)), float(np.std(vals_ld)), float(np.mean(vals_off))]
    if vals_share:
        out += [float(np.mean(vals_share)), float(np.mean(vals_k)) / 8.0]
    else:
        out += [0.0, 0.0]
    return out


def features(h: amg.Hierarchy, saddle: bool) -> np.ndarray:
    """The 13 inputs of the network for hierarchy h (levels 0 and 1)."""
    L = h.levels
    l0 = L[0]
    dofs = 3 * l0.n + (l0.npres if saddle else 0)
    f = [np.log10(dofs) / 7.0]
    for l in range(2):
        if l < len(L):
            f += _level_stats(L[l], l + 1 < len(L))
        else:
            f += [0.0] * 5
    pres = 0.0
    if saddle and l0.npres > 0 and "schur_diag" in l0.extra:
        s = l0.extra["schur_diag"]
        cd = l0.C.diagonal()
        keep = s > 0.0
        pres = float(np.mean(cd[keep] / s[keep])) if keep.any() else 0.0
    f += [pres, 1.0 if saddle else 0.0]
    return np.array(f, dtype=np.float64)


def _pressure_mean(lv) -> float:
    if lv.npres <= 0 or "schur_diag" not in lv.extra:
        return 0.0
    s = lv.extra["schur_diag"]
    cd = lv.C.diagonal()
    keep = s > 0.0
    return float(np.mean(cd[keep] / s[keep])) if keep.any() else 0.0


def level_features(h: amg.Hierarchy, l: int, saddle: bool) -> np.ndarray:
    """The 13 per-level inputs of non-coarsest level l (see the module text)."""
    L = h.levels
    lv = L[l]
    dofs = 3 * lv.n + (lv.npres if saddle else 0)
    f = [np.log10(dofs) / 7.0]
    f += _level_stats(lv, l + 1 < len(L))
    f += _level_stats(L[l + 1], l + 2 < len(L))[:4]
    f += [l / 4.0, _pressure_mean(lv) if saddle else 0.0, 1.0 if saddle else 0.0]
    return np.array(f, dtype=np.float64)
