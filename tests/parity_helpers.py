"""Comparisons of a GPU hierarchy with the oracle's, shared by the GPU parity tests
(imported by them; not a test module).

check_hierarchy: level sizes, block patterns, tags, C/F states, prolongation
patterns and weights, colourings and (saddle) B, C, pressure C/F states and H
patterns bit-exact; Galerkin values within vals_tol of the largest entry, D^-1
within 1e-10.  coarse_check: the GPU's generalised inverse of the coarsest matrix
solves a consistent system and gives the oracle's complete-pivot solution of it
(both pivot on the first of the near-tied largest entries, so they pick the same
solution of a singular Stokes coarse matrix too).
"""
import numpy as np
import scipy.sparse as sp

from oracle import amg

STATE = {amg.STATE_C: 1, amg.STATE_F: 2}


def check_hierarchy(h, oh, vals_tol=1e-12, check_colour=True):
    assert h.n_levels == len(oh.levels), (h.n_levels, [lv.n for lv in oh.levels])
    for l, lv in enumerate(oh.levels):
        info = h.level_info(l)
        last = l == len(oh.levels) - 1
        assert info.n_nodes == lv.n
        assert np.array_equal(h.level_array(l, "a_rowptr"), lv.rowptr)
        assert np.array_equal(h.level_array(l, "a_col"), lv.col)
        assert np.array_equal(h.level_array(l, "tags"), lv.tags)
        v = h.level_array(l, "a_val").reshape(-1, 3, 3)
        assert np.abs(v - lv.val).max() <= vals_tol * np.abs(lv.val).max()
        d = h.level_array(l, "dinv").reshape(-1, 3, 3)
        assert np.abs(d - lv.dinv).max() <= 1e-10 * np.abs(lv.dinv).max()
        if not last:
            st = h.level_array(l, "cf_state")
            assert np.array_equal(st, np.vectorize(STATE.get)(lv.state))
            prow = h.level_array(l, "p_rowptr")
            pcol = h.level_array(l, "p_col")
            ps = lv.P_structure.tocsr()
            ps.sort_indices()
            assert np.array_equal(prow, ps.indptr) and np.array_equal(pcol, ps.indices)
            rows = np.repeat(np.arange(lv.n), np.diff(prow))
            want = np.asarray(lv.P[rows, pcol]).ravel()
            assert np.array_equal(h.level_array(l, "p_val"), want)
            if check_colour and not oh.saddle:
                assert np.array_equal(h.level_array(l, "colour"), lv.colour)
        if oh.saddle:
            assert info.n_pres == lv.npres
            nb = 3 * lv.n
            bc = h.level_array(l, "b_col")
            brow = h.level_array(l, "b_rowptr")
            bv = h.level_array(l, "b_val").reshape(-1, 3)
            Bg = sp.csr_matrix((bv.ravel(), (np.repeat(np.repeat(np.arange(lv.npres),
                                                                  np.diff(brow)), 3),
                                              (3 * bc[:, None] + np.arange(3)).ravel())),
                               shape=(lv.npres, nb))
            assert abs(Bg - lv.B).max() <= vals_tol * max(abs(lv.B).max(), 1e-300)
            crow = h.level_array(l, "c_rowptr")
            Cg = sp.csr_matrix((h.level_array(l, "c_val"), h.level_array(l, "c_col"), crow),
                               shape=(lv.npres, lv.npres))
            assert abs(Cg - lv.C).max() <= vals_tol * max(abs(lv.C).max(), 1e-300) + 1e-300
            if not last:
                assert np.array_equal(h.level_array(l, "pcf_state"),
                                      np.vectorize(STATE.get)(lv.p_state))
                hs = lv.H_structure.tocsr()
                hs.sort_indices()
                assert np.array_equal(h.level_array(l, "h_rowptr"), hs.indptr)
                assert np.array_equal(h.level_array(l, "h_col"), hs.indices)


def coarse_check(h, oh):
    L = len(oh.levels) - 1
    m = 3 * oh.levels[L].n + oh.levels[L].npres
    X = h.level_array(L, "coarse_inv").reshape(m, m)
    rng = np.random.default_rng(5)
    bvec = rng.standard_normal(m)
    if oh.saddle:
        from oracle import saddle as sd
        K = sd.coarse_matrix(oh.levels[L])
    else:
        K = oh.levels[L].A.toarray()
    bvec = K @ bvec          # consistent right-hand side
    want = amg.complete_pivot_solve(oh.coarse_factor[1], bvec)
    got = X @ bvec
    assert np.abs(K @ got - bvec).max() <= 1e-9 * np.abs(bvec).max()
    # the same pivot sequence gives the same solution, also of a singular matrix
    assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max()
