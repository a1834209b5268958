"""Pins of the oracle's Braess-Sarazin smoother (no GPU).

* One step equals a preconditioned Richardson step with the matrix of Eq.
  (bssmpre), K^ = [A^ B^T; B B A^{-1} B^T - S^], written densely with S^ the
  inverse of the S-cycle's matrix: K^ (x_new - x) = b - K x.
* The S-cycle on a two-level S hierarchy equals the closed-form two-grid
  operator (I - E) S^{-1}, E = (I - w D^{-1} S)(I - H S_c^{-1} H^T S)(I - w D^{-1} S),
  with S = C + B A^{-1} B^T and A^ = 2 diag(A) formed densely.
* BS-preconditioned FGMRES reaches the dense direct solution.
"""
import numpy as np

from fem_inputs import problems as fp
from oracle import amg, saddle


def _hier(prob):
    return amg.build_hierarchy(prob, amg.Options(smoother="bs"))


def _dense_s_cycle(h, l, m):
    return np.column_stack([saddle.s_cycle(h, l, e) for e in np.eye(m)])


def test_bs_step_solves_the_preconditioner_of_eq_bssmpre():
    prob = fp.mixed_elasticity_problem(2, nu=0.45, seed=1)
    h = _hier(prob)
    lv = h.levels[0]
    nu, npres = 3 * lv.n, lv.npres
    A = lv.A.toarray()
    Bm = lv.B.toarray()
    ahat = np.diag(2.0 * np.diag(A))
    Ms = _dense_s_cycle(h, 0, npres)
    Shat = np.linalg.inv(Ms)
    Khat = np.block([[ahat, Bm.T], [Bm, Bm @ np.linalg.inv(ahat) @ Bm.T - Shat]])
    rng = np.random.default_rng(0)
    x = rng.standard_normal(nu + npres)
    b = rng.standard_normal(nu + npres)
    r = b - saddle.apply_K(lv, x)
    x1 = saddle.smooth(h, 0, x, b, post=False)
    assert np.linalg.norm(Khat @ (x1 - x) - r) <= 1e-10 * np.linalg.norm(r)


def test_s_cycle_is_the_two_grid_operator():
    prob = fp.mixed_elasticity_problem(2, nu=0.45, seed=1)
    h = _hier(prob)
    assert len(h.levels) == 2          # S hierarchy of level 0: S_0 and S_1 = H^T S_0 H
    lv = h.levels[0]
    A = lv.A.toarray()
    Bm = lv.B.toarray()
    S = lv.C.toarray() + Bm @ np.diag(1.0 / (2.0 * np.diag(A))) @ Bm.T
    H = lv.H.toarray()
    Sc = H.T @ S @ H
    n = S.shape[0]
    J = np.eye(n) - 0.5 * np.diag(1.0 / np.diag(S)) @ S
    E = J @ (np.eye(n) - H @ np.linalg.solve(Sc, H.T @ S)) @ J
    want = (np.eye(n) - E) @ np.linalg.inv(S)
    got = _dense_s_cycle(h, 0, n)
    assert np.linalg.norm(got - want) <= 1e-11 * np.linalg.norm(want)
    assert np.linalg.norm(got - got.T) <= 1e-12 * np.linalg.norm(got)   # symmetric V(1,1)


def test_bs_fgmres_reaches_the_direct_solution():
    prob = fp.mixed_elasticity_problem(3, nu=0.49, seed=2)
    res, h = amg.solve(prob, amg.Options(smoother="bs"), tol=1e-12)
    assert res.converged
    K = saddle.coarse_matrix(h.levels[0])
    x = np.linalg.solve(K, prob.rhs())
    assert np.linalg.norm(res.x - x) <= 1e-9 * np.linalg.norm(x)


# --------------------------------------------------------------------------- Vanka

def test_vanka_local_solve_is_the_patch_inverse():
    """Block elimination of Eq. (locpatchsm)'s local matrix equals a dense solve
    of [A_k B_k^T; B_k -C_kk] assembled from the level's matrices."""
    prob = fp.paper_setting_problem("mixed", 3)
    h = amg.build_hierarchy(prob, amg.Options(smoother="vanka"))
    lv = h.levels[0]
    vk = lv.extra["vanka"]
    A, Bm, Cm = lv.A.toarray(), lv.B.toarray(), lv.C.toarray()
    rng = np.random.default_rng(1)
    checked = 0
    for k in range(0, lv.npres, 7):
        dofs = vk["dofs"][k]
        m = len(dofs)
        K = np.zeros((m + 1, m + 1))
        K[:m, :m] = A[np.ix_(dofs, dofs)]
        K[m, :m] = K[:m, m] = Bm[k, dofs]
        K[m, m] = -Cm[k, k]
        r = rng.standard_normal(m + 1)
        du, dp = saddle.vanka_local_solve(vk, k, r[:m], r[m])
        want = np.linalg.solve(K, r)
        assert np.linalg.norm(np.concatenate([du, [dp]]) - want) <= 1e-9 * np.linalg.norm(want)
        checked += 1
    assert checked > 3


def test_vanka_patches_and_colouring():
    """Patch k holds the velocity nodes of row k of B; patches of one colour share
    no velocity node; the colouring is first-fit in patch order."""
    prob = fp.mixed_elasticity_problem(3, nu=0.49, seed=2)
    h = amg.build_hierarchy(prob, amg.Options(smoother="vanka"))
    for lv in h.levels[:-1]:
        vk = lv.extra["vanka"]
        bp = lv.extra["b_pattern"]
        col = vk["colour"]
        owner = {}
        for k in range(lv.npres):
            nodes = bp.indices[bp.indptr[k]:bp.indptr[k + 1]]
            assert np.array_equal(np.unique(vk["dofs"][k] // 3), np.sort(nodes))
            for j in nodes:
                for k2 in owner.get(j, []):
                    assert col[k2] != col[k]
                owner.setdefault(j, []).append(k)
        # first fit: every patch's colour is the smallest not used by earlier conflicting ones
        for k in range(lv.npres):
            nb = {col[k2] for j in bp.indices[bp.indptr[k]:bp.indptr[k + 1]]
                  for k2 in owner[j] if k2 < k}
            assert col[k] == min(set(range(len(nb) + 1)) - nb)


def test_vanka_fgmres_reaches_the_direct_solution():
    prob = fp.mixed_elasticity_problem(3, nu=0.49, seed=2)
    res, h = amg.solve(prob, amg.Options(smoother="vanka"), tol=1e-12)
    assert res.converged
    K = saddle.coarse_matrix(h.levels[0])
    x = np.linalg.solve(K, prob.rhs())
    assert np.linalg.norm(res.x - x) <= 1e-9 * np.linalg.norm(x)
