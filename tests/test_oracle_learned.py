"""Pins of the oracle's learned-weights parts (no GPU): the network's gradient
against central finite differences of its loss, its forward pass against a
network built by hand, and the hierarchy statistics against closed forms and
a second, matrix-level formulation of the same definitions."""
import numpy as np
import scipy.sparse as sp

from fem_inputs import problems as fp
from oracle import amg, features, mlp


def test_mlp_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    theta = mlp.init(5) + 0.05 * rng.standard_normal(mlp.NPARAM)
    X = rng.standard_normal((24, mlp.NI))
    t = rng.standard_normal(24)
    g = mlp.grad(theta, X, t)
    idx = rng.choice(mlp.NPARAM, 200, replace=False)
    idx = np.concatenate([idx, [mlp.NPARAM - 1, 0, 64 * 16, 64 * 16 + 64]])  # b3, W1, b1, W2
    h = 1e-6
    fd = np.empty(len(idx))
    for k, i in enumerate(idx):
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        fd[k] = (mlp.loss(theta + e, X, t) - mlp.loss(theta - e, X, t)) / (2 * h)
    assert np.abs(fd - g[idx]).max() <= 1e-6 * max(1.0, np.abs(g[idx]).max())


def test_mlp_forward_of_a_hand_built_network():
    """W1 picks input 13, W2 copies unit 0, W3 scales by c: y = c * relu(x_13) + b3."""
    p = {k: np.zeros(s) for k, s in mlp.SIZES}
    p["W1"][0, 13] = 1.0
    p["W2"][0, 0] = 1.0
    p["W3"][0] = -2.5
    p["b3"][0] = 0.75
    theta = mlp.pack(p)
    X = np.zeros((4, mlp.NI))
    X[:, 13] = [0.6, 1.0, 1.6, -0.3]
    y, _ = mlp.forward(theta, X)
    assert np.allclose(y, -2.5 * np.maximum(X[:, 13], 0.0) + 0.75, rtol=0, atol=1e-15)
    assert mlp.NPARAM == 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1


def test_features_vector_laplacian_closed_form():
    """Blocks a_ij I_3: |D_i| |D_i^-1| = sqrt(3) a * sqrt(3) / a = 3 on every level."""
    prob = fp.vector_laplace_problem(4, seed=0)
    h = amg.build_hierarchy(prob)
    f = features.features(h, False)
    assert abs(f[1] - np.log10(3.0)) <= 1e-13
    assert abs(f[6] - np.log10(3.0)) <= 1e-13
    assert f[0] == np.log10(prob.n_dof) / 7.0
    assert f[11] == 0.0 and f[12] == 0.0


def test_features_are_scale_free():
    prob = fp.elasticity_problem(4, seed=2)
    f1 = features.features(amg.build_hierarchy(prob), False)
    prob.a_val = prob.a_val * 7.3
    f2 = features.features(amg.build_hierarchy(prob), False)
    assert np.allclose(f1, f2, rtol=0, atol=1e-12)


def _share_and_size(lv):
    """The F-node statistics as matrix products: N (Frobenius norms of the
    off-diagonal blocks), M (1 where column j is a C node in the pattern of row
    i of P), share_i = (N o M) 1 / N 1."""
    n = lv.n
    norms = np.linalg.norm(lv.val.reshape(-1, 9), axis=1)
    rows = np.repeat(np.arange(n), np.diff(lv.rowptr))
    off = rows != lv.col
    N = sp.csr_matrix((norms[off], (rows[off], lv.col[off])), shape=(n, n))
    c_nodes = np.nonzero(lv.state == amg.STATE_C)[0]
    E = sp.csr_matrix((np.ones(len(c_nodes)), (lv.coarse_of_fine[c_nodes], c_nodes)),
                      shape=(lv.P_structure.shape[1], n))
    M = (lv.P_structure @ E).tocsr()
    M.data[:] = 1.0
    num = np.asarray(N.multiply(M).sum(axis=1)).ravel()
    den = np.asarray(N.sum(axis=1)).ravel()
    psize = np.diff(lv.P_structure.tocsr().indptr)
    sel = (lv.state == amg.STATE_F) & ((lv.tags & amg.TAG_DIRICHLET) == 0) & (psize > 0)
    share = np.where(den[sel] > 0, num[sel] / np.where(den[sel] > 0, den[sel], 1.0), 0.0)
    return share.mean(), psize[sel].mean() / 8.0


def test_features_interpolation_statistics_by_matrix_products():
    for prob, saddle in [(fp.elasticity_problem(4, seed=2), False),
                         (fp.mixed_elasticity_family(4, [0.49], seed=3)[0], True)]:
        h = amg.build_hierarchy(prob)
        f = features.features(h, saddle)
        for l, base in [(0, 1), (1, 6)]:
            if l + 1 >= len(h.levels):
                continue
            share, size = _share_and_size(h.levels[l])
            assert abs(f[base + 3] - share) <= 1e-13
            assert abs(f[base + 4] - size) <= 1e-15
            assert 0.0 < share <= 1.0
        assert f[12] == (1.0 if saddle else 0.0)
        if saddle:
            assert 0.0 < f[11] < 1.0


def test_committed_training_data_and_network():
    """The committed dataset of measured convergence factors and the network trained
    on it: shapes, the target's definition (each problem's plain row is 0, targets
    clipped to [-1, 1]), the input layout (13 per-level statistics with the level
    index l / 4 as input 10, ws, wc, log2 wp), and the network's picks on the
    validation problems (FP64 forward pass): the measured candidate it ranks first
    converges closer to the best measured one than always keeping the plain weights
    does, and far closer than a random pick."""
    import os
    from paper_1503_01287_gb300.train_weights import selection_regret
    here = os.path.join(os.path.dirname(__file__), "..", "paper_1503_01287_gb300", "weights")
    d = np.load(os.path.join(here, "mlp_theta.data.npz"))
    X, T, owner, R = d["X"], d["T"].astype(np.float64), d["owner"], d["rows"]
    nprob = int(owner.max()) + 1
    per = len(T) // nprob
    assert X.shape == (nprob * per, mlp.NI) and T.shape == (nprob * per,)
    assert np.all(owner.reshape(nprob, per) == np.arange(nprob)[:, None])
    assert np.all(np.abs(T) <= 1.0)
    first = np.arange(nprob) * per                 # each problem's plain row
    assert np.all(T[first] == 0.0) and np.all(R[first, 0] == 0)
    assert np.all(X[first, 13] == 1.0) and np.all(X[first, 14] == 1.0)
    assert np.all(X[first, 15] == 0.0)
    assert np.array_equal(X[:, 10], (R[:, 0] / 4.0).astype(np.float32))   # level index
    assert np.all((X[:, 12] == 0.0) | (X[:, 12] == 1.0))
    theta = np.load(os.path.join(here, "mlp_theta.npy")).astype(np.float64)
    assert theta.shape == (mlp.NPARAM,) and np.all(np.isfinite(theta))
    # validation problems: the 10 % held out by the training script's permutation
    perm = np.random.default_rng(11).permutation(nprob)
    val = np.isin(owner, perm[:max(1, nprob // 10)])
    plain = np.zeros(len(T), dtype=bool)
    plain[first] = True
    y, _ = mlp.forward(theta, X[val].astype(np.float64))
    r_net = selection_regret(y, T[val], owner[val])
    r_plain = selection_regret(-plain[val].astype(np.float64), T[val], owner[val])
    r_rand = selection_regret(np.random.default_rng(0).standard_normal(val.sum()), T[val],
                              owner[val])
    assert r_net < r_plain and r_net < 0.1 * r_rand, (r_net, r_plain, r_rand)


def test_mlp_backward_matches_central_differences():
    """backward(theta, X, dy) is the gradient of sum_i dy_i y_i(theta)."""
    rng = np.random.default_rng(6)
    theta = mlp.init(2) + 0.05 * rng.standard_normal(mlp.NPARAM)
    X = rng.standard_normal((16, mlp.NI))
    dy = rng.standard_normal(16)
    g = mlp.backward(theta, X, dy)
    f = lambda th: float(dy @ mlp.forward(th, X)[0])   # noqa: E731
    idx = rng.choice(mlp.NPARAM, 150, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        fd = (f(theta + e) - f(theta - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, np.abs(g).max())
