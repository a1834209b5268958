"""Host-side parts of the weight-network training (no GPU): the listwise ranking
loss's gradient against central differences, and its limits (a network that orders
the candidates as measured has the lowest loss); the selection regret."""
import numpy as np

from paper_1503_01287_gb300.train_weights import rank_loss_grad, selection_regret


def test_rank_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    y = 0.05 * rng.standard_normal(28)
    T = 0.05 * rng.standard_normal(28)
    L, d = rank_loss_grad(y, T, 4)
    h = 1e-7
    for i in range(28):
        e = np.zeros(28)
        e[i] = h
        fd = (rank_loss_grad(y + e, T, 4)[0] - rank_loss_grad(y - e, T, 4)[0]) / (2 * h)
        assert abs(fd - d[i]) <= 1e-6 * max(1.0, np.abs(d).max())
    # the gradient of each problem sums to zero (a common shift of its outputs is free)
    assert np.allclose(d.reshape(4, -1).sum(axis=1), 0.0, atol=1e-12)


def test_rank_loss_prefers_the_measured_order():
    T = np.array([0.0, 0.03, -0.02, 0.05, 0.01, 0.04, 0.02])
    L_same, _ = rank_loss_grad(T.copy(), T, 1)
    L_rev, _ = rank_loss_grad(-T, T, 1)
    assert L_same < L_rev


def test_selection_regret():
    owner = np.repeat(np.arange(3), 3)
    T = np.array([0.0, -0.1, 0.2, 0.0, 0.1, 0.3, 0.0, -0.2, -0.3])
    y = np.array([1.0, 0.0, 2.0, 0.0, 1.0, 2.0, 0.0, 1.0, 2.0])  # picks -0.1, 0.0, 0.0
    assert abs(selection_regret(y, T, owner) - (0.0 + 0.0 + 0.3) / 3) <= 1e-15
