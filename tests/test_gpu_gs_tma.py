"""The TMA-staged multicolour Gauss-Seidel colour kernel (gs_tma, FP32 cycle), forced
on, against the oracle's colour-by-colour sweep (Sec. 3.3).

Checked: single FP32 sweeps in both colour orders on every coloured level, entry by
entry against the FP64 oracle (FP32 rounding: within 1e-4 of the largest entry, the
bound of the other FP32 sweep tests); the same sweeps bit for bit against the
register-prefetch colour kernel of a handle whose tuned lanes per row agree on that
level (the two kernels sum a row in the same order); one FP32 preconditioner
application; whole solves against the oracle's; and that the stats report where the
kernel ran.
"""
import numpy as np
import pytest

from fem_inputs import problems as fp
from oracle import amg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def B():
    from paper_1503_01287_gb300 import binding
    return binding


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def handle(prob, tma, **opts):
    o = dict(precision=1, gs_tma=tma, gs_stream=0, gs_flow=0, gs_cluster=0, cluster_from=0,
             cycle_kernel=1)
    o.update(opts)
    return B().setup_problem(prob, B().default_options(**o))


MAKERS = [
    lambda: fp.elasticity_problem(9, seed=4),
    lambda: fp.elasticity_problem((5, 9, 4), seed=2, lengths=(1.0, 2.5, 3.0), nu=0.4),
    lambda: fp.elasticity_problem(16, seed=1),
    lambda: fp.vector_laplace_problem(12, seed=3),
]


@pytest.mark.parametrize("maker", MAKERS)
def test_tma_sweep_matches_oracle_and_prefetch_kernel(maker):
    prob = maker()
    ht = handle(prob, 1)
    hp = handle(prob, 0)
    oh = amg.build_hierarchy(prob)
    st_t = ht.solve(cuda(prob.rhs()), torch.zeros(prob.n_dof, dtype=torch.float64,
                                                  device="cuda"), 1e-6, device_ptrs=True)
    st_p = hp.solve(cuda(prob.rhs()), torch.zeros(prob.n_dof, dtype=torch.float64,
                                                  device="cuda"), 1e-6, device_ptrs=True)
    assert all(v == 1 for v in st_t.level_gs_tma[:st_t.n_levels - 1]), list(st_t.level_gs_tma)
    assert not any(st_p.level_gs_tma[:st_p.n_levels - 1])
    rng = np.random.default_rng(1)
    same_g = 0
    for l in range(len(oh.levels) - 1):
        lv = oh.levels[l]
        for post in (False, True):
            x0 = rng.standard_normal(3 * lv.n)
            b = rng.standard_normal(3 * lv.n)
            xt, xp = cuda(x0), cuda(x0)
            ht.level_smooth(l, xt, cuda(b), post=post, precision=B().AMG_FP32)
            hp.level_smooth(l, xp, cuda(b), post=post, precision=B().AMG_FP32)
            want = amg.gs_sweep(lv, x0, b, reverse=post)
            got = xt.cpu().numpy()
            assert np.all(np.abs(got - want) <= 1e-4 * np.abs(want).max()), (l, post)
            if st_t.level_group[l] == st_p.level_group[l]:
                assert np.array_equal(got, xp.cpu().numpy()), (l, post)
                same_g += 1
    ht.free()
    hp.free()


@pytest.mark.parametrize("okw", [{}, {"post_order": 1}, {"nu": 2, "m_pre": 2, "m_post": 2}])
def test_tma_preconditioner_matches_oracle(okw):
    prob = fp.elasticity_problem(10, seed=6)
    h = handle(prob, 1, **okw)
    o = {k: v for k, v in okw.items() if k in ("nu", "m_pre", "m_post")}
    if okw.get("post_order") == 1:
        o["post_order"] = "same"
    oh = amg.build_hierarchy(prob, amg.Options(smoother="gs", **o))
    r = np.random.default_rng(2).standard_normal(prob.n_dof)
    z = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
    for rep in range(2):
        h.apply_preconditioner(cuda(r), z)
        want = amg.precondition(oh, r)
        got = z.cpu().numpy()
        assert np.all(np.abs(got - want) <= 1e-4 * np.abs(want).max()), rep
    h.free()


@pytest.mark.parametrize("maker", [MAKERS[0], MAKERS[2]])
def test_tma_solve_matches_oracle(maker):
    prob = maker()
    h = handle(prob, 1)
    b = cuda(prob.rhs())
    x = torch.zeros_like(b)
    st = h.solve(b, x, 1e-8, device_ptrs=True)
    assert st.converged and st.true_rel_residual <= 1.5e-8
    ref, _ = amg.solve(prob, tol=1e-8, method="fcg")
    assert abs(st.iterations - ref.iterations) <= 1
    A = prob.a_scipy().tocsr()
    xv = x.cpu().numpy()
    assert np.linalg.norm(prob.rhs() - A @ xv) <= 1.5e-8 * np.linalg.norm(prob.rhs())
    h.free()


def test_tma_chosen_by_timing_keeps_results():
    """The default (gs_tma = -1) keeps the staged kernel per level only where it is
    faster; whatever it picks, the solve still matches the oracle's."""
    prob = fp.elasticity_problem(14, seed=2)
    h = B().setup_problem(prob, B().default_options(precision=1))
    b = cuda(prob.rhs())
    x = torch.zeros_like(b)
    st = h.solve(b, x, 1e-8, device_ptrs=True)
    ref, _ = amg.solve(prob, tol=1e-8, method="fcg")
    assert st.converged and abs(st.iterations - ref.iterations) <= 1
    h.free()


def test_tma_option_range():
    prob = fp.elasticity_problem(4, seed=1)
    for bad in (-2, 2):
        with pytest.raises(B().AmgError):
            B().setup_problem(prob, B().default_options(precision=1, gs_tma=bad))
