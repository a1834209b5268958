"""The multicolour Gauss-Seidel sweep as one dataflow launch (gs_flow), against
the oracle's colour-by-colour sweep (Sec. 3.3).

gs_flow = 1 forces the dataflow sweep on every coloured level.  Checked: single
sweeps in both colour orders on every level, entry by entry (FP64: within 1e-12
of the largest entry; the same arithmetic as the colour chain, so only the
summation order within a row can differ); one preconditioner application in
FP64 and FP32 with both post-smoothing orders, W-cycles and two smoothing steps;
whole solves against the oracle's; repeated sweeps (the device-side sweep
number advances once per launch) and the stats report where it ran.
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


def flow_handle(prob, **opts):
    o = dict(gs_flow=1, gs_cluster=0, cluster_from=0, cycle_kernel=1)
    o.update(opts)
    return B().setup_problem(prob, B().default_options(**o))


@pytest.mark.parametrize("maker", [
    lambda: fp.elasticity_problem(8, seed=4),
    lambda: fp.elasticity_problem((5, 9, 4), seed=2, lengths=(1.0, 2.5, 3.0), nu=0.4),
    lambda: fp.vector_laplace_problem(7, seed=3),
])
def test_flow_sweep_matches_oracle(maker):
    prob = maker()
    h = flow_handle(prob)
    oh = amg.build_hierarchy(prob)
    rng = np.random.default_rng(1)
    for l in range(len(oh.levels) - 1):
        lv = oh.levels[l]
        for rep in range(2):                    # the sweep number advances per launch
            for post in (False, True):
                x0 = rng.standard_normal(3 * lv.n)
                b = rng.standard_normal(3 * lv.n)
                xg = cuda(x0)
                h.level_smooth(l, xg, cuda(b), post=post)
                want = amg.gs_sweep(lv, x0, b, reverse=post)
                got = xg.cpu().numpy()
                assert np.all(np.abs(got - want) <= 1e-12 * np.abs(want).max()), (l, post, rep)
    h.free()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("okw", [{}, {"post_order": 1}, {"nu": 2, "m_pre": 2, "m_post": 2}])
def test_flow_preconditioner_matches_oracle(precision, okw):
    prob = fp.elasticity_problem(9, seed=6)
    h = flow_handle(prob, precision=precision, **okw)
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
        # FP32 cycle: float rounding of every level's values and sums (the bound
        # the other FP32-cycle tests use)
        tol = 1e-10 if precision == 0 else 1e-4
        assert np.all(np.abs(got - want) <= tol * np.abs(want).max()), rep
    h.free()


@pytest.mark.parametrize("precision", [0, 1])
def test_flow_solve_matches_oracle(precision):
    prob = fp.elasticity_problem(10, seed=1)
    h = flow_handle(prob, precision=precision)
    b = cuda(prob.rhs())
    x = torch.zeros_like(b)
    st = h.solve(b, x, 1e-8, device_ptrs=True)
    assert st.converged
    assert any(v > 0 for v in st.level_gs_flow[:st.n_levels - 1]), list(st.level_gs_flow)
    ref, _ = amg.solve(prob, tol=1e-8, method="fcg" if precision else None)
    assert abs(st.iterations - ref.iterations) <= 1
    xv = x.cpu().numpy()
    if st.iterations == ref.iterations:
        assert np.linalg.norm(xv - ref.x) <= 1e-10 * np.linalg.norm(ref.x)
    A = prob.a_scipy().tocsr()
    assert np.linalg.norm(prob.rhs() - A @ xv) <= 1.5e-8 * np.linalg.norm(prob.rhs())
    h.free()


def test_flow_chosen_by_timing_keeps_results():
    """The default (gs_flow = -1) picks the dataflow sweep per level only where it
    is faster; whatever it picks, the solve still matches the oracle's."""
    prob = fp.elasticity_problem(12, seed=2)
    h = B().setup_problem(prob, B().default_options(precision=1))
    b = cuda(prob.rhs())
    x = torch.zeros_like(b)
    st = h.solve(b, x, 1e-8, device_ptrs=True)
    ref, _ = amg.solve(prob, tol=1e-8, method="fcg")
    assert st.converged and abs(st.iterations - ref.iterations) <= 1
    h.free()
