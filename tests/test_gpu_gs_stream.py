"""The grid-stride multicolour Gauss-Seidel colour kernel (gs_stream), forced on,
against the oracle's colour-by-colour sweep (Sec. 3.3): single sweeps in both
colour orders on every level, entry by entry (FP64: within 1e-12 of the largest
entry), one preconditioner application in FP64 and FP32 for several grid sizes,
and a whole solve."""
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


def stream_handle(prob, cps, **opts):
    o = dict(gs_stream=cps, gs_flow=0, gs_cluster=0, cluster_from=0, cycle_kernel=1)
    o.update(opts)
    return B().setup_problem(prob, B().default_options(**o))


@pytest.mark.parametrize("cps", [1, 3])
@pytest.mark.parametrize("maker", [
    lambda: fp.elasticity_problem(9, seed=4),
    lambda: fp.elasticity_problem((5, 9, 4), seed=2, lengths=(1.0, 2.5, 3.0), nu=0.4),
])
def test_stream_sweep_matches_oracle(maker, cps):
    prob = maker()
    h = stream_handle(prob, cps)
    oh = amg.build_hierarchy(prob)
    rng = np.random.default_rng(1)
    for l in range(len(oh.levels) - 1):
        lv = oh.levels[l]
        for post in (False, True):
            x0 = rng.standard_normal(3 * lv.n)
            b = rng.standard_normal(3 * lv.n)
            xg = cuda(x0)
            h.level_smooth(l, xg, cuda(b), post=post)
            want = amg.gs_sweep(lv, x0, b, reverse=post)
            got = xg.cpu().numpy()
            assert np.all(np.abs(got - want) <= 1e-12 * np.abs(want).max()), (l, post)
    h.free()


@pytest.mark.parametrize("precision,cps", [(0, 1), (0, 2), (1, 1), (1, 4)])
def test_stream_preconditioner_and_solve(precision, cps):
    prob = fp.elasticity_problem(10, seed=6)
    h = stream_handle(prob, cps, precision=precision)
    oh = amg.build_hierarchy(prob)
    r = np.random.default_rng(2).standard_normal(prob.n_dof)
    z = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
    h.apply_preconditioner(cuda(r), z)
    want = amg.precondition(oh, r)
    tol = 1e-10 if precision == 0 else 1e-4
    assert np.all(np.abs(z.cpu().numpy() - want) <= tol * np.abs(want).max())
    b = cuda(prob.rhs())
    x = torch.zeros_like(b)
    st = h.solve(b, x, 1e-8, device_ptrs=True)
    assert st.converged and st.level_gs_stream[0] == cps
    ref, _ = amg.solve(prob, tol=1e-8, h=oh, method="fcg" if precision else None)
    assert abs(st.iterations - ref.iterations) <= 1
    if st.iterations == ref.iterations:
        assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-10 * np.linalg.norm(ref.x)
    h.free()
