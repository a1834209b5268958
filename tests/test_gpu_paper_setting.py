"""GPU path vs the oracle at the paper's own scale: the Sec. 4.1 setting (unit cube,
u = 0 on z = 0, u = (0, 0, 1) on z = 1; elasticity and mixed elasticity with
mu = 1.15e6, lambda = 1.73e6) at L1 and L2 (4^3 and 8^3), the systems behind
Tables 4-16.

Per kind: the hierarchy bit-exact (C/F splits, prolongations, patterns,
colourings; Galerkin values within 1e-12 of the largest entry); one
preconditioner application entry by entry within 1e-10 of the largest entry;
the Krylov solution (PCG, or FGMRES for the mixed form) within 1e-9 of the
oracle's (the mixed form: its residual recomputed by the oracle, and the
solution within 1e-7); and the stand-alone AMG iteration with GS-1-1 within one iteration
of the oracle's, which with the post-smoothing colours in the pre-smoothing
order lies near Table 4's count.
"""
import numpy as np
import pytest

from fem_inputs import problems as fp
from oracle import amg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from parity_helpers import check_hierarchy, coarse_check  # noqa: E402


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


CASES = [(k, n) for k in ("laplace", "elasticity", "mixed") for n in (4, 8)]


@pytest.mark.parametrize("kind,n", CASES)
def test_paper_setting_matches_oracle(kind, n):
    prob = fp.paper_setting_problem(kind, n)
    h = B().setup_problem(prob, B().default_options())
    oh = amg.build_hierarchy(prob, amg.Options(smoother="sgs" if prob.saddle else "gs"))
    check_hierarchy(h, oh)
    coarse_check(h, oh)
    # one preconditioner application, entry by entry
    r = np.random.default_rng(n).standard_normal(prob.n_dof)
    z = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
    h.apply_preconditioner(cuda(r), z)
    want = amg.precondition(oh, r)
    got = z.cpu().numpy()
    assert np.all(np.abs(got - want) <= 1e-10 * np.abs(want).max())
    # the Krylov solve
    b = prob.rhs()
    x = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
    st = h.solve(cuda(b), x, 1e-10, device_ptrs=True)
    ref, _ = amg.solve(prob, tol=1e-10, h=oh)
    assert st.converged and ref.converged
    assert abs(st.iterations - ref.iterations) <= (2 if prob.saddle else 1)
    xv = x.cpu().numpy()
    if prob.saddle:
        # Two iterates with ||b - K x|| <= 1e-10 ||b|| differ by up to about
        # 2e-10 ||K^{-1}|| ||b||; the indefinite system's conditioning at this scale
        # allows no 1e-9 bound on the solution, so the GPU's residual is checked in
        # the oracle's FP64 operator and the solutions to the bound that the
        # existing saddle tests use.
        from oracle import saddle as sd
        assert np.linalg.norm(b - sd.apply_K(oh.levels[0], xv)) <= 1.5e-10 * np.linalg.norm(b)
        assert np.linalg.norm(xv - ref.x) <= 1e-7 * np.linalg.norm(ref.x)
    else:
        assert np.linalg.norm(xv - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    h.free()


@pytest.mark.parametrize("kind", ["laplace", "elasticity"])
def test_paper_setting_standalone_gs(kind):
    """Stand-alone AMG, V-cycle, GS-1-1 to 1e-11 at 4^3 (Tables 4 and 8, L1)."""
    prob = fp.paper_setting_problem(kind, 4)
    h = B().setup_problem(prob, B().default_options(krylov=B().AMG_KRYLOV_NONE,
                                                    max_iterations=400))
    b = prob.rhs()
    x = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
    st = h.solve(cuda(b), x, 1e-11, device_ptrs=True)
    ref, _ = amg.solve(prob, amg.Options(smoother="gs", post_order="same"), tol=1e-11,
                       method="amg", maxit=400)
    assert st.converged and ref.converged
    assert abs(st.iterations - ref.iterations) <= 1, (st.iterations, ref.iterations)
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
    h.free()
