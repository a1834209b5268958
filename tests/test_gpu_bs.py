"""Braess-Sarazin smoother (Sec. 3.3.2) on the GPU against the oracle, through the C ABI.

S = C + B A^{-1} B^T per saddle level within 1e-12 relative (Frobenius); one
smoothing step and one preconditioner application within 1e-10 relative (the
bounds of the other smoothers: FP64 sums in a different order through a few
levels); FGMRES solutions within 1e-7 of the oracle's and iteration counts
within 2.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from fem_inputs import problems as fp
from oracle import amg, saddle

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


def gpu(prob, **kw):
    return B().setup_problem(prob, B().default_options(smoother=B().AMG_SMOOTHER_BS, **kw))


def oracle(prob):
    return amg.build_hierarchy(prob, amg.Options(smoother="bs"))


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


PROBS = {"mixed": lambda: fp.mixed_elasticity_problem(4, nu=0.49, seed=5),
         "mixed_jittered": lambda: fp.mixed_elasticity_family(5, [0.4999], seed=3)[0],
         "stokes": lambda: fp.stokes_lid_problem(4)}


@pytest.mark.parametrize("kind", sorted(PROBS))
def test_schur_matrices_match_oracle(kind):
    prob = PROBS[kind]()
    h = gpu(prob)
    oh = oracle(prob)
    assert h.n_levels == len(oh.levels)
    for l in range(len(oh.levels) - 1):
        want = oh.levels[l].extra["bs"]["S"][0]
        rp = h.level_array(l, "s_rowptr")
        got = sp.csr_matrix((h.level_array(l, "s_val"), h.level_array(l, "s_col"), rp),
                            shape=want.shape)
        assert np.all(np.diff(rp) > 0)
        assert sp.linalg.norm(got - want) <= 1e-12 * sp.linalg.norm(want), l
    h.free()


@pytest.mark.parametrize("kind", ["mixed", "mixed_jittered"])
def test_bs_step_matches_oracle(kind):
    prob = PROBS[kind]()
    h = gpu(prob)
    oh = oracle(prob)
    rng = np.random.default_rng(2)
    x0 = rng.standard_normal(prob.n_dof)
    b = rng.standard_normal(prob.n_dof)
    xg = cuda(x0)
    h.level_smooth(0, xg, cuda(b))
    want = saddle.smooth(oh, 0, x0, b, post=False)
    got = xg.cpu().numpy()
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)
    h.free()


@pytest.mark.parametrize("cluster_from,cycle_kernel", [(0, 1), (1, 1), (0, 2), (-1, 0)])
def test_bs_preconditioner_matches_oracle(cluster_from, cycle_kernel):
    prob = PROBS["mixed"]()
    h = gpu(prob, cluster_from=cluster_from, cycle_kernel=cycle_kernel)
    oh = oracle(prob)
    r = np.random.default_rng(3).standard_normal(prob.n_dof)
    z = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
    h.apply_preconditioner(cuda(r), z)
    want = amg.precondition(oh, r)
    assert np.linalg.norm(z.cpu().numpy() - want) <= 1e-10 * np.linalg.norm(want)
    h.free()


@pytest.mark.parametrize("kind", ["mixed", "stokes"])
def test_bs_fgmres_matches_oracle(kind):
    prob = PROBS[kind]()
    h = gpu(prob)
    b = cuda(prob.rhs())
    x = torch.zeros_like(b)
    st = h.solve(b, x, 1e-10, device_ptrs=True)
    xv = x.cpu().numpy()
    ref, oh = amg.solve(prob, amg.Options(smoother="bs"), tol=1e-10)
    assert st.converged and st.true_rel_residual <= 1e-9
    assert abs(st.iterations - ref.iterations) <= 2, (st.iterations, ref.iterations)
    n3 = 3 * prob.n_nodes
    assert np.linalg.norm(xv[:n3] - ref.x[:n3]) <= 1e-7 * np.linalg.norm(ref.x[:n3])
    h.free()


def test_bs_fp32_cycle():
    prob = fp.mixed_elasticity_problem(5, nu=0.499, seed=5)
    h = gpu(prob, precision=B().AMG_FP32)
    b = cuda(prob.rhs())
    x = torch.zeros_like(b)
    st = h.solve(b, x, 1e-8, device_ptrs=True)
    assert st.converged and st.true_rel_residual <= 1.5e-8
    sg = B().setup_problem(prob, B().default_options(precision=B().AMG_FP32))
    st_sgs = sg.solve(b, torch.zeros_like(b), 1e-8, device_ptrs=True)
    print(f"\nBS {st.iterations} iterations, sGS {st_sgs.iterations}")
    h.free()
    sg.free()


# --------------------------------------------------------------------------- Vanka

def vanka(prob, **kw):
    return B().setup_problem(prob, B().default_options(smoother=B().AMG_SMOOTHER_VANKA, **kw))


@pytest.mark.parametrize("kind", ["mixed", "mixed_jittered", "stokes"])
def test_vanka_step_matches_oracle(kind):
    prob = PROBS[kind]()
    h = vanka(prob)
    oh = amg.build_hierarchy(prob, amg.Options(smoother="vanka"))
    rng = np.random.default_rng(4)
    x0 = rng.standard_normal(prob.n_dof)
    b = rng.standard_normal(prob.n_dof)
    for post in (False, True):
        xg = cuda(x0)
        h.level_smooth(0, xg, cuda(b), post=post)
        want = saddle.smooth(oh, 0, x0, b, post=post)
        got = xg.cpu().numpy()
        assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want), post
    h.free()


def test_vanka_preconditioner_matches_oracle():
    prob = PROBS["mixed"]()
    h = vanka(prob)
    oh = amg.build_hierarchy(prob, amg.Options(smoother="vanka"))
    r = np.random.default_rng(3).standard_normal(prob.n_dof)
    z = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
    h.apply_preconditioner(cuda(r), z)
    want = amg.precondition(oh, r)
    assert np.linalg.norm(z.cpu().numpy() - want) <= 1e-10 * np.linalg.norm(want)
    h.free()


@pytest.mark.parametrize("kind", ["mixed", "stokes"])
def test_vanka_fgmres_matches_oracle(kind):
    prob = PROBS[kind]()
    h = vanka(prob)
    b = cuda(prob.rhs())
    x = torch.zeros_like(b)
    st = h.solve(b, x, 1e-10, device_ptrs=True)
    xv = x.cpu().numpy()
    ref, _ = amg.solve(prob, amg.Options(smoother="vanka"), tol=1e-10)
    assert st.converged and st.true_rel_residual <= 1e-9
    assert abs(st.iterations - ref.iterations) <= 2, (st.iterations, ref.iterations)
    n3 = 3 * prob.n_nodes
    assert np.linalg.norm(xv[:n3] - ref.x[:n3]) <= 1e-7 * np.linalg.norm(ref.x[:n3])
    h.free()


def test_vanka_fp32_cycle():
    prob = fp.mixed_elasticity_problem(5, nu=0.499, seed=5)
    h = vanka(prob, precision=B().AMG_FP32)
    b = cuda(prob.rhs())
    x = torch.zeros_like(b)
    st = h.solve(b, x, 1e-8, device_ptrs=True)
    assert st.converged and st.true_rel_residual <= 1.5e-8
    print(f"\nVanka FP32 cycle: {st.iterations} iterations")
    h.free()
