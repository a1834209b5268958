"""The FP32-pair Krylov operator of FP32-cycle solves, through the C ABI.

Each FP64 value and vector entry is split into hi + lo floats (to about 2^-48),
each product a_hi x_hi is formed exactly (rounded product plus its FMA error),
the cross terms a_hi x_lo + a_lo x_hi are added and a_lo x_lo (about 2^-48 of
the product) is dropped; the rounded products are summed with TwoSum and the
error terms in a second float.  Per entry the result then lies within a small
multiple of 2^-48 (3.6e-15) of sum_j |a_ij x_j|: the test allows 1e-12 of that
sum, the bound of the FP64 kernel's test, and asks the error to be far below
the plain FP32 kernel's (which carries about 2^-24).  The solves with the pair
operator and with the FP64 operator must reach the same tolerance, verified by
an FP64 residual on the device and again on the host from the oracle's matrix,
in the same number of iterations (+-1).
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


@pytest.mark.parametrize("kind,n", [("elasticity", 6), ("elasticity", 11), ("laplace", 7)])
def test_pair_operator_matches_oracle(kind, n):
    prob = (fp.elasticity_problem(n, seed=3) if kind == "elasticity"
            else fp.vector_laplace_problem(n, seed=2))
    h = B().setup_problem(prob, B().default_options(precision=B().AMG_FP32))
    oh = amg.build_hierarchy(prob)
    A = oh.levels[0].A
    rng = np.random.default_rng(n)
    # scales far from 1 as well: the pair form keeps the relative accuracy
    for scale in (1.0, 1e-20, 3e15):
        x = scale * rng.standard_normal(prob.n_dof)
        want = A @ x
        bound = abs(A) @ np.abs(x)
        y = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
        h.level_apply(0, cuda(x), y, B().AMG_FP32_PAIR)
        err_pair = np.abs(y.cpu().numpy() - want)
        assert np.all(err_pair <= 1e-12 * bound), (err_pair / bound).max()
        h.level_apply(0, cuda(x), y, B().AMG_FP32)
        err_f32 = np.abs(y.cpu().numpy() - want)
        assert (err_pair / bound).max() * 1e5 <= (err_f32 / bound).max()
    h.free()


@pytest.mark.parametrize("kind", ["mixed", "stokes"])
def test_pair_saddle_operator_matches_oracle(kind):
    """Saddle kinds: the velocity block in pairs, B^T p and B u - C p in FP64; per
    entry within 1e-12 of sum_j |k_ij x_j| against the oracle's K."""
    from oracle import saddle
    prob = (fp.mixed_elasticity_problem(5, nu=0.499, seed=5) if kind == "mixed"
            else fp.stokes_lid_problem(5))
    h = B().setup_problem(prob, B().default_options(precision=B().AMG_FP32))
    oh = amg.build_hierarchy(prob, amg.Options(smoother="sgs"))
    lv0 = oh.levels[0]
    import scipy.sparse as sp
    K = sp.bmat([[lv0.A, lv0.B.T], [lv0.B, -lv0.C]]).tocsr()
    rng = np.random.default_rng(3)
    for scale in (1.0, 1e-12, 1e9):
        x = scale * rng.standard_normal(prob.n_dof)
        want = saddle.apply_K(lv0, x)
        bound = abs(K) @ np.abs(x)
        y = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
        h.level_apply(0, cuda(x), y, B().AMG_FP32_PAIR)
        err = np.abs(y.cpu().numpy() - want)
        assert np.all(err <= 1e-12 * bound), (err / np.maximum(bound, 1e-300)).max()
    h.free()


@pytest.mark.parametrize("kind", ["mixed", "stokes"])
def test_pair_saddle_solve_matches_fp64_operator_solve(kind):
    """FGMRES with the FP32 cycle: the pair operator and the FP64 operator reach the
    same tolerance in the same number of iterations (+-1), the FP64 residual checked
    on the host from the oracle's K."""
    from oracle import saddle
    prob = (fp.mixed_elasticity_problem(6, nu=0.49, seed=5) if kind == "mixed"
            else fp.stokes_lid_problem(6))
    b = cuda(prob.rhs())
    out = {}
    for pair in (0, 1):
        h = B().setup_problem(prob, B().default_options(precision=B().AMG_FP32,
                                                        outer_pair=pair))
        x = torch.zeros_like(b)
        st = h.solve(b, x, 1e-10, device_ptrs=True)
        assert st.converged and st.true_rel_residual <= 1.5e-10
        out[pair] = (st.iterations, x.cpu().numpy())
        h.free()
    assert abs(out[0][0] - out[1][0]) <= 1, (out[0][0], out[1][0])
    lv0 = amg.build_hierarchy(prob, amg.Options(smoother="sgs")).levels[0]
    bh = prob.rhs()
    for pair in (0, 1):
        rel = np.linalg.norm(bh - saddle.apply_K(lv0, out[pair][1])) / np.linalg.norm(bh)
        assert rel <= 1.5e-10, (pair, rel)


@pytest.mark.parametrize("kind", ["elasticity", "laplace"])
def test_pair_solve_matches_fp64_operator_solve(kind):
    prob = (fp.elasticity_problem(12, seed=1) if kind == "elasticity"
            else fp.vector_laplace_problem(10, seed=1))
    b = cuda(prob.rhs())
    out = {}
    for pair in (0, 1):
        h = B().setup_problem(prob, B().default_options(precision=B().AMG_FP32,
                                                        outer_pair=pair))
        x = torch.zeros_like(b)
        st = h.solve(b, x, 1e-10, device_ptrs=True)
        assert st.converged and st.true_rel_residual <= 1.5e-10
        out[pair] = (st.iterations, x.cpu().numpy())
        h.free()
    assert abs(out[0][0] - out[1][0]) <= 1, (out[0][0], out[1][0])
    # the residual of both solutions recomputed on the host from the oracle's matrix
    A = amg.build_hierarchy(prob).levels[0].A
    bh = prob.rhs()
    for pair in (0, 1):
        rel = np.linalg.norm(bh - A @ out[pair][1]) / np.linalg.norm(bh)
        assert rel <= 1.5e-10, (pair, rel)


def test_pair_operator_availability():
    prob = fp.elasticity_problem(4, seed=1)
    x = torch.ones(prob.n_dof, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    for opts in ({"precision": B().AMG_FP64}, {"precision": B().AMG_FP32, "outer_pair": 0}):
        h = B().setup_problem(prob, B().default_options(**opts))
        with pytest.raises(B().AmgError):
            h.level_apply(0, x, y, B().AMG_FP32_PAIR)
        h.free()
    h = B().setup_problem(prob, B().default_options(precision=B().AMG_FP32))
    xi = torch.ones(3 * h.level_info(1).n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(B().AmgError):
        h.level_apply(1, xi, torch.zeros_like(xi), B().AMG_FP32_PAIR)
    ms, nl = h.time_level_op("apply", 0, B().AMG_FP32_PAIR, reps=3, warmup=1)
    assert ms > 0 and nl == 1
    h.free()
