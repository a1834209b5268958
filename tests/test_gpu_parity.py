"""GPU path vs CPU oracle, through the C ABI.

Bit-exact: C/F splits, prolongation patterns and weights, coarse patterns,
colourings.  Floating point: Galerkin values and FP64 operator applications
within 1e-12 relative (per entry, relative to |A||x|); smoothing sweeps and
preconditioner applications within 1e-10; final FP64 solutions within 1e-9
relative.  FP32 tolerances follow from float rounding: each of the <= ~200
products of a row is rounded once (2^-24) plus the accumulation, bounded here
by 2e-5 relative to |A||x|.
"""
import numpy as np
import pytest

from fem_inputs import problems as fp
from oracle import amg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from parity_helpers import STATE, check_hierarchy, coarse_check  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def B():
    from paper_1503_01287_gb300 import binding
    return binding


def gpu(prob, **opts):
    o = B().default_options(**opts)
    return B().setup_problem(prob, o)


def oracle_opts(prob, **kw):
    sm = kw.pop("smoother", None)
    if sm is None:
        sm = "sgs" if prob.saddle else "gs"
    return amg.Options(smoother=sm, **kw)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


# --------------------------------------------------------------------------- setup parity

@pytest.mark.parametrize("maker", [
    lambda: fp.vector_laplace_problem(4, seed=0),
    lambda: fp.elasticity_problem(6, seed=1),
    lambda: fp.elasticity_problem((5, 7, 4), seed=2, lengths=(1.0, 2.5, 3.0), nu=0.4),
    lambda: fp.elasticity_quadratic_problem(5, seed=2, jitter=0.2),
])
def test_hierarchy_matches_oracle(maker):
    prob = maker()
    h = gpu(prob)
    oh = amg.build_hierarchy(prob, oracle_opts(prob))
    check_hierarchy(h, oh)
    coarse_check(h, oh)


def test_nonseparating_hierarchy_matches_oracle():
    prob = fp.elasticity_problem(6, seed=1)
    h = gpu(prob, separate=0)
    oh = amg.build_hierarchy(prob, oracle_opts(prob, separate=False))
    check_hierarchy(h, oh)


@pytest.mark.parametrize("maker", [
    lambda: fp.mixed_elasticity_problem(4, nu=0.49, seed=5),
    lambda: fp.stokes_lid_problem(4),
])
def test_saddle_hierarchy_matches_oracle(maker):
    prob = maker()
    h = gpu(prob)
    oh = amg.build_hierarchy(prob, oracle_opts(prob))
    check_hierarchy(h, oh)
    coarse_check(h, oh)


# --------------------------------------------------------------------------- kernels

def _abs_bound(A, x):
    return abs(A) @ np.abs(x)


@pytest.mark.parametrize("n", [6, 10])
def test_operator_apply_fp64_and_fp32(n):
    prob = fp.elasticity_problem(n, seed=3)
    h = gpu(prob, precision=B().AMG_FP32)
    oh = amg.build_hierarchy(prob, oracle_opts(prob))
    rng = np.random.default_rng(n)
    for l, lv in enumerate(oh.levels):
        x = rng.standard_normal(3 * lv.n)
        y = torch.zeros(3 * lv.n, dtype=torch.float64, device="cuda")
        h.level_apply(l, cuda(x), y, B().AMG_FP64)
        want = lv.A @ x
        bound = _abs_bound(lv.A, x)
        assert np.all(np.abs(y.cpu().numpy() - want) <= 1e-12 * bound + 1e-300)
        h.level_apply(l, cuda(x), y, B().AMG_FP32)
        assert np.all(np.abs(y.cpu().numpy() - want) <= 2e-5 * bound + 1e-30)


@pytest.mark.parametrize("smoother", ["gs", "jacobi"])
def test_smoothing_sweep_matches_oracle(smoother):
    prob = fp.elasticity_problem(7, seed=4)
    code = {"gs": B().AMG_SMOOTHER_GS, "jacobi": B().AMG_SMOOTHER_JACOBI}[smoother]
    h = gpu(prob, smoother=code)
    oh = amg.build_hierarchy(prob, oracle_opts(prob, smoother=smoother))
    rng = np.random.default_rng(1)
    for l in range(len(oh.levels) - 1):
        lv = oh.levels[l]
        for post in (False, True):
            x0 = rng.standard_normal(3 * lv.n)
            b = rng.standard_normal(3 * lv.n)
            xg = cuda(x0)
            h.level_smooth(l, xg, cuda(b), post=post)
            if smoother == "gs":
                want = amg.gs_sweep(lv, x0, b, reverse=post)
            else:
                want = amg.jacobi_sweep(lv, x0, b, 0.5)
            got = xg.cpu().numpy()
            assert np.all(np.abs(got - want) <= 1e-11 * np.abs(want).max()), (l, post)


@pytest.mark.parametrize("kind,cluster_from,cycle_kernel", [
    ("elasticity", 0, 1), ("elasticity", 1, 1), ("elasticity", 2, 1), ("elasticity", 0, 2),
    ("laplace", -1, 0), ("laplace", 1, 1), ("laplace", 0, 2),
    ("mixed", 0, 1), ("mixed", 1, 1), ("mixed", 0, 2), ("stokes", 0, 1), ("stokes", 1, 1),
    ("stokes", 0, 2)])
def test_preconditioner_matches_oracle(kind, cluster_from, cycle_kernel):
    """One preconditioner application.  cluster_from: from which level the cycle
    runs as one thread-block-cluster launch (0: one launch per operation);
    cycle_kernel 2: the whole cycle as one persistent launch."""
    prob = {"elasticity": lambda: fp.elasticity_problem(8, seed=7),
            "laplace": lambda: fp.vector_laplace_problem(5, seed=1),
            "mixed": lambda: fp.mixed_elasticity_problem(4, nu=0.49, seed=5),
            "stokes": lambda: fp.stokes_lid_problem(4)}[kind]()
    h = gpu(prob, cluster_from=cluster_from, cycle_kernel=cycle_kernel)
    oh = amg.build_hierarchy(prob, oracle_opts(prob))
    if kind == "stokes":
        # the singular Galerkin Stokes coarsest matrix: the GPU's generalised inverse
        # must give the oracle's own complete-pivot solution (same tie rule)
        coarse_check(h, oh)
    r = np.random.default_rng(3).standard_normal(prob.n_dof)
    z = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
    h.apply_preconditioner(cuda(r), z)
    want = amg.precondition(oh, r)
    got = z.cpu().numpy()
    assert np.all(np.abs(got - want) <= 1e-10 * np.abs(want).max())


# --------------------------------------------------------------------------- full solves

def _solve(h, prob, tol):
    b = cuda(prob.rhs())
    x = torch.zeros_like(b)
    st = h.solve(b, x, tol, device_ptrs=True)
    return st, x.cpu().numpy()


def test_solve_vector_laplace_workload():
    """The 4^3 vector-Laplacian workload: AMG-PCG to 1e-10, exact quadratic solution."""
    prob = fp.vector_laplace_problem(4, seed=0)
    h = gpu(prob)
    st, x = _solve(h, prob, 1e-10)
    ref, _ = amg.solve(prob, tol=1e-10)
    assert st.converged and st.true_rel_residual <= 1e-10 * 1.5
    assert abs(st.iterations - ref.iterations) <= 1
    assert np.linalg.norm(x - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    u = x.reshape(-1, 3) + prob.lift
    assert np.abs(u - prob.exact_u).max() <= 1e-8 * np.abs(prob.exact_u).max()


@pytest.mark.parametrize("opts,okw", [
    ({}, {}),
    ({"cluster_from": 0}, {}),
    ({"cluster_from": 1, "nu": 2}, {"nu": 2}),
    ({"cluster_from": 2, "smoother": 1}, {"smoother": "jacobi"}),
    ({"cycle_kernel": 2}, {}),
    ({"cycle_kernel": 2, "nu": 2, "m_pre": 2, "m_post": 2}, {"nu": 2, "m_pre": 2, "m_post": 2}),
    ({"smoother": 1}, {"smoother": "jacobi"}),
    ({"nu": 2}, {"nu": 2}),
    ({"m_pre": 2, "m_post": 2}, {"m_pre": 2, "m_post": 2}),
    ({"cycles": 2}, {"cycles": 2}),
    ({"separate": 0}, {"separate": False}),
])
def test_pcg_fp64_matches_oracle(opts, okw):
    prob = fp.elasticity_problem(8, seed=1)
    h = gpu(prob, **opts)
    st, x = _solve(h, prob, 1e-10)
    ref, _ = amg.solve(prob, oracle_opts(prob, **okw), tol=1e-10)
    assert st.converged
    assert abs(st.iterations - ref.iterations) <= 1, (st.iterations, ref.iterations)
    assert np.linalg.norm(x - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    d = (prob.tags & fp.TAG_DIRICHLET) != 0
    assert np.all(x.reshape(-1, 3)[d] == 0.0)


@pytest.mark.parametrize("kind,opts", [
    ("laplace", {}), ("elasticity", {}), ("elasticity", {"cycle_kernel": 2}),
    ("elasticity", {"cluster_from": 1}), ("elasticity", {"m_pre": 2, "m_post": 2}),
    ("laplace", {"post_order": 0}), ("mixed", {}),
])
def test_standalone_amg_matches_oracle(kind, opts):
    """The stand-alone AMG iteration (Sec. 4.2): by default its post-smoothing sweeps
    the colours in the pre-smoothing order (post_order 0 forces the reversed order)."""
    prob = {"laplace": lambda: fp.vector_laplace_problem(6, seed=2),
            "elasticity": lambda: fp.elasticity_problem(6, seed=4),
            # the stand-alone sGS iteration diverges on the random-traction mixed
            # problems (in the oracle too); the Sec. 4.1 mixed setting converges
            "mixed": lambda: fp.paper_setting_problem("mixed", 4)}[kind]()
    h = gpu(prob, krylov=B().AMG_KRYLOV_NONE, max_iterations=400, **opts)
    st, x = _solve(h, prob, 1e-8)
    okw = {k: v for k, v in opts.items() if k in ("m_pre", "m_post")}
    order = "reverse" if opts.get("post_order") == 0 else "same"
    ref, _ = amg.solve(prob, oracle_opts(prob, post_order=order, **okw), tol=1e-8,
                       method="amg", maxit=400)
    assert st.converged and ref.converged
    assert abs(st.iterations - ref.iterations) <= 1, (st.iterations, ref.iterations)
    assert np.linalg.norm(x - ref.x) <= 1e-7 * np.linalg.norm(ref.x)


@pytest.mark.parametrize("opts", [{}, {"cycle_kernel": 2}, {"cluster_from": 1},
                                  {"gs_cluster": 1}, {"nu": 2, "m_pre": 2, "m_post": 2}])
def test_preconditioner_same_post_order_matches_oracle(opts):
    """One cycle with post_order = 1 (post-smoothing colours ascending) in every cycle
    variant, entry by entry against the oracle."""
    prob = fp.elasticity_problem(7, seed=9)
    h = gpu(prob, post_order=1, **opts)
    okw = {k: v for k, v in opts.items() if k in ("nu", "m_pre", "m_post")}
    oh = amg.build_hierarchy(prob, oracle_opts(prob, post_order="same", **okw))
    r = np.random.default_rng(8).standard_normal(prob.n_dof)
    z = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
    h.apply_preconditioner(cuda(r), z)
    want = amg.precondition(oh, r)
    got = z.cpu().numpy()
    assert np.all(np.abs(got - want) <= 1e-10 * np.abs(want).max())


@pytest.mark.parametrize("cluster_from,cycle_kernel", [(0, 1), (1, 1), (2, 1), (0, 2)])
def test_fp32_cycle_flexible_cg(cluster_from, cycle_kernel):
    prob = fp.elasticity_problem(10, seed=1)
    h = gpu(prob, precision=B().AMG_FP32, cluster_from=cluster_from, cycle_kernel=cycle_kernel)
    st, x = _solve(h, prob, 1e-8)
    assert st.converged and st.true_rel_residual <= 1.5e-8
    # against the FP64 oracle's flexible CG to the same tolerance: the FP32 cycle
    # (with the FP32-pair operator) follows the FP64 iteration to about 1e-12 (4e-13
    # to 7e-13 measured at 8^3-16^3) when both stop at the same iteration
    ref8, _ = amg.solve(prob, tol=1e-8, method="fcg")
    assert abs(st.iterations - ref8.iterations) <= 1, (st.iterations, ref8.iterations)
    err = np.linalg.norm(x - ref8.x) / np.linalg.norm(ref8.x)
    if st.iterations == ref8.iterations:
        assert err <= 1e-10, err
    else:      # one iteration apart: the difference is one step of the iteration
        ref12, _ = amg.solve(prob, tol=1e-13)
        e_or = np.linalg.norm(ref8.x - ref12.x)
        assert np.linalg.norm(x - ref12.x) <= 2 * e_or + 1e-12 * np.linalg.norm(ref12.x)


@pytest.mark.parametrize("kind", ["mixed", "stokes"])
def test_saddle_fgmres_matches_oracle(kind):
    prob = (fp.mixed_elasticity_problem(4, nu=0.49, seed=5) if kind == "mixed"
            else fp.stokes_lid_problem(4))
    h = gpu(prob)
    st, x = _solve(h, prob, 1e-10)
    ref, oh = amg.solve(prob, tol=1e-10)
    assert st.converged and st.true_rel_residual <= 1e-9
    assert abs(st.iterations - ref.iterations) <= 2, (st.iterations, ref.iterations)
    from oracle import saddle as sd
    K0 = oh.levels[0]
    nb = np.linalg.norm(prob.rhs())
    assert np.linalg.norm(sd.apply_K(K0, x) - prob.rhs()) <= 1.5e-10 * nb
    if kind == "mixed":
        assert np.linalg.norm(x - ref.x) <= 1e-7 * np.linalg.norm(ref.x)
    else:
        n3 = 3 * prob.n_nodes
        assert np.linalg.norm(x[:n3] - ref.x[:n3]) <= 1e-7 * np.linalg.norm(ref.x[:n3])
        assert abs(prob.p_weights @ x[n3:]) <= 1e-12 * np.abs(x[n3:]).max() * prob.n_pres


@pytest.mark.parametrize("cycle_kernel", [1, 2])
def test_fp32_saddle(cycle_kernel):
    prob = fp.mixed_elasticity_problem(5, nu=0.499, seed=5)
    h = gpu(prob, precision=B().AMG_FP32, cycle_kernel=cycle_kernel)
    st, x = _solve(h, prob, 1e-8)
    assert st.converged and st.true_rel_residual <= 1.5e-8


# --------------------------------------------------------------------------- full size

@pytest.mark.slow
def test_full_size_elasticity_32():
    """The 32^3 elasticity workload (823,875 DOF) in the launch configuration the
    bench times: coarsening, prolongation and colouring bit-exact on levels 0-1,
    sampled Galerkin blocks, and the solve checked by its recomputed residual."""
    prob = fp.elasticity_problem(32, seed=1)
    h = gpu(prob, precision=B().AMG_FP32)
    oo = oracle_opts(prob)
    lv0 = amg.Level(prob.n_nodes, prob.a_rowptr, prob.a_col, np.array(prob.a_val), prob.tags)
    lv0.A = amg.scalar_view(lv0.rowptr, lv0.col, lv0.val, lv0.n)
    lv1 = amg.coarsen_level(lv0, oo)
    assert np.array_equal(h.level_array(0, "cf_state"), np.vectorize(STATE.get)(lv0.state))
    assert np.array_equal(h.level_array(0, "p_col"), lv0.P_structure.tocsr().indices)
    assert np.array_equal(h.level_array(1, "a_rowptr"), lv1.rowptr)
    assert np.array_equal(h.level_array(1, "a_col"), lv1.col)
    v1 = h.level_array(1, "a_val").reshape(-1, 3, 3)
    idx = np.random.default_rng(0).choice(len(lv1.col), 20000, replace=False)
    assert np.abs(v1[idx] - lv1.val[idx]).max() <= 1e-12 * np.abs(lv1.val).max()
    col0 = amg.greedy_colouring(amg.block_pattern(lv0.rowptr, lv0.col, lv0.n))
    assert np.array_equal(h.level_array(0, "colour"), col0)
    st, x = _solve(h, prob, 1e-8)
    assert st.converged
    A = prob.a_scipy().tocsr()
    b = prob.rhs()
    assert np.linalg.norm(b - A @ x) <= 1.5e-8 * np.linalg.norm(b)


@pytest.mark.slow
def test_full_size_elasticity_32_solution_matches_oracle():
    """The 32^3 elasticity workload solved by the oracle on the host (FP64 AMG-PCG,
    1e-8) and on the GPU in the bench's two arms: the plain FP64 PCG within 1e-9 of
    the oracle's solution, and the chosen FP32-cycle flexible CG with the FP32-pair
    operator within 1e-9 as well (both follow the oracle's iteration, which stops
    at the same count)."""
    prob = fp.elasticity_problem(32, seed=1)
    ref, _ = amg.solve(prob, tol=1e-8)
    assert ref.converged
    for precision in (B().AMG_FP64, B().AMG_FP32):
        h = gpu(prob, precision=precision)
        st, x = _solve(h, prob, 1e-8)
        assert st.converged and abs(st.iterations - ref.iterations) <= 1
        err = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
        assert err <= 1e-9, (precision, err)
        h.free()


def _sweep_row_scale(lv, x, b):
    """|D_i^-1| (|b_i| + sum_j |A_ij| |x_j|) per unknown: the size of the terms a
    row update combines, the scale of its rounding error."""
    t = np.abs(b) + abs(lv.A) @ np.abs(x)
    return np.einsum("nij,nj->ni", np.abs(lv.dinv), t.reshape(-1, 3)).ravel()


@pytest.mark.slow
def test_full_size_sweeps_match_oracle_entrywise():
    """The 32^3 elasticity workload in the bench's configuration (FP32 cycle, launch
    variants chosen by the setup's timing): one sweep of every level in both colour
    orders, with the FP32 kernels the solves run and with the FP64 kernels, against
    the oracle's sweep entry by entry.  FP64: every unknown within 1e-12 of its
    row's own scale |D_i^-1| (|b_i| + sum |A_ij| |x_j|).  FP32: every unknown within
    1e-4 of the largest entry, the bound of the other FP32-cycle tests (float
    rounding of the values, the iterate and ~30 products per row is about 1e-6 of a
    row's scale, but it reaches a row also from neighbours of larger scale through
    the earlier colours: 3e-4 of the row's own scale was measured at one unknown)."""
    prob = fp.elasticity_problem(32, seed=1)
    h = gpu(prob, precision=B().AMG_FP32)
    oh = amg.build_hierarchy(prob)
    rng = np.random.default_rng(32)
    for l in range(len(oh.levels) - 1):
        lv = oh.levels[l]
        for post in (False, True):
            x0 = rng.standard_normal(3 * lv.n)
            b = rng.standard_normal(3 * lv.n)
            want = amg.gs_sweep(lv, x0, b, reverse=post)
            scale = _sweep_row_scale(lv, want, b) + 1e-300
            for prec in (B().AMG_FP64, B().AMG_FP32):
                xg = cuda(x0)
                h.level_smooth(l, xg, cuda(b), post=post, precision=prec)
                diff = np.abs(xg.cpu().numpy() - want)
                rel_row = (diff / scale).max()
                if prec == B().AMG_FP64:
                    assert rel_row <= 1e-12, (l, post, rel_row)
                else:
                    rel_max = diff.max() / np.abs(want).max()
                    assert rel_max <= 1e-4, (l, post, rel_max, rel_row)
    # one FP32 preconditioner application, entry by entry
    r = rng.standard_normal(prob.n_dof)
    z = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
    h.apply_preconditioner(cuda(r), z)
    want = amg.precondition(oh, r)
    assert np.all(np.abs(z.cpu().numpy() - want) <= 1e-4 * np.abs(want).max())


# --------------------------------------------------------------------------- errors

def test_invalid_inputs_are_rejected():
    prob = fp.elasticity_problem(2, seed=1)
    bad = fp.elasticity_problem(2, seed=1)
    bad.a_col = bad.a_col.copy()
    bad.a_col[[0, 1]] = bad.a_col[[1, 0]]          # unsorted row
    with pytest.raises(B().AmgError) as e:
        gpu(bad)
    assert e.value.code == -1
    bad = fp.elasticity_problem(2, seed=1)
    bad.a_val = bad.a_val.copy()
    bad.a_val[5, 1, 1] = np.nan
    with pytest.raises(B().AmgError):
        gpu(bad)
    h = gpu(prob, max_iterations=2)
    st, x = _solve(h, prob, 1e-14)
    assert not st.converged and st.iterations == 2 and np.all(np.isfinite(x))
    b = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
    x = torch.ones_like(b)
    st = h.solve(b, x, 1e-8, device_ptrs=True)
    assert st.iterations == 0 and torch.all(x == 0)


def test_host_pointer_solve_matches_device():
    prob = fp.elasticity_problem(6, seed=1)
    h = gpu(prob)
    st_d, xd = _solve(h, prob, 1e-9)
    xh = np.zeros(prob.n_dof)
    st_h = h.solve(np.ascontiguousarray(prob.rhs()), xh, 1e-9, device_ptrs=False)
    assert st_h.iterations == st_d.iterations
    assert np.array_equal(xh, xd)
