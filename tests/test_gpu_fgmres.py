"""Flexible GMRES(m) on the GPU (Sec. 4: the accelerator of the saddle-point
systems) against the oracle's FGMRES(m) with the same restart length.

The GPU orthogonalises with delayed reorthogonalisation (each basis vector is
reorthogonalised in the next step's sweep, and the last one before every stop
or restart); the oracle uses modified Gram-Schmidt.  Both build the same Krylov
basis up to rounding, so with the FP64 cycle the iteration counts agree and the
solutions agree to the conditioning of the system.  Short restart lengths make
every restart's finalisation run many times.  The per-step graph (preconditioner,
pressure projection and operator captured once per solve) must give the same
bits as the plain launches.
"""
import numpy as np
import pytest

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


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def make(kind):
    if kind == "elasticity":
        return fp.elasticity_problem(5, seed=3)
    if kind == "stokes":
        return fp.stokes_lid_problem(4)
    return fp.mixed_elasticity_problem(4, nu=0.499, seed=5)


def oracle_fgmres(prob, tol, m):
    if prob.saddle:
        h = amg.build_hierarchy(prob, amg.Options(smoother="sgs"))
        lv0 = h.levels[0]
        K = lambda v: saddle.apply_K(lv0, v)              # noqa: E731
        proj = saddle.pressure_projector(h)
    else:
        h = amg.build_hierarchy(prob)
        A = prob.a_scipy().tocsr()
        K = lambda v: A @ v                               # noqa: E731
        proj = None
    res = amg.fgmres(K, lambda r: amg.precondition(h, r), prob.rhs(), tol, restart=m,
                     maxit=2000, project=proj)
    if proj is not None:
        res.x = proj(res.x)
    return res, K


def gpu_solve(prob, tol, **opts):
    o = dict(krylov=B().AMG_KRYLOV_FGMRES, max_iterations=2000)
    o.update(opts)
    h = B().setup_problem(prob, B().default_options(**o))
    b = cuda(prob.rhs())
    x = torch.zeros_like(b)
    st = h.solve(b, x, tol, device_ptrs=True)
    h.free()
    return st, x.cpu().numpy()


@pytest.mark.parametrize("kind,m", [("elasticity", 5), ("elasticity", 12), ("elasticity", 300),
                                    ("stokes", 5), ("stokes", 12), ("stokes", 300),
                                    ("mixed", 12), ("mixed", 300)])
def test_fgmres_restart_matches_oracle(kind, m):
    prob = make(kind)
    tol = 1e-10
    ref, K = oracle_fgmres(prob, tol, m)
    st, x = gpu_solve(prob, tol, gmres_restart=m)
    assert st.converged and ref.converged
    # rounding differs between the two orthogonalisations: over hundreds of restarted
    # iterations the count may drift by 1%
    assert abs(st.iterations - ref.iterations) <= max(1, ref.iterations // 100), \
        (st.iterations, ref.iterations)
    b = prob.rhs()
    assert np.linalg.norm(b - K(x)) <= 1.5 * tol * np.linalg.norm(b)
    # the estimate the stopping rule used is the true residual up to rounding
    assert abs(st.rel_residual - st.true_rel_residual) <= 1e-3 * tol
    nv = 3 * prob.n_nodes if kind == "stokes" else len(x)   # Stokes: p up to its mean
    assert np.linalg.norm(x[:nv] - ref.x[:nv]) <= 1e-7 * np.linalg.norm(ref.x[:nv])


@pytest.mark.parametrize("kind", ["stokes", "mixed"])
@pytest.mark.parametrize("m", [8, 300])
def test_fgmres_step_graph_is_bitwise_plain(kind, m):
    """FP64 cycle: the graph replays the same kernels on the same data."""
    prob = make(kind)
    st0, x0 = gpu_solve(prob, 1e-9, gmres_restart=m, use_graphs=0)
    st1, x1 = gpu_solve(prob, 1e-9, gmres_restart=m, use_graphs=1)
    assert st0.converged and st1.converged
    assert st0.iterations == st1.iterations
    assert np.array_equal(x0, x1)


@pytest.mark.parametrize("kind", ["stokes", "mixed"])
def test_fgmres_step_graph_fp32(kind):
    """FP32 cycle: each handle picks its colour-kernel lane widths by timing at setup,
    and the widths set the order of a row's float sums, so two handles may round
    differently; one handle repeats its own bits, and the graph and the plain
    launches agree to the FP32 cycle's accuracy."""
    prob = make(kind)
    o = dict(krylov=B().AMG_KRYLOV_FGMRES, precision=1, gmres_restart=300)
    h = B().setup_problem(prob, B().default_options(**o))
    b = cuda(prob.rhs())
    xs = []
    for _ in range(2):
        x = torch.zeros_like(b)
        st = h.solve(b, x, 1e-9, device_ptrs=True)
        assert st.converged
        xs.append(x.cpu().numpy())
    h.free()
    assert np.array_equal(xs[0], xs[1])
    st0, x0 = gpu_solve(prob, 1e-9, precision=1, gmres_restart=300, use_graphs=0)
    assert st0.converged and abs(st0.iterations - st.iterations) <= 1
    nv = 3 * prob.n_nodes if kind == "stokes" else len(x0)
    assert np.linalg.norm(x0[:nv] - xs[0][:nv]) <= 1e-7 * np.linalg.norm(xs[0][:nv])


def test_fgmres_restart_limit_and_iteration_cap():
    """Stopping on the iteration cap in the middle of a restart cycle: the column
    is finalised, the iterate is the minimiser over the basis so far and the
    status says not converged."""
    prob = make("mixed")
    st, x = gpu_solve(prob, 1e-12, gmres_restart=12, max_iterations=17)
    assert not st.converged and st.iterations == 17
    ref, K = oracle_fgmres(prob, 1e-12, 12)
    b = prob.rhs()
    # the oracle's history holds its estimate after each iteration
    assert abs(st.rel_residual - ref.history[17]) <= 1e-6 * ref.history[17]
    assert abs(np.linalg.norm(b - K(x)) / np.linalg.norm(b) - st.rel_residual) \
        <= 1e-6 * st.rel_residual
