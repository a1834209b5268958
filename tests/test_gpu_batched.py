"""Batched multi-right-hand-side solves (amg_solve_batched) against single solves
and a sparse direct solve: uneven problems, 1..16 right-hand sides, FP32 and
FP64 cycles, all problems in one graph launch."""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

from fem_inputs import problems as fp

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


def _problems():
    return [fp.elasticity_problem(4, seed=1, nu=0.3),
            fp.elasticity_problem((5, 7, 4), seed=2, lengths=(1.0, 2.5, 3.0), nu=0.42),
            fp.elasticity_problem(6, seed=3, nu=0.25, n_rhs=5, traction="gaussian")]


def _rhs(prob, k, rng):
    """k right-hand sides of the problem: its own load(s) then seeded Gaussian ones
    (zero on Dirichlet nodes)."""
    n3 = 3 * prob.n_nodes
    d = np.repeat((prob.tags & fp.TAG_DIRICHLET) != 0, 3)
    out = np.zeros((k, n3))
    f = prob.f.reshape(-1, n3) if prob.f.ndim == 3 else prob.f.reshape(1, n3)
    for r in range(k):
        out[r] = f[r] if r < len(f) else rng.standard_normal(n3)
        out[r][d] = 0.0
    return out


@pytest.mark.parametrize("precision,k,tile,pair", [
    (0, 5, -1, 1), (1, 5, -1, 1), (1, 16, -1, 1), (1, 1, -1, 1), (1, 5, 0, 1), (1, 5, 1, 1),
    (1, 5, 2, 1), (1, 5, 3, 1), (0, 3, 1, 1), (0, 3, 3, 1), (1, 5, -1, 0), (1, 16, 3, 0),
    (1, 5, 4, 1), (1, 16, 5, 1), (1, 5, 6, 1), (1, 16, 7, 1), (0, 3, 5, 1), (0, 16, 6, 1)])
def test_batched_matches_single_and_direct(precision, k, tile, pair):
    """tile -1: the SpMM tile chosen per level by timing, the colour kernel's the same; 0..7: the
    colour kernel's tile forced (4..7: 4 or 8 lane groups a row, combined through
    shared memory), the SpMM's tile t mod 4.  pair: with the FP32 cycle, the operator
    products in FP32 pairs (1) or FP64 (0)."""
    probs = _problems()
    rng = np.random.default_rng(7)
    handles, Bs, Xs, rhs = [], [], [], []
    for p in probs:
        h = B().setup_problem(p, B().default_options(precision=precision, batch_tile=tile,
                                                     outer_pair=pair))
        r = _rhs(p, k, rng)
        if k >= 3:
            r[2] = 0.0                       # a zero right-hand side converges at once
        handles.append(h)
        rhs.append(r)
        Bs.append(torch.from_numpy(r.ravel()).cuda())
        Xs.append(torch.zeros(k * 3 * p.n_nodes, dtype=torch.float64, device="cuda"))
    rc, stats = B().solve_batched(handles, Bs, Xs, k, 1e-8)
    assert rc == 0
    for p, h, r, X, st in zip(probs, handles, rhs, Xs, stats):
        A = p.a_scipy().tocsc()
        x = X.cpu().numpy().reshape(k, -1)
        for j in range(k):
            nb = np.linalg.norm(r[j])
            if nb == 0:
                assert np.all(x[j] == 0)
                continue
            assert np.linalg.norm(r[j] - A @ x[j]) <= 1.5e-8 * nb
            xd = spl.spsolve(A, r[j])
            assert np.linalg.norm(x[j] - xd) <= 1e-5 * np.linalg.norm(xd)
        assert st.true_rel_residual <= 1.5e-8 and st.converged
        # the same right-hand side through amg_solve
        b0 = torch.from_numpy(np.ascontiguousarray(r[0])).cuda()
        x0 = torch.zeros_like(b0)
        s1 = h.solve(b0, x0, 1e-8, device_ptrs=True)
        # the batch loop runs until its slowest right-hand side has converged
        assert st.iterations >= s1.iterations - 1
        if precision == 0:
            assert np.linalg.norm(x0.cpu().numpy() - x[0]) <= 1e-7 * np.linalg.norm(x[0])


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_matches_oracle_per_rhs(precision):
    """Every right-hand side of the batch against the oracle's solve of the same
    system and right-hand side at the same tolerance (FP64 cycle: PCG; FP32 cycle:
    flexible CG, as the batched path runs per right-hand side).  A right-hand side
    whose residual reaches the tolerance one iteration apart from the oracle's
    (rounding decides the crossing) differs from it by one step of the iteration, so
    the check is: the GPU solution's error against the converged solution (oracle,
    1e-13) is at most twice the oracle's own error at 1e-8, plus 1e-12."""
    from oracle import amg
    probs = _problems()
    k = 4
    rng = np.random.default_rng(17)
    handles, Bs, Xs, rhs = [], [], [], []
    for p in probs:
        h = B().setup_problem(p, B().default_options(precision=precision))
        r = _rhs(p, k, rng)
        handles.append(h)
        rhs.append(r)
        Bs.append(torch.from_numpy(r.ravel()).cuda())
        Xs.append(torch.zeros(k * 3 * p.n_nodes, dtype=torch.float64, device="cuda"))
    rc, stats = B().solve_batched(handles, Bs, Xs, k, 1e-8)
    assert rc == 0
    for p, r, X in zip(probs, rhs, Xs):
        oh = amg.build_hierarchy(p)
        x = X.cpu().numpy().reshape(k, -1)
        for j in range(k):
            K, M = amg.operator(oh, 0), (lambda v: amg.precondition(oh, v))
            ref = amg.pcg(K, M, r[j], 1e-8, flexible=precision == 1)
            conv = amg.pcg(K, M, r[j], 1e-13)
            assert ref.converged and conv.converged
            e_or = np.linalg.norm(ref.x - conv.x)
            e_gpu = np.linalg.norm(x[j] - conv.x)
            assert e_gpu <= 2 * e_or + 1e-12 * np.linalg.norm(conv.x), (p.name, j, e_gpu, e_or)


@pytest.mark.slow
def test_batched_workload_sample_matches_oracle():
    """Problems of the 64 x 16 batched workload at their full sizes: problem 20
    (24^3 cubes, 1.5e5 nodes) and problem 11 (10^3 cubes, aspect ratio 3.3, the
    slowest to converge), each with its 16 Gaussian traction loads, in one batched
    FP32-cycle solve.  Every right-hand side's FP64 residual is recomputed; right-
    hand sides of both problems are compared with the oracle's flexible CG, by the
    criterion of the small-problem test (error against the converged solution at
    most twice the oracle's own error at 1e-8)."""
    from fem_inputs import configs
    from oracle import amg
    specs = configs.batched_specs(64, seed=4)
    picks = [20, 11]
    probs = [fp.elasticity_problem(specs[i]["n"], seed=specs[i]["seed"], nu=specs[i]["nu"],
                                   lengths=specs[i]["lengths"], n_rhs=16, traction="gaussian")
             for i in picks]
    handles, Bs, Xs, F = [], [], [], []
    for p in probs:
        handles.append(B().setup_problem(p, B().default_options(precision=1)))
        f = np.ascontiguousarray(p.f.reshape(16, -1))
        F.append(f)
        Bs.append(torch.from_numpy(f.ravel().copy()).cuda())
        Xs.append(torch.zeros(16 * 3 * p.n_nodes, dtype=torch.float64, device="cuda"))
    rc, stats = B().solve_batched(handles, Bs, Xs, 16, 1e-8)
    assert rc == 0
    for k, (p, f, X) in enumerate(zip(probs, F, Xs)):
        A = p.a_scipy().tocsr()
        x = X.cpu().numpy().reshape(16, -1)
        for j in range(16):
            assert np.linalg.norm(f[j] - A @ x[j]) <= 1.5e-8 * np.linalg.norm(f[j]), (k, j)
        oh = amg.build_hierarchy(p)
        K, M = amg.operator(oh, 0), (lambda v: amg.precondition(oh, v))
        for j in ((0,) if k == 0 else (0, 15)):
            ref = amg.pcg(K, M, f[j], 1e-8, flexible=True)
            conv = amg.pcg(K, M, f[j], 1e-13)
            e_or = np.linalg.norm(ref.x - conv.x)
            e_gpu = np.linalg.norm(x[j] - conv.x)
            assert e_gpu <= 2 * e_or + 1e-12 * np.linalg.norm(conv.x), (picks[k], j, e_gpu, e_or)
    for h in handles:
        h.free()


def test_batched_rejects_a_repeated_handle():
    """Each problem runs on its own handle's stream and work vectors: a handle listed
    twice would race with itself, so the call refuses it before any launch."""
    p = fp.elasticity_problem(4, seed=1, nu=0.3)
    h = B().setup_problem(p, B().default_options(precision=1))
    b = torch.from_numpy(np.ascontiguousarray(p.f.reshape(-1))).cuda()
    xs = [torch.zeros(3 * p.n_nodes, dtype=torch.float64, device="cuda") for _ in range(2)]
    with pytest.raises(B().AmgError) as ei:
        B().solve_batched([h, h], [b, b], xs, 1, 1e-8)
    assert ei.value.code == -1                # AMG_ERR_INVALID
    # the handle still works
    rc, st = B().solve_batched([h], [b], xs[:1], 1, 1e-8)
    assert rc == 0 and st[0].converged
    h.free()


def test_batched_rejects_tile_out_of_range():
    p = fp.elasticity_problem(4, seed=1, nu=0.3)
    h = B().setup_problem(p, B().default_options(precision=1, batch_tile=8))
    b = torch.from_numpy(np.ascontiguousarray(p.f.reshape(-1))).cuda()
    x = torch.zeros(3 * p.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(B().AmgError):
        B().solve_batched([h], [b], [x], 1, 1e-8)
    h.free()
