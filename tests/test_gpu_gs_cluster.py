"""The multicolour Gauss-Seidel sweep of a small level as one launch (a CTA, or a
thread-block cluster whose CTAs exchange new values by st.async counted on an
mbarrier a colour; x, b and the row offsets in shared memory), through the C ABI.

The sweep computes what the one-launch-per-colour chain computes (Sec. 3.3, the
block Gauss-Seidel smoother in colour order, colours descending after the coarse
correction), so the bounds are those of the other sweep tests: one FP64 sweep of
every eligible level within 1e-11 of the oracle's, one FP64 preconditioner
application (which also takes the zero-initial-guess form of the kernel) within
1e-10, FP32 cycles within the FP32 bound of the cycle and converged solves.  Every
cluster size is forced in turn; the stats show which levels took the kernel.
"""
import numpy as np
import pytest

from fem_inputs import problems as fp
from oracle import amg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [1, 2, 4, 8, 16]


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


def _levels_used(h, prob):
    b = cuda(prob.rhs())
    st = h.solve(b, torch.zeros_like(b), 1e-8, device_ptrs=True)
    assert st.converged and st.true_rel_residual <= 1.5e-8
    return st.as_dict()["level_gs_cluster"]


@pytest.mark.parametrize("cs", SIZES)
def test_cluster_sweep_matches_oracle(cs):
    prob = fp.elasticity_problem(6, seed=4)
    h = B().setup_problem(prob, B().default_options(gs_cluster=cs))
    oh = amg.build_hierarchy(prob)
    used = _levels_used(h, prob)
    # 6^3 cubes: level 0 has 2197 nodes (x and b 70 KB each in FP64), so every
    # coloured level fits; a cluster size the device cannot hold leaves 0
    coloured = [l for l in range(len(oh.levels) - 1)]
    assert all(used[l] in (0, cs) for l in coloured)
    if cs <= 8:                                   # portable cluster sizes
        assert all(used[l] == cs for l in coloured), used
    rng = np.random.default_rng(1)
    for l in coloured:
        lv = oh.levels[l]
        for post in (False, True):
            x0 = rng.standard_normal(3 * lv.n)
            b = rng.standard_normal(3 * lv.n)
            xg = cuda(x0)
            h.level_smooth(l, xg, cuda(b), post=post)
            want = amg.gs_sweep(lv, x0, b, reverse=post)
            got = xg.cpu().numpy()
            assert np.linalg.norm(got - want) <= 1e-11 * np.linalg.norm(want), (l, post)
    h.free()


@pytest.mark.parametrize("kind,cs", [("elasticity", 1), ("elasticity", 4), ("elasticity", 16),
                                     ("laplace", 2), ("laplace", 8)])
def test_cluster_preconditioner_matches_oracle(kind, cs):
    prob = (fp.elasticity_problem(8, seed=7) if kind == "elasticity"
            else fp.vector_laplace_problem(5, seed=1))
    h = B().setup_problem(prob, B().default_options(gs_cluster=cs, cluster_from=0,
                                                    cycle_kernel=1))
    used = _levels_used(h, prob)
    assert any(u > 0 for u in used) or cs == 16
    oh = amg.build_hierarchy(prob)
    r = np.random.default_rng(3).standard_normal(prob.n_dof)
    z = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
    h.apply_preconditioner(cuda(r), z)
    want = amg.precondition(oh, r)
    assert np.linalg.norm(z.cpu().numpy() - want) <= 1e-10 * np.linalg.norm(want)
    h.free()


@pytest.mark.parametrize("precision", ["fp32", "fp32_bf16"])
@pytest.mark.parametrize("cs", [1, 8])
def test_cluster_fp32_cycle(precision, cs):
    """The FP32 cycle (FP32 iterate in shared memory; BF16 operator values on the
    coarse levels) against the FP64 oracle's preconditioner, and its solve."""
    prec = {"fp32": B().AMG_FP32, "fp32_bf16": B().AMG_FP32_BF16}[precision]
    prob = fp.elasticity_problem(12, seed=2)
    h = B().setup_problem(prob, B().default_options(precision=prec, gs_cluster=cs,
                                                    cluster_from=0, cycle_kernel=1))
    used = _levels_used(h, prob)
    assert sum(u == cs for u in used) >= 2, used
    if precision == "fp32":
        ref = B().setup_problem(prob, B().default_options(precision=prec, gs_cluster=0,
                                                          cluster_from=0, cycle_kernel=1))
        r = np.random.default_rng(5).standard_normal(prob.n_dof)
        z = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
        zr = torch.zeros_like(z)
        h.apply_preconditioner(cuda(r), z)
        ref.apply_preconditioner(cuda(r), zr)
        want = amg.precondition(amg.build_hierarchy(prob), r)
        # both FP32 cycles sit within the FP32 bound of the FP64 result ...
        for got in (z, zr):
            assert np.linalg.norm(got.cpu().numpy() - want) <= 1e-4 * np.linalg.norm(want)
        # ... and the two kernels differ only in the order of FP32 sums
        assert torch.linalg.norm(z - zr) <= 1e-5 * torch.linalg.norm(zr)
        ref.free()
    h.free()


def test_timed_choice_and_invalid_size():
    prob = fp.elasticity_problem(8, seed=7)
    h = B().setup_problem(prob, B().default_options(precision=B().AMG_FP32))
    used = _levels_used(h, prob)
    assert all(u in (0, 1, 2, 4, 8, 16) for u in used)
    h.free()
    for bad in (3, 32, -2):
        with pytest.raises(B().AmgError) as e:
            B().setup_problem(prob, B().default_options(gs_cluster=bad))
        assert e.value.code == -1
