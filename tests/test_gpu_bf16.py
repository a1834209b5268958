"""AMG_FP32_BF16: the FP32 cycle with the operator values of levels >= 1 stored in
BF16, through the C ABI.

Parity: one preconditioner application against the FP64 oracle whose level >= 1
operators are rounded to BF16 the way the library rounds them (nearest even,
directly from the FP64 Galerkin values), D^{-1} and the transfers left exact:
both sides then multiply the same operator values and the difference is the
FP32 arithmetic of the cycle, bounded here by 1e-4 relative (each level pass
rounds every product once, 2^-24, and the cycle chains ~10 passes and the
D^{-1} applications).  Against the unrounded oracle the same application must
differ by far more, which shows the BF16 values are the ones used.
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


def bf16_from_f64(a):
    """Nearest BF16 value (8 significant bits, ties to even) of FP64 values."""
    u = np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)
    lsb = (u >> np.uint64(45)) & np.uint64(1)
    u = (u + np.uint64((1 << 44) - 1) + lsb) & ~np.uint64((1 << 45) - 1)
    return u.view(np.float64)


def _round_coarse(oh):
    for lv in oh.levels[1:]:
        lv.A = lv.A.copy()
        lv.A.data = bf16_from_f64(lv.A.data)
        if lv.colour_rows is not None:
            lv.colour_A = [lv.A[(3 * rows[:, None] + np.arange(3)).ravel()]
                           for rows in lv.colour_rows]


def test_bf16_rounding_helper():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -40, -3.14159])
    assert list(bf16_from_f64(x)) == [1.0, 1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7, -3.140625]


@pytest.mark.parametrize("kind", ["elasticity", "laplace"])
def test_bf16_preconditioner_matches_rounded_oracle(kind):
    prob = (fp.elasticity_problem(8, seed=7) if kind == "elasticity"
            else fp.vector_laplace_problem(6, seed=1))
    h = B().setup_problem(prob, B().default_options(precision=B().AMG_FP32_BF16))
    assert h.n_levels >= 3
    r = np.random.default_rng(3).standard_normal(prob.n_dof)
    z = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
    h.apply_preconditioner(torch.from_numpy(r).cuda(), z)
    got = z.cpu().numpy()
    exact = amg.precondition(amg.build_hierarchy(prob), r)
    oh = amg.build_hierarchy(prob)
    _round_coarse(oh)
    want = amg.precondition(oh, r)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    err_exact = np.linalg.norm(got - exact) / np.linalg.norm(exact)
    assert err <= 1e-4, err
    assert err_exact >= 10 * err, (err, err_exact)
    h.free()


@pytest.mark.parametrize("kind", ["elasticity", "mixed"])
def test_bf16_solve_converges(kind):
    prob = (fp.elasticity_problem(16, seed=1) if kind == "elasticity"
            else fp.mixed_elasticity_problem(6, nu=0.49, seed=5))
    b = torch.from_numpy(prob.rhs()).cuda()
    out = {}
    for prec in (B().AMG_FP32, B().AMG_FP32_BF16):
        h = B().setup_problem(prob, B().default_options(precision=prec))
        x = torch.zeros_like(b)
        st = h.solve(b, x, 1e-8, device_ptrs=True)
        assert st.converged and st.true_rel_residual <= 1.5e-8
        out[prec] = st.iterations
        h.free()
    print(f"\nFP32 {out[B().AMG_FP32]} iterations, FP32 with BF16 coarse values "
          f"{out[B().AMG_FP32_BF16]}")
    assert out[B().AMG_FP32_BF16] <= out[B().AMG_FP32] + 5
