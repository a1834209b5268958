"""The allocation-free preconditioner entry point, for callers that cannot allocate
device memory during a call (stream capture in global mode, frameworks whose
allocator already owns the device memory, latency-bound loops).

amg_apply_preconditioner_noalloc must give the result of amg_apply_preconditioner
on two consecutive calls (its static staging array keeps the previous call's
contents, which must not leak into the next result), and must refuse problems
larger than its staging array.  This file is collected last so that a run that
stops at the first failure has already run every other test; it also passes on
its own in a fresh process.
"""
import numpy as np
import pytest

from fem_inputs import problems as fp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _binding():
    from paper_1503_01287_gb300 import binding
    return binding


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_allocating_entry_point(precision):
    B = _binding()
    prob = fp.elasticity_problem(8, seed=2)
    h = B.setup_problem(prob, B.default_options(precision=precision))
    rng = np.random.default_rng(11)
    for call in range(2):            # two calls in a row share the static array
        r = torch.from_numpy(rng.standard_normal(prob.n_dof)).cuda()
        z_ref = torch.zeros_like(r)
        z = torch.full_like(r, float("nan"))
        h.apply_preconditioner(r, z_ref)
        h.apply_preconditioner_noalloc(r, z)
        zr, zn = z_ref.cpu().numpy(), z.cpu().numpy()
        assert np.all(np.isfinite(zn)), call
        assert np.linalg.norm(zn - zr) <= 1e-12 * np.linalg.norm(zr), call
    h.free()


def test_noalloc_rejects_problems_beyond_its_array():
    B = _binding()
    prob = fp.elasticity_problem(35, seed=2)      # 4 * n_nodes > 1,310,720
    assert 4 * prob.n_nodes > 1310720
    h = B.setup_problem(prob, B.default_options(precision=1))
    r = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    with pytest.raises(B.AmgError) as e:
        h.apply_preconditioner_noalloc(r, z)
    assert e.value.code == -1 and "1310720" in str(e.value)
    h.free()
