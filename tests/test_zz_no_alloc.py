"""The allocation-free preconditioner entry point.

amg_apply_preconditioner_noalloc serves callers that cannot let a library call
allocate device memory: applications whose framework allocator already holds
nearly all of the device memory, and loops with a latency budget in which
cudaMalloc / cudaFree may synchronise the whole device.  It stages its vectors
in a static device array of the library instead of buffers of the handle.

It must give the result of amg_apply_preconditioner on two consecutive calls
(the static array keeps the previous call's contents, which must not leak into
the next result), in both FP64 cycle variants (per-operation launches and the
persistent cycle kernel, which copies through the level's own vectors) and for
the saddle layout with its pressure block; its repeated calls must leave the
device's free memory unchanged; and it must refuse problems larger than its
array.  This file is collected last so that a run that stops at the first
failure has already run every other test; it also passes on its own in a fresh
process.
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


PROBLEMS = {
    "elasticity": lambda: fp.elasticity_problem(8, seed=2),
    "mixed": lambda: fp.mixed_elasticity_problem(4, nu=0.49, seed=5),
    "stokes": lambda: fp.stokes_lid_problem(4),
}


@pytest.mark.parametrize("kind,precision,cycle_kernel", [
    ("elasticity", 0, 1), ("elasticity", 0, 2), ("elasticity", 1, 1), ("elasticity", 1, 2),
    ("mixed", 0, 1), ("mixed", 1, 2), ("stokes", 0, 2),
])
def test_noalloc_matches_allocating_entry_point(kind, precision, cycle_kernel):
    B = _binding()
    prob = PROBLEMS[kind]()
    h = B.setup_problem(prob, B.default_options(precision=precision, cycle_kernel=cycle_kernel))
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


def test_noalloc_leaves_free_device_memory_unchanged():
    """20^3 elasticity: each staged vector holds 4 * 68,921 doubles (2.2 MB), more
    than the granularity at which cudaMemGetInfo reports free memory.  Repeated
    calls must not change it; the allocating entry point's first call, which
    allocates its two staging vectors, must (a check that the measurement sees
    allocations of this size)."""
    B = _binding()
    prob = fp.elasticity_problem(20, seed=3)
    h = B.setup_problem(prob, B.default_options(precision=1))
    rng = np.random.default_rng(12)
    rs = [torch.from_numpy(rng.standard_normal(prob.n_dof)).cuda() for _ in range(3)]
    zs = [torch.zeros_like(rs[0]) for _ in range(3)]
    z_ref = torch.zeros_like(rs[0])
    h.apply_preconditioner_noalloc(rs[0], zs[0])   # first call: looks up the array's address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for r, z in zip(rs, zs):
        h.apply_preconditioner_noalloc(r, z)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    h.apply_preconditioner(rs[2], z_ref)           # allocates 2 x (4 n_nodes) doubles
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    assert free0 - free2 >= 2 * 4 * prob.n_nodes * 8 * 0.9, (free0, free2)
    zr, zn = z_ref.cpu().numpy(), zs[2].cpu().numpy()
    assert np.linalg.norm(zn - zr) <= 1e-12 * np.linalg.norm(zr)
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
