"""Host-side checks of the C-ABI library: it builds, loads, exports every entry
point declared in include/amgp2.h, and its structs have the layout the binding
assumes.  No GPU work."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "amgp2.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(amg_\w+)\(", txt, re.M)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1503_01287_gb300 import binding
    return binding.load_library()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    from paper_1503_01287_gb300 import binding
    assert sorted(binding.EXPORTED) == names


def test_struct_layout_matches_header(lib):
    """Compile a C program against the header and compare sizeof/offsetof with ctypes."""
    from paper_1503_01287_gb300 import binding as B
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "amgp2.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(amg_matrix), sizeof(amg_options), sizeof(amg_stats),
         sizeof(amg_level_info));
  printf("%zu %zu %zu %zu\n", offsetof(amg_matrix, device_ptrs), offsetof(amg_options, omega_p),
         offsetof(amg_stats, level_colours), offsetof(amg_options, cycle_kernel));
  printf("%zu %zu %d %d %d\n", sizeof(amg_learned), offsetof(amg_learned, probe_iterations_learned),
         AMG_N_FEATURES, AMG_MLP_INPUTS, AMG_MLP_NPARAM);
  printf("%.17g %.17g %d %.17g %.17g %d %.17g %.17g %d\n", AMG_WS_MIN, AMG_WS_MAX, AMG_GRID_NWS,
         AMG_WC_MIN, AMG_WC_MAX, AMG_GRID_NWC, AMG_WP_LOG2_MIN, AMG_WP_LOG2_MAX, AMG_GRID_NWP);
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(v) for v in out[:13]]
    grid = [float(v) for v in out[13:]]
    assert sizes[0] == ctypes.sizeof(B.AmgMatrix)
    assert sizes[1] == ctypes.sizeof(B.AmgOptions)
    assert sizes[2] == ctypes.sizeof(B.AmgStats)
    assert sizes[3] == ctypes.sizeof(B.AmgLevelInfo)
    assert sizes[4] == B.AmgMatrix.device_ptrs.offset
    assert sizes[5] == B.AmgOptions.omega_p.offset
    assert sizes[6] == B.AmgStats.level_colours.offset
    assert sizes[7] == B.AmgOptions.cycle_kernel.offset
    assert sizes[8] == ctypes.sizeof(B.AmgLearned)
    assert sizes[9] == B.AmgLearned.probe_iterations_learned.offset
    assert sizes[10:13] == [B.N_FEATURES, B.MLP_INPUTS, B.MLP_NPARAM]
    assert grid == [*B.WS_RANGE, B.GRID[0], *B.WC_RANGE, B.GRID[1], *B.WP_LOG2_RANGE, B.GRID[2]]
    # inputs = features + (ws, wc, log2 wp); parameter count of 16 -> 64 -> 64 -> 1
    assert B.MLP_INPUTS == B.N_FEATURES + 3
    assert B.MLP_NPARAM == 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1


def test_default_options(lib):
    from paper_1503_01287_gb300 import binding as B
    o = B.default_options()
    assert (o.m_pre, o.m_post, o.nu, o.cycles, o.max_levels, o.coarse_dofs) == (1, 1, 1, 1, 5, 300)
    assert o.omega == 0.5 and o.omega_p == 0.125 and o.separate == 1


def test_setup_rejects_bad_arguments_without_gpu(lib):
    """Argument validation happens before any CUDA call."""
    from paper_1503_01287_gb300 import binding as B
    h = ctypes.c_void_p()
    rc = lib.amg_setup(None, None, 1, None, None, ctypes.byref(h))
    assert rc == -1 and not h.value
    assert b"null" in lib.amg_last_error(None)
    assert lib.amg_solve(None, None, None, 1e-8, 0, None) == -1
    lib.amg_free(None)   # NULL-safe
    assert B.AMG_OK == 0
    assert lib.amg_features(None, None) == -1
    assert lib.amg_set_weights(None, None) == -1
    assert lib.amg_learn_weights(None, None, None) == -1
    assert lib.amg_mlp_forward(None, None, -1, None, None) == -1
    assert lib.amg_mlp_adam(None, None, None, None, 0, 0.0, None) == -1
