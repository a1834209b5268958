"""ctypes binding of the amgp2 C ABI (include/amgp2.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts numpy /
torch buffers into the plain pointers and sizes the C entry points take.  If
the library is missing the import of the native symbols fails loudly: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libamgp2.so")

# enums (include/amgp2.h)
AMG_VECTOR_LAPLACE, AMG_ELASTICITY, AMG_MIXED_ELASTICITY, AMG_STOKES = 0, 1, 2, 3
AMG_SMOOTHER_GS, AMG_SMOOTHER_JACOBI, AMG_SMOOTHER_SGS, AMG_SMOOTHER_BS, AMG_SMOOTHER_VANKA = (
    0, 1, 2, 3, 4)
AMG_FP64, AMG_FP32, AMG_FP32_BF16, AMG_FP32_PAIR = 0, 1, 2, 3
AMG_KRYLOV_AUTO, AMG_KRYLOV_PCG, AMG_KRYLOV_FCG, AMG_KRYLOV_FGMRES, AMG_KRYLOV_NONE = 0, 1, 2, 3, 4
AMG_OK, AMG_NOT_CONVERGED = 0, 1
AMG_MAX_LEVELS = 8

ITEMS = {
    "a_rowptr": (0, np.int32), "a_col": (1, np.int32), "a_val": (2, np.float64),
    "tags": (3, np.int32), "cf_state": (4, np.int32), "p_rowptr": (5, np.int32),
    "p_col": (6, np.int32), "p_val": (7, np.float64), "colour": (8, np.int32),
    "dinv": (9, np.float64), "b_rowptr": (10, np.int32), "b_col": (11, np.int32),
    "b_val": (12, np.float64), "c_rowptr": (13, np.int32), "c_col": (14, np.int32),
    "c_val": (15, np.float64), "pcf_state": (16, np.int32), "h_rowptr": (17, np.int32),
    "h_col": (18, np.int32), "h_val": (19, np.float64), "coarse_inv": (20, np.float64),
    "s_rowptr": (21, np.int32), "s_col": (22, np.int32), "s_val": (23, np.float64),
}

KINDS = {"laplace": AMG_VECTOR_LAPLACE, "elasticity": AMG_ELASTICITY,
         "mixed": AMG_MIXED_ELASTICITY, "stokes": AMG_STOKES}

EXPORTED = ["amg_default_options", "amg_setup", "amg_solve", "amg_free", "amg_last_error",
            "amg_level_info_get", "amg_level_copy", "amg_apply_preconditioner",
            "amg_level_apply", "amg_level_smooth", "amg_level_smooth_precision",
            "amg_set_pressure_weights",
            "amg_time_level_op", "amg_solve_batched", "amg_apply_preconditioner_noalloc",
            "amg_features", "amg_set_weights", "amg_get_weights", "amg_learn_weights",
            "amg_level_features", "amg_set_level_weights",
            "amg_mlp_forward", "amg_mlp_gradient", "amg_mlp_adam", "amg_mlp_backward"]

N_FEATURES = 13
MLP_INPUTS = 16
MLP_NPARAM = 5313
# candidate grid of amg_learn_weights (the header's AMG_WS_* / AMG_WC_* / AMG_WP_* values)
WS_RANGE, WC_RANGE, WP_LOG2_RANGE = (0.6, 1.6), (0.8, 1.9), (-1.0, 2.0)
GRID = (11, 12, 7)

OPS = {"apply": 0, "residual": 1, "smooth": 2, "restrict": 3, "prolong": 4, "precond": 5}


class AmgMatrix(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_pres", C.c_int32), ("nnzb", C.c_int64),
                ("a_rowptr", C.c_void_p), ("a_col", C.c_void_p), ("a_val", C.c_void_p),
                ("b_nnz", C.c_int64), ("b_rowptr", C.c_void_p), ("b_col", C.c_void_p),
                ("b_val", C.c_void_p), ("c_nnz", C.c_int64), ("c_rowptr", C.c_void_p),
                ("c_col", C.c_void_p), ("c_val", C.c_void_p), ("device_ptrs", C.c_int32)]


class AmgOptions(C.Structure):
    _fields_ = [("smoother", C.c_int32), ("m_pre", C.c_int32), ("m_post", C.c_int32),
                ("nu", C.c_int32), ("cycles", C.c_int32), ("precision", C.c_int32),
                ("krylov", C.c_int32), ("max_levels", C.c_int32), ("coarse_dofs", C.c_int32),
                ("gmres_restart", C.c_int32), ("separate", C.c_int32),
                ("max_iterations", C.c_int32), ("use_graphs", C.c_int32),
                ("cluster_from", C.c_int32), ("cycle_kernel", C.c_int32),
                ("omega", C.c_double), ("omega_p", C.c_double),
                ("batch_tile", C.c_int32), ("gs_cluster", C.c_int32),
                ("outer_pair", C.c_int32), ("post_order", C.c_int32),
                ("gs_flow", C.c_int32), ("gs_stream", C.c_int32), ("gs_tma", C.c_int32)]


class AmgStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("n_levels", C.c_int32),
                ("pad0", C.c_int32), ("rel_residual", C.c_double),
                ("true_rel_residual", C.c_double), ("setup_ms", C.c_double),
                ("solve_ms", C.c_double), ("kernel_launches", C.c_int64),
                ("level_nodes", C.c_int32 * AMG_MAX_LEVELS),
                ("level_pres", C.c_int32 * AMG_MAX_LEVELS),
                ("level_nnzb", C.c_int64 * AMG_MAX_LEVELS),
                ("level_colours", C.c_int32 * AMG_MAX_LEVELS),
                ("level_group", C.c_int32 * AMG_MAX_LEVELS),
                ("cluster_from", C.c_int32), ("cycle_kernel", C.c_int32),
                ("level_gs_cluster", C.c_int32 * AMG_MAX_LEVELS),
                ("level_gs_flow", C.c_int32 * AMG_MAX_LEVELS),
                ("level_gs_stream", C.c_int32 * AMG_MAX_LEVELS),
                ("level_gs_tma", C.c_int32 * AMG_MAX_LEVELS)]

    def as_dict(self) -> dict:
        nl = self.n_levels
        return {"iterations": self.iterations, "converged": bool(self.converged),
                "n_levels": nl, "rel_residual": self.rel_residual,
                "true_rel_residual": self.true_rel_residual, "setup_ms": self.setup_ms,
                "solve_ms": self.solve_ms, "kernel_launches": self.kernel_launches,
                "level_nodes": list(self.level_nodes[:nl]),
                "level_pres": list(self.level_pres[:nl]),
                "level_nnzb": list(self.level_nnzb[:nl]),
                "level_colours": list(self.level_colours[:nl]),
                "level_group": list(self.level_group[:nl]),
                "cluster_from": self.cluster_from, "cycle_kernel": self.cycle_kernel,
                "level_gs_cluster": list(self.level_gs_cluster[:nl]),
                "level_gs_flow": list(self.level_gs_flow[:nl]),
                "level_gs_stream": list(self.level_gs_stream[:nl]),
                "level_gs_tma": list(self.level_gs_tma[:nl])}


class AmgLearned(C.Structure):
    _fields_ = [("weights", C.c_double * 3), ("predicted", C.c_double),
                ("rho_plain", C.c_double), ("rho_learned", C.c_double),
                ("fell_back", C.c_int32), ("n_candidates", C.c_int32),
                ("probe_iterations_plain", C.c_int32), ("probe_iterations_learned", C.c_int32),
                ("level_weights", C.c_double * (3 * AMG_MAX_LEVELS)),
                ("level_predicted", C.c_double * AMG_MAX_LEVELS),
                ("n_levels", C.c_int32), ("pad0", C.c_int32)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "pad0"}
        d["weights"] = list(self.weights)
        nl = self.n_levels
        d["level_weights"] = [list(self.level_weights[3 * l:3 * l + 3]) for l in range(nl)]
        d["level_predicted"] = list(self.level_predicted[:nl])
        return d


class AmgLevelInfo(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_pres", C.c_int32), ("nnzb", C.c_int64),
                ("p_nnz", C.c_int64), ("h_nnz", C.c_int64), ("b_nnz", C.c_int64),
                ("c_nnz", C.c_int64), ("n_colours", C.c_int32), ("is_coarsest", C.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load libamgp2.so (build it with paper_1503_01287_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    lib.amg_default_options.argtypes = [C.POINTER(AmgOptions)]
    lib.amg_default_options.restype = None
    lib.amg_setup.argtypes = [C.POINTER(AmgMatrix), vp, i32, C.POINTER(AmgOptions), vp,
                              C.POINTER(vp)]
    lib.amg_setup.restype = C.c_int
    lib.amg_solve.argtypes = [vp, vp, vp, dbl, i32, C.POINTER(AmgStats)]
    lib.amg_solve.restype = C.c_int
    lib.amg_free.argtypes = [vp]
    lib.amg_free.restype = None
    lib.amg_last_error.argtypes = [vp]
    lib.amg_last_error.restype = C.c_char_p
    lib.amg_level_info_get.argtypes = [vp, i32, C.POINTER(AmgLevelInfo)]
    lib.amg_level_info_get.restype = C.c_int
    lib.amg_level_copy.argtypes = [vp, i32, i32, vp, i64]
    lib.amg_level_copy.restype = C.c_int
    lib.amg_apply_preconditioner.argtypes = [vp, vp, vp]
    lib.amg_apply_preconditioner.restype = C.c_int
    lib.amg_level_apply.argtypes = [vp, i32, i32, vp, vp]
    lib.amg_level_apply.restype = C.c_int
    lib.amg_level_smooth.argtypes = [vp, i32, i32, vp, vp]
    lib.amg_level_smooth.restype = C.c_int
    lib.amg_level_smooth_precision.argtypes = [vp, i32, i32, i32, vp, vp]
    lib.amg_level_smooth_precision.restype = C.c_int
    lib.amg_set_pressure_weights.argtypes = [vp, vp, i32]
    lib.amg_set_pressure_weights.restype = C.c_int
    lib.amg_time_level_op.argtypes = [vp, i32, i32, i32, i32, i32, C.POINTER(dbl),
                                      C.POINTER(i32)]
    lib.amg_time_level_op.restype = C.c_int
    lib.amg_solve_batched.argtypes = [C.POINTER(vp), i32, i32, C.POINTER(vp), C.POINTER(vp), dbl,
                                      C.POINTER(AmgStats)]
    lib.amg_solve_batched.restype = C.c_int
    lib.amg_apply_preconditioner_noalloc.argtypes = [vp, vp, vp]
    lib.amg_apply_preconditioner_noalloc.restype = C.c_int
    lib.amg_features.argtypes = [vp, vp]
    lib.amg_features.restype = C.c_int
    lib.amg_set_weights.argtypes = [vp, vp]
    lib.amg_set_weights.restype = C.c_int
    lib.amg_level_features.argtypes = [vp, i32, vp]
    lib.amg_level_features.restype = C.c_int
    lib.amg_set_level_weights.argtypes = [vp, vp, i32]
    lib.amg_set_level_weights.restype = C.c_int
    lib.amg_get_weights.argtypes = [vp, vp, i32]
    lib.amg_get_weights.restype = C.c_int
    lib.amg_learn_weights.argtypes = [vp, vp, C.POINTER(AmgLearned)]
    lib.amg_learn_weights.restype = C.c_int
    lib.amg_mlp_forward.argtypes = [vp, vp, i32, vp, vp]
    lib.amg_mlp_forward.restype = C.c_int
    lib.amg_mlp_gradient.argtypes = [vp, vp, vp, i32, vp, vp, vp]
    lib.amg_mlp_gradient.restype = C.c_int
    lib.amg_mlp_backward.argtypes = [vp, vp, vp, i32, vp, vp]
    lib.amg_mlp_backward.restype = C.c_int
    lib.amg_mlp_adam.argtypes = [vp, vp, vp, vp, i32, C.c_float, vp]
    lib.amg_mlp_adam.restype = C.c_int
    _lib = lib
    return lib


class AmgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"amgp2 error {code}: {msg}")
        self.code = code


def _check(rc: int, handle=None):
    if rc < 0:
        msg = load_library().amg_last_error(handle)
        raise AmgError(rc, (msg or b"").decode())
    return rc


def default_options(**over) -> AmgOptions:
    o = AmgOptions()
    load_library().amg_default_options(C.byref(o))
    for k, v in over.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr(a):
    """Address of a C-contiguous numpy array or torch tensor (None -> NULL).

    For a CUDA tensor the caller's current stream is synchronised first: the
    library works on its own stream, so work the caller queued on that tensor
    (a fill, a copy) must be complete before the library reads or writes it."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        if a.is_cuda:
            import torch
            torch.cuda.current_stream(a.device).synchronize()
        return a.data_ptr()
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


class Handle:
    """Owns one amg_handle.  Arrays passed in are kept alive only for the call."""

    def __init__(self, a_rowptr, a_col, a_val, tags, kind, options: AmgOptions | None = None,
                 b=None, c=None, stream=None, device_ptrs: bool = False):
        lib = load_library()
        m = AmgMatrix()
        m.n_nodes = len(tags)
        m.nnzb = len(a_col)
        m.a_rowptr, m.a_col, m.a_val = _ptr(a_rowptr), _ptr(a_col), _ptr(a_val)
        if b is not None:
            b_rowptr, b_col, b_val = b
            c_rowptr, c_col, c_val = c
            m.n_pres = len(b_rowptr) - 1
            m.b_nnz, m.b_rowptr, m.b_col, m.b_val = len(b_col), _ptr(b_rowptr), _ptr(b_col), \
                _ptr(b_val)
            m.c_nnz, m.c_rowptr, m.c_col, m.c_val = len(c_col), _ptr(c_rowptr), _ptr(c_col), \
                _ptr(c_val)
        m.device_ptrs = 1 if device_ptrs else 0
        self._keep = (a_rowptr, a_col, a_val, tags, b, c)
        self.kind = KINDS[kind] if isinstance(kind, str) else int(kind)
        self.options = options or default_options()
        h = C.c_void_p()
        rc = lib.amg_setup(C.byref(m), _ptr(tags), self.kind, C.byref(self.options), stream,
                           C.byref(h))
        _check(rc, None)
        self.h = h
        self._keep = None
        self.n_nodes = m.n_nodes
        self.n_pres = m.n_pres

    @property
    def n_dof(self) -> int:
        return 3 * self.n_nodes + self.n_pres

    def free(self):
        if getattr(self, "h", None):
            load_library().amg_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def solve(self, b, x, tol: float, device_ptrs: bool) -> AmgStats:
        st = AmgStats()
        rc = load_library().amg_solve(self.h, _ptr(b), _ptr(x), tol, 1 if device_ptrs else 0,
                                      C.byref(st))
        _check(rc, self.h)
        return st

    def set_pressure_weights(self, w):
        _check(load_library().amg_set_pressure_weights(self.h, _ptr(w), 0), self.h)

    def level_info(self, level: int) -> AmgLevelInfo:
        info = AmgLevelInfo()
        _check(load_library().amg_level_info_get(self.h, level, C.byref(info)), self.h)
        return info

    @property
    def n_levels(self) -> int:
        n = 0
        while True:
            info = AmgLevelInfo()
            if load_library().amg_level_info_get(self.h, n, C.byref(info)) != 0:
                return n
            n += 1

    def level_array(self, level: int, item: str) -> np.ndarray:
        info = self.level_info(level)
        code, dt = ITEMS[item]
        sizes = {
            "a_rowptr": info.n_nodes + 1, "a_col": info.nnzb, "a_val": 9 * info.nnzb,
            "tags": info.n_nodes, "cf_state": info.n_nodes, "p_rowptr": info.n_nodes + 1,
            "p_col": info.p_nnz, "p_val": info.p_nnz, "colour": info.n_nodes,
            "dinv": 9 * info.n_nodes, "b_rowptr": info.n_pres + 1, "b_col": info.b_nnz,
            "b_val": 3 * info.b_nnz, "c_rowptr": info.n_pres + 1, "c_col": info.c_nnz,
            "c_val": info.c_nnz, "pcf_state": info.n_pres, "h_rowptr": info.n_pres + 1,
            "h_col": info.h_nnz, "h_val": info.h_nnz,
            "coarse_inv": (3 * info.n_nodes + info.n_pres) ** 2,
            "s_rowptr": info.n_pres + 1,
        }
        if item in ("s_col", "s_val"):
            sizes[item] = int(self.level_array(level, "s_rowptr")[-1])
        out = np.empty(int(sizes[item]), dtype=dt)
        _check(load_library().amg_level_copy(self.h, level, code, out.ctypes.data, out.nbytes),
               self.h)
        return out

    def apply_preconditioner(self, r_dev, z_dev):
        _check(load_library().amg_apply_preconditioner(self.h, _ptr(r_dev), _ptr(z_dev)), self.h)

    def apply_preconditioner_noalloc(self, r_dev, z_dev):
        """z = M^{-1} r without any device allocation in the call (static staging)."""
        _check(load_library().amg_apply_preconditioner_noalloc(self.h, _ptr(r_dev),
                                                               _ptr(z_dev)), self.h)

    def level_apply(self, level: int, x_dev, y_dev, precision: int = AMG_FP64):
        _check(load_library().amg_level_apply(self.h, level, precision, _ptr(x_dev), _ptr(y_dev)),
               self.h)

    def time_level_op(self, op: str, level: int, precision: int, reps: int = 20,
                      warmup: int = 3):
        """(ms per repetition, kernel launches per repetition) of a level operation."""
        ms = C.c_double()
        nl = C.c_int32()
        _check(load_library().amg_time_level_op(self.h, OPS[op], level, precision, reps, warmup,
                                                C.byref(ms), C.byref(nl)), self.h)
        return ms.value, nl.value

    def level_smooth(self, level: int, x_dev, b_dev, post: bool = False,
                     precision: int | None = None):
        """One sweep (post: colours descending); precision None/AMG_FP64 or AMG_FP32."""
        if precision is None:
            _check(load_library().amg_level_smooth(self.h, level, 1 if post else 0,
                                                   _ptr(x_dev), _ptr(b_dev)), self.h)
        else:
            _check(load_library().amg_level_smooth_precision(
                self.h, level, 1 if post else 0, precision, _ptr(x_dev), _ptr(b_dev)), self.h)

    def features(self) -> np.ndarray:
        """The 13 statistics of the hierarchy that the weight network reads."""
        out = np.zeros(N_FEATURES)
        _check(load_library().amg_features(self.h, out.ctypes.data), self.h)
        return out

    def level_features(self, level: int) -> np.ndarray:
        """amg_level_features: the 13 network inputs of non-coarsest level `level`."""
        out = np.zeros(N_FEATURES, dtype=np.float64)
        _check(load_library().amg_level_features(self.h, level, out.ctypes.data), self.h)
        return out

    def set_level_weights(self, w):
        """amg_set_level_weights with w of shape (n_levels, 3): (ws, wc, wp) per level."""
        w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1, 3)
        _check(load_library().amg_set_level_weights(self.h, w.ctypes.data, len(w)), self.h)

    def set_weights(self, ws: float, wc: float, wp: float = 1.0):
        w = np.array([ws, wc, wp], dtype=np.float64)
        _check(load_library().amg_set_weights(self.h, w.ctypes.data), self.h)

    def weights(self) -> np.ndarray:
        """Per-level (ws, wc, wp, 1) as an (n_levels, 4) array."""
        out = np.zeros((self.n_levels, 4))
        _check(load_library().amg_get_weights(self.h, out.ctypes.data, out.size), self.h)
        return out

    def learn_weights(self, theta) -> AmgLearned:
        """amg_learn_weights with host float32 network parameters."""
        th = np.ascontiguousarray(theta, dtype=np.float32)
        assert th.size == MLP_NPARAM
        res = AmgLearned()
        _check(load_library().amg_learn_weights(self.h, th.ctypes.data, C.byref(res)), self.h)
        return res


def mlp_forward(theta, x, y, stream=None):
    """y[i] = net(theta, x[i]) on device tensors (float32; x of shape (n, 16))."""
    n = int(x.shape[0])
    _check(load_library().amg_mlp_forward(_ptr(theta), _ptr(x), n, _ptr(y), stream))


def mlp_gradient(theta, x, t, grad, loss, stream=None):
    """grad, loss of the mean squared error of the net on (x, t), device tensors."""
    n = int(x.shape[0])
    _check(load_library().amg_mlp_gradient(_ptr(theta), _ptr(x), _ptr(t), n, _ptr(grad),
                                           _ptr(loss), stream))


def mlp_backward(theta, x, dy, grad, stream=None):
    """grad = sum_i dy[i] d net(x[i]) / d theta on device tensors (float32)."""
    n = int(x.shape[0])
    _check(load_library().amg_mlp_backward(_ptr(theta), _ptr(x), _ptr(dy), n, _ptr(grad),
                                           stream))


def mlp_adam(theta, grad, m, v, step: int, lr: float, stream=None):
    _check(load_library().amg_mlp_adam(_ptr(theta), _ptr(grad), _ptr(m), _ptr(v), step,
                                       float(lr), stream))


def setup_problem(prob, options: AmgOptions | None = None, stream=None) -> Handle:
    """amg_setup on a fem_inputs.Problem-like object (host arrays)."""
    a_val = np.ascontiguousarray(prob.a_val, dtype=np.float64).reshape(-1)
    args = dict(a_rowptr=np.ascontiguousarray(prob.a_rowptr, dtype=np.int32),
                a_col=np.ascontiguousarray(prob.a_col, dtype=np.int32), a_val=a_val,
                tags=np.ascontiguousarray(prob.tags, dtype=np.int32), kind=prob.kind,
                options=options, stream=stream)
    if prob.kind in ("mixed", "stokes"):
        args["b"] = (np.ascontiguousarray(prob.b_rowptr, dtype=np.int32),
                     np.ascontiguousarray(prob.b_col, dtype=np.int32),
                     np.ascontiguousarray(prob.b_val, dtype=np.float64).reshape(-1))
        args["c"] = (np.ascontiguousarray(prob.c_rowptr, dtype=np.int32),
                     np.ascontiguousarray(prob.c_col, dtype=np.int32),
                     np.ascontiguousarray(prob.c_val, dtype=np.float64))
    h = Handle(**args)
    if prob.kind == "stokes" and getattr(prob, "p_weights", None) is not None:
        h.set_pressure_weights(np.ascontiguousarray(prob.p_weights, dtype=np.float64))
    return h


def solve_batched(handles, B_list, X_list, n_rhs: int, tol: float):
    """amg_solve_batched over device tensors: B_list[p], X_list[p] hold n_rhs vectors of
    3*n_nodes doubles each (vector r at offset r*3*n_nodes).  Returns (rc, [stats])."""
    n = len(handles)
    hs = (C.c_void_p * n)(*[h.h.value for h in handles])
    bs = (C.c_void_p * n)(*[_ptr(b) for b in B_list])
    xs = (C.c_void_p * n)(*[_ptr(x) for x in X_list])
    st = (AmgStats * n)()
    rc = load_library().amg_solve_batched(C.cast(hs, C.POINTER(C.c_void_p)), n, n_rhs,
                                          C.cast(bs, C.POINTER(C.c_void_p)),
                                          C.cast(xs, C.POINTER(C.c_void_p)), tol, st)
    _check(rc, handles[0].h)
    return rc, [st[i] for i in range(n)]
