"""Python binding of the C ABI in include/fdbem.h (argument marshalling only).

Every entry point has the name of its C function. Device vectors are torch CUDA
tensors (complex128 / complex64, column-major N x nrhs, i.e. shape (nrhs, N)
row-major); streams are torch streams. All arithmetic runs in the CUDA library:
if _libfdbem.so is missing or cannot be loaded this module raises, there is no
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_libfdbem.so")

FDA_OK = 0
FDA_E_INVALID_ARG = -1
FDA_E_OOM = -2
FDA_E_CUDA = -3
FDA_E_NOT_CONVERGED = -4
FDA_E_BREAKDOWN = -5
FDA_E_NAN = -6
FDA_E_TIMEOUT = -7
FDA_E_STATE = -8
FDA_CPLX128 = 0
FDA_CPLX64 = 1
FDA_PREC_FP64 = 0
FDA_PREC_FP32 = 1
FDA_PREC_TF32 = 2


class FdaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class fda_config_t(C.Structure):
    _fields_ = [("eps", C.c_double), ("precision", C.c_int), ("lowrank", C.c_int), ("nrhs_max", C.c_int),
                ("m2l_tensor", C.c_int), ("op", C.c_int), ("near_split", C.c_int),
                ("drop_fp64", C.c_int), ("near_form", C.c_int), ("gamma_re", C.c_double),
                ("gamma_im", C.c_double)]


class bm_gmres_opts_t(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart", C.c_int), ("max_iter", C.c_int), ("x0_given", C.c_int),
                ("refine", C.c_int), ("inner_restart", C.c_int), ("inner_tol", C.c_double),
                ("refine_residual", C.c_int), ("reserved", C.c_int * 5)]


class bm_gmres_stats_t(C.Structure):
    _fields_ = [("iterations", C.c_int), ("outer_iterations", C.c_int), ("rel_residual", C.c_double),
                ("ms_total", C.c_double), ("ms_matvec", C.c_double), ("status", C.c_int),
                ("reserved", C.c_int * 5)]


_i64p = C.POINTER(C.c_int64)
_i32p = C.POINTER(C.c_int32)
_u64p = C.POINTER(C.c_uint64)
_dp = C.POINTER(C.c_double)


class fda_tree_view_t(C.Structure):
    _fields_ = [("n_points", C.c_int64), ("n_boxes", C.c_int64), ("n_levels", C.c_int64), ("n_direct", C.c_int64),
                ("n_m2l", C.c_int64), ("corner", C.c_double * 3), ("side", C.c_double),
                ("perm", _i64p), ("keys", _u64p), ("box_level", _i32p), ("box_ix", _i32p), ("box_iy", _i32p),
                ("box_iz", _i32p), ("box_nchild", _i32p), ("box_leaf", _i32p), ("box_parent", _i64p),
                ("box_child_begin", _i64p), ("box_pbeg", _i64p), ("box_pend", _i64p), ("level_hf", _i32p),
                ("level_T", _i32p), ("level_n", _i32p), ("direct", _i64p), ("m2l_box", _i64p),
                ("m2l_info", _i32p)]


class fda_tune_report_t(C.Structure):
    _fields_ = [("entries", C.c_int32), ("level", C.c_int32 * 64), ("stage", C.c_int32 * 64),
                ("ms_fma", C.c_double * 64), ("ms_tensor", C.c_double * 64), ("chosen", C.c_int32 * 64),
                ("near_ms", C.c_double * 2), ("near_rhs_per_pass", C.c_int32), ("near_split", C.c_int32),
                ("near_split_ms", C.c_double * 2), ("near_window_ms", C.c_double), ("overlap", C.c_int32),
                ("near_evict_first", C.c_int32), ("far_levels_concurrent", C.c_int32),
                ("near_form", C.c_int32), ("schedule_ms", C.c_double * 16),
                ("near_form_ms", (C.c_double * 3) * 3), ("m2l_rechosen", C.c_int32), ("near_slim", C.c_int32),
                ("schedule_slim_ms", C.c_double * 16), ("product_ms", C.c_double), ("near_tc_ms", C.c_double)]


class fda_plan_info_t(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("lmin", C.c_int32), ("precision", C.c_int32), ("lowrank", C.c_int32),
                ("s", C.c_int32 * 32), ("n_equiv", C.c_int32 * 32), ("n_check", C.c_int32 * 32),
                ("n_wedges", C.c_int32 * 32), ("m2l_pairs", C.c_int64 * 32), ("m2l_offsets", C.c_int64 * 32),
                ("m2l_lowrank", C.c_int64 * 32), ("n_leaves", C.c_int64), ("n_direct_blocks", C.c_int64),
                ("near_entries", C.c_int64), ("corr_entries", C.c_int64), ("bytes_near", C.c_double),
                ("bytes_s2m_l2t", C.c_double), ("flops_m2l", C.c_double), ("flops_m2m_l2l", C.c_double),
                ("flops_near", C.c_double), ("device_bytes", C.c_double), ("setup_ms", C.c_double * 8),
                ("launches_per_matvec", C.c_int64), ("m2l_flops_lev", C.c_double * 32),
                ("m2l_op_bytes_lev", C.c_double * 32)]


_LIB = None

# (name, restype, argtypes) of every exported function
_SIGS = [
    ("bm_problem_create", C.c_int, [_dp, C.c_int64, _i32p, C.c_int64, C.c_double, C.c_double, C.c_double,
                                    C.POINTER(C.c_void_p)]),
    ("bm_problem_geometry", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("bm_particles_create", C.c_int, [_dp, _dp, C.c_int64, C.c_double, C.c_double, C.c_double,
                                      C.POINTER(C.c_void_p)]),
    ("bm_rhs_plane_wave", C.c_int, [C.c_void_p, _dp, C.c_int, C.c_void_p, C.c_void_p]),
    ("bm_rhs_plane_wave_noalloc", C.c_int, [C.c_void_p, _dp, C.c_int, C.c_void_p, C.c_void_p]),
    ("bm_problem_destroy", None, [C.c_void_p]),
    ("fda_build_tree", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    ("fda_tree_export", C.c_int, [C.c_void_p, C.POINTER(fda_tree_view_t)]),
    ("fda_tree_destroy", None, [C.c_void_p]),
    ("fda_precompute_translations", C.c_int, [C.c_void_p, C.POINTER(fda_config_t), C.POINTER(C.c_void_p)]),
    ("fda_matvec", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    ("fda_plan_info", C.c_int, [C.c_void_p, C.POINTER(fda_plan_info_t)]),
    ("fda_matvec_graph_create", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                          C.POINTER(C.c_void_p)]),
    ("fda_graph_launch", C.c_int, [C.c_void_p, C.c_void_p]),
    ("fda_plan_check", C.c_int, [C.c_void_p]),
    ("fda_wait_selftest", C.c_int, [C.c_double, C.POINTER(C.c_int)]),
    ("fda_autotune", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(fda_tune_report_t)]),
    ("fda_m2l_force", C.c_int, [C.c_void_p, C.c_int]),
    ("fda_overlap_force", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int]),
    ("fda_graph_nodes", C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    ("fda_graph_destroy", None, [C.c_void_p]),
    ("fda_corrections_export", C.c_int, [C.c_void_p, _i64p, C.c_int64, C.c_int64, _i64p, _i64p, _dp]),
    ("fda_plan_destroy", None, [C.c_void_p]),
    ("bm_gmres_solve", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(bm_gmres_opts_t),
                                 C.POINTER(bm_gmres_stats_t), C.c_void_p]),
    ("fda_matvec_ex", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    ("fda_matvec_phases", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                    _dp]),
    ("fda_device_peaks", C.c_int, [_dp, _dp]),
    ("bm_net_create", C.c_int, [C.c_int, C.c_uint64, C.POINTER(C.c_void_p)]),
    ("bm_net_params", C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(C.c_int)]),
    ("bm_net_destroy", None, [C.c_void_p]),
    ("bm_precond_create", C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    ("bm_precond_destroy", None, [C.c_void_p]),
    ("bm_precond_apply", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("bm_precond_train_step", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                        _dp, C.POINTER(C.c_float), C.c_void_p]),
    ("bm_residual_pair", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p]),
    ("bm_fgmres_solve", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                  C.POINTER(bm_gmres_opts_t), C.POINTER(bm_gmres_stats_t), C.c_void_p]),
    ("fda_tc_selftest", C.c_int, [C.c_int, C.c_int, _dp, C.POINTER(C.c_int)]),
    ("fda_last_error", C.c_char_p, []),
]


def lib():
    """Load the CUDA library (raises if it is missing: there is no CPU path)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} not built; run paper_1311_5202_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(rc: int):
    if rc != FDA_OK:
        raise FdaError(rc, lib().fda_last_error().decode(errors="replace"))
    return rc


def _ptr(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


# ----------------------------------------------------------------------------- raw entry points
def bm_problem_create(nodes, elems, k, alpha=None):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    elems = np.ascontiguousarray(elems, dtype=np.int32)
    if alpha is None:
        alpha = 1j / k
    h = C.c_void_p()
    _check(lib().bm_problem_create(_ptr(nodes), nodes.shape[0], _ptr(elems, C.c_int32), elems.shape[0], float(k),
                                   complex(alpha).real, complex(alpha).imag, C.byref(h)))
    return h


def bm_problem_geometry(prob, x_dev, n_dev, w_dev):
    _check(lib().bm_problem_geometry(prob, x_dev.data_ptr(), n_dev.data_ptr(), w_dev.data_ptr()))


def bm_particles_create(x, n, k, alpha=None):
    """Particle-summation problem: points x (N x 3) with unit normals n (N x 3); alpha defaults to i/k."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    a = complex(1j / k) if alpha is None else complex(alpha)
    h = C.c_void_p()
    _check(lib().bm_particles_create(_ptr(x), _ptr(n), x.shape[0], float(k), a.real, a.imag, C.byref(h)))
    return h


def bm_rhs_plane_wave(prob, dirs, b_dev, stream=None):
    dirs = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
    _check(lib().bm_rhs_plane_wave(prob, _ptr(dirs), dirs.shape[0], C.c_void_p(b_dev.data_ptr()), _stream(stream)))


def bm_rhs_plane_wave_noalloc(prob, dirs, b_dev, stream=None, raise_on_error=True):
    """Plane-wave right-hand side without device allocation (at most 1024 directions per call)."""
    dirs = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
    rc = lib().bm_rhs_plane_wave_noalloc(prob, _ptr(dirs), dirs.shape[0], C.c_void_p(b_dev.data_ptr()),
                                         _stream(stream))
    if raise_on_error:
        _check(rc)
    return rc


def bm_problem_destroy(prob):
    lib().bm_problem_destroy(prob)


def fda_build_tree(prob, leaf_max):
    h = C.c_void_p()
    _check(lib().fda_build_tree(prob, int(leaf_max), C.byref(h)))
    return h


def fda_tree_export(tree) -> dict:
    v = fda_tree_view_t()
    _check(lib().fda_tree_export(tree, C.byref(v)))
    N, nb, nl, nd, nm = v.n_points, v.n_boxes, v.n_levels, v.n_direct, v.n_m2l

    def arr(p, n, dt):
        if n == 0:
            return np.zeros(0, dtype=dt)
        return np.ctypeslib.as_array(p, shape=(n,)).astype(dt, copy=True)

    m2l_info = arr(v.m2l_info, 6 * nm, np.int32).reshape(nm, 6)
    m2l_box = arr(v.m2l_box, 2 * nm, np.int64).reshape(nm, 2)
    return dict(corner=np.array(v.corner[:]), side=v.side, perm=arr(v.perm, N, np.int64),
                keys=arr(v.keys, N, np.uint64), level=arr(v.box_level, nb, np.int32), ix=arr(v.box_ix, nb, np.int32),
                iy=arr(v.box_iy, nb, np.int32), iz=arr(v.box_iz, nb, np.int32),
                nchild=arr(v.box_nchild, nb, np.int32), leaf=arr(v.box_leaf, nb, np.int32),
                parent=arr(v.box_parent, nb, np.int64), child_begin=arr(v.box_child_begin, nb, np.int64),
                pbeg=arr(v.box_pbeg, nb, np.int64), pend=arr(v.box_pend, nb, np.int64),
                lev_hf=arr(v.level_hf, nl, np.int32), lev_T=arr(v.level_T, nl, np.int32),
                lev_n=arr(v.level_n, nl, np.int32), direct=arr(v.direct, 2 * nd, np.int64).reshape(nd, 2),
                m2l_tgt=m2l_box[:, 0].copy(), m2l_src=m2l_box[:, 1].copy(), m2l_level=m2l_info[:, 0].copy(),
                m2l_off=m2l_info[:, 1:4].copy(), m2l_wout=m2l_info[:, 4].copy(), m2l_win=m2l_info[:, 5].copy())


def fda_tree_destroy(tree):
    lib().fda_tree_destroy(tree)


def fda_precompute_translations(tree, eps, precision=FDA_PREC_FP64, lowrank=1, nrhs_max=1, m2l_tensor=0, op=0,
                                near_split=0, gamma=0.0, drop_fp64=False, near_form=0):
    cfg = fda_config_t()
    cfg.drop_fp64 = int(bool(drop_fp64))
    cfg.near_form = int(near_form)
    cfg.gamma_re = complex(gamma).real
    cfg.gamma_im = complex(gamma).imag
    cfg.eps = float(eps)
    cfg.precision = int(precision)
    cfg.lowrank = int(lowrank)
    cfg.nrhs_max = int(nrhs_max)
    cfg.m2l_tensor = int(m2l_tensor)
    cfg.op = int(op)
    cfg.near_split = int(near_split)
    h = C.c_void_p()
    _check(lib().fda_precompute_translations(tree, C.byref(cfg), C.byref(h)))
    return h


def fda_matvec(plan, x, y, stream=None):
    """y = A x for torch CUDA tensors of shape (N,) or (nrhs, N), complex128 or complex64."""
    import torch
    assert x.is_cuda and y.is_cuda and x.is_contiguous() and y.is_contiguous() and x.dtype == y.dtype
    nrhs = 1 if x.dim() == 1 else x.shape[0]
    dt = FDA_CPLX128 if x.dtype == torch.complex128 else FDA_CPLX64
    _check(lib().fda_matvec(plan, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), nrhs, dt, _stream(stream)))


PHASES = ("perm", "near", "s2m", "m2m", "m2l", "l2l", "l2t", "assemble")


def fda_matvec_ex(plan, precision, x, y, stream=None):
    import torch
    nrhs = 1 if x.dim() == 1 else x.shape[0]
    dt = FDA_CPLX128 if x.dtype == torch.complex128 else FDA_CPLX64
    _check(lib().fda_matvec_ex(plan, int(precision), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), nrhs, dt,
                               _stream(stream)))


def fda_matvec_phases(plan, precision, x, y, stream=None) -> dict:
    """Like fda_matvec_ex, synchronous, returning the device milliseconds of each phase."""
    import torch
    nrhs = 1 if x.dim() == 1 else x.shape[0]
    dt = FDA_CPLX128 if x.dtype == torch.complex128 else FDA_CPLX64
    ms = np.zeros(8)
    _check(lib().fda_matvec_phases(plan, int(precision), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), nrhs,
                                   dt, _stream(stream), _ptr(ms)))
    return dict(zip(PHASES, ms.tolist()))


def fda_device_peaks() -> tuple:
    a = C.c_double()
    b = C.c_double()
    _check(lib().fda_device_peaks(C.byref(a), C.byref(b)))
    return a.value, b.value


def fda_matvec_graph_create(plan, precision, x, y, stream=None):
    """Capture one product y = A x (fixed x, y tensors) into a CUDA graph; returns the graph handle."""
    import torch
    nrhs = 1 if x.dim() == 1 else x.shape[0]
    dt = FDA_CPLX128 if x.dtype == torch.complex128 else FDA_CPLX64
    g = C.c_void_p()
    _check(lib().fda_matvec_graph_create(plan, int(precision), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                         nrhs, dt, _stream(stream), C.byref(g)))
    return g


def fda_autotune(plan, nrhs=1, stream=None) -> dict:
    """Pick the faster M2L kernel per (level, stage), the near-field batch width and the correction split,
    for this nrhs."""
    R = fda_tune_report_t()
    _check(lib().fda_autotune(plan, int(nrhs), _stream(stream), C.byref(R)))
    rows = [dict(level=R.level[e], stage=R.stage[e], ms_fma=R.ms_fma[e], ms_tensor=R.ms_tensor[e],
                 chosen=("fma", "tensor", "tensor-alt1", "tensor-alt2", "tensor-alt3", "tensor-bulk",
                         "tensor-bulk-1stage", "vhat-swapped", "vhat-swapped-2stage", "uhat-persistent",
                         "tensor-bulk-narrow", "vhat-tma-4stage", "vhat-tma-3stage", "vhat-swapped-k16-2stage",
                         "vhat-swapped-k16-3stage")[R.chosen[e]])
            for e in range(R.entries)]
    return dict(m2l=rows, near_ms=list(R.near_ms), near_rhs_per_pass=R.near_rhs_per_pass,
                near_split=R.near_split, near_split_ms=list(R.near_split_ms), near_window_ms=R.near_window_ms,
                overlap=R.overlap, near_evict_first=R.near_evict_first,
                far_levels_concurrent=R.far_levels_concurrent, schedule_ms=list(R.schedule_ms),
                near_form=R.near_form, near_form_ms=[list(r) for r in R.near_form_ms],
                m2l_rechosen=R.m2l_rechosen, product_ms=R.product_ms, near_slim=R.near_slim, near_tc_ms=R.near_tc_ms,
                schedule_slim_ms=list(R.schedule_slim_ms))


def fda_m2l_force(plan, variant):
    """Force one M2L kernel variant for every (level, stage) (-1: the plan's default; see include/fdbem.h)."""
    _check(lib().fda_m2l_force(plan, int(variant)))


def fda_overlap_force(plan, mode, evict_first=0, far_levels=0):
    """FP32 product schedule: mode 0 serial, 1, 2 or 3 far field on the plan's stream beside the near field (two,
    one or three near-field CTAs per SM); evict_first = 1 gives the near-field matrix copies an L2 evict-first policy;
    far_levels = 1 runs the M2L of each level on its own stream."""
    _check(lib().fda_overlap_force(plan, int(mode), int(evict_first), int(far_levels)))


def fda_plan_check(plan):
    """FDA_OK, or FDA_E_TIMEOUT if a bounded device wait gave up in an earlier product (flag cleared)."""
    return lib().fda_plan_check(plan)


def fda_wait_selftest(limit_ms=50.0) -> int:
    """Run one kernel whose wait can never complete, bounded by limit_ms; returns 1 when it timed out."""
    t = C.c_int(0)
    _check(lib().fda_wait_selftest(float(limit_ms), C.byref(t)))
    return int(t.value)


def fda_graph_launch(g, stream=None):
    _check(lib().fda_graph_launch(g, _stream(stream)))


def fda_graph_nodes(g) -> int:
    n = C.c_int64()
    _check(lib().fda_graph_nodes(g, C.byref(n)))
    return int(n.value)


def fda_graph_destroy(g):
    lib().fda_graph_destroy(g)


def fda_plan_info(plan) -> dict:
    I = fda_plan_info_t()
    _check(lib().fda_plan_info(plan, C.byref(I)))
    out = {}
    for name, _ in fda_plan_info_t._fields_:
        v = getattr(I, name)
        out[name] = list(v) if hasattr(v, "__len__") else v
    return out


def fda_corrections_export(plan, rows, cap=512):
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    R = len(rows)
    cnt = np.zeros(R, dtype=np.int64)
    cols = np.zeros((R, cap), dtype=np.int64)
    vals = np.zeros((R, cap, 2))
    _check(lib().fda_corrections_export(plan, _ptr(rows, C.c_int64), R, cap, _ptr(cnt, C.c_int64),
                                        _ptr(cols, C.c_int64), _ptr(vals)))
    out = []
    for r in range(R):
        n = int(min(cnt[r], cap))
        out.append((cols[r, :n].copy(), vals[r, :n, 0] + 1j * vals[r, :n, 1]))
    return out


def fda_plan_destroy(plan):
    lib().fda_plan_destroy(plan)


def bm_gmres_solve(plan, b, x, tol=1e-6, restart=50, max_iter=1000, x0_given=False, refine=False,
                   inner_restart=0, inner_tol=1e-4, stream=None, raise_on_error=True, refine_residual=0):
    o = bm_gmres_opts_t()
    o.refine_residual = int(refine_residual)
    o.tol = float(tol)
    o.restart = int(restart)
    o.max_iter = int(max_iter)
    o.x0_given = int(bool(x0_given))
    o.refine = int(bool(refine))
    o.inner_restart = int(inner_restart)
    o.inner_tol = float(inner_tol)
    st = bm_gmres_stats_t()
    nrhs = 1 if b.dim() == 1 else b.shape[0]
    rc = lib().bm_gmres_solve(plan, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), nrhs, C.byref(o),
                              C.byref(st), _stream(stream))
    # the return code is the status (a call that fails before it fills the statistics still returns it)
    stats = dict(iterations=st.iterations, outer_iterations=st.outer_iterations, rel_residual=st.rel_residual,
                 ms_total=st.ms_total, ms_matvec=st.ms_matvec, status=int(rc))
    if raise_on_error:
        _check(rc)
    return stats


def bm_net_create(hidden=32, seed=1):
    h = C.c_void_p()
    _check(lib().bm_net_create(int(hidden), int(seed), C.byref(h)))
    return h


def bm_net_params(net, set_values=None):
    """Return the parameters (float32 numpy); optionally set them first."""
    n = C.c_int()
    _check(lib().bm_net_params(net, None, None, C.byref(n)))
    if set_values is not None:
        sv = np.ascontiguousarray(set_values, dtype=np.float32)
        assert sv.size == n.value
        _check(lib().bm_net_params(net, None, sv.ctypes.data_as(C.POINTER(C.c_float)), C.byref(n)))
    out = np.zeros(n.value, dtype=np.float32)
    _check(lib().bm_net_params(net, out.ctypes.data_as(C.POINTER(C.c_float)), None, C.byref(n)))
    return out


def bm_net_destroy(net):
    lib().bm_net_destroy(net)


def bm_precond_create(plan):
    h = C.c_void_p()
    _check(lib().bm_precond_create(plan, C.byref(h)))
    return h


def bm_precond_destroy(pc):
    lib().bm_precond_destroy(pc)


def bm_precond_apply(pc, net, r, z, stream=None):
    _check(lib().bm_precond_apply(pc, net, C.c_void_p(r.data_ptr()), C.c_void_p(z.data_ptr()), _stream(stream)))


def bm_precond_train_step(pc, net, R, E, lr=1e-3, want_grad=False, stream=None):
    """R, E: (npairs, N) complex128 device tensors. Returns (loss, grad or None)."""
    npairs = 1 if R.dim() == 1 else R.shape[0]
    loss = C.c_double()
    g = None
    gp = None
    if want_grad:
        n = C.c_int()
        _check(lib().bm_net_params(net, None, None, C.byref(n)))
        g = np.zeros(n.value, dtype=np.float32)
        gp = g.ctypes.data_as(C.POINTER(C.c_float))
    _check(lib().bm_precond_train_step(pc, net, C.c_void_p(R.data_ptr()), C.c_void_p(E.data_ptr()), npairs,
                                       float(lr), C.byref(loss), gp, _stream(stream)))
    return loss.value, g


def bm_residual_pair(plan, b, xstar, x, r, e, stream=None):
    _check(lib().bm_residual_pair(plan, C.c_void_p(b.data_ptr()), C.c_void_p(xstar.data_ptr()),
                                  C.c_void_p(x.data_ptr()), C.c_void_p(r.data_ptr()), C.c_void_p(e.data_ptr()),
                                  _stream(stream)))


def bm_fgmres_solve(plan, pc, net, b, x, tol=1e-6, restart=50, max_iter=1000, x0_given=False, refine=False,
                    inner_restart=0, inner_tol=1e-4, stream=None, raise_on_error=True, refine_residual=0):
    o = bm_gmres_opts_t()
    o.refine_residual = int(refine_residual)
    o.tol = float(tol)
    o.restart = int(restart)
    o.max_iter = int(max_iter)
    o.x0_given = int(bool(x0_given))
    o.refine = int(bool(refine))
    o.inner_restart = int(inner_restart)
    o.inner_tol = float(inner_tol)
    st = bm_gmres_stats_t()
    nrhs = 1 if b.dim() == 1 else b.shape[0]
    rc = lib().bm_fgmres_solve(plan, pc, net, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), nrhs,
                               C.byref(o), C.byref(st), _stream(stream))
    stats = dict(iterations=st.iterations, outer_iterations=st.outer_iterations, rel_residual=st.rel_residual,
                 ms_total=st.ms_total, ms_matvec=st.ms_matvec, status=int(rc))
    if raise_on_error:
        _check(rc)
    return stats


def fda_tc_selftest(K=64, split=0):
    e = C.c_double()
    wf = C.c_int()
    _check(lib().fda_tc_selftest(int(K), int(split), C.byref(e), C.byref(wf)))
    return e.value, wf.value


def fda_last_error() -> str:
    return lib().fda_last_error().decode(errors="replace")


# ----------------------------------------------------------------------------- owning wrappers
class ParticleSum:
    """Particle summation (Eq. sum) on points with normals: problem + tree + plan with ordered destruction."""

    def __init__(self, x, n, k, eps=1e-4, leaf_max=64, precision=FDA_PREC_FP64, lowrank=1, nrhs_max=1,
                 alpha=None, m2l_tensor=0):
        self.k = float(k)
        self.prob = bm_particles_create(x, n, k, alpha)
        self.tree = fda_build_tree(self.prob, leaf_max)
        self.plan = fda_precompute_translations(self.tree, eps, precision, lowrank, nrhs_max, m2l_tensor)
        self.N = int(np.asarray(x).shape[0])

    def matvec(self, x, y, stream=None):
        fda_matvec(self.plan, x, y, stream)

    def info(self):
        return fda_plan_info(self.plan)

    def close(self):
        if getattr(self, "plan", None):
            fda_plan_destroy(self.plan)
            self.plan = None
        if getattr(self, "tree", None):
            fda_tree_destroy(self.tree)
            self.tree = None
        if getattr(self, "prob", None):
            bm_problem_destroy(self.prob)
            self.prob = None


class Solver:
    """Problem + tree + plan with ordered destruction."""

    def __init__(self, nodes, elems, k, eps=1e-4, leaf_max=64, precision=FDA_PREC_FP64, lowrank=1, nrhs_max=1,
                 alpha=None, m2l_tensor=0, op=0, near_split=0, gamma=0.0, drop_fp64=False, near_form=0):
        self.k = float(k)
        self.prob = bm_problem_create(nodes, elems, k, alpha)
        self.tree = fda_build_tree(self.prob, leaf_max)
        self.plan = fda_precompute_translations(self.tree, eps, precision, lowrank, nrhs_max, m2l_tensor, op,
                                                near_split, gamma, drop_fp64, near_form)
        self.N = 6 * int(np.asarray(elems).shape[0])

    def matvec(self, x, y, stream=None):
        fda_matvec(self.plan, x, y, stream)

    def solve(self, b, x, **kw):
        return bm_gmres_solve(self.plan, b, x, **kw)

    def info(self):
        return fda_plan_info(self.plan)

    def close(self):
        if getattr(self, "plan", None):
            fda_plan_destroy(self.plan)
            self.plan = None
        if getattr(self, "tree", None):
            fda_tree_destroy(self.tree)
            self.tree = None
        if getattr(self, "prob", None):
            bm_problem_destroy(self.prob)
            self.prob = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
