"""Thin ctypes binding of libsic (include/sic.h).

Argument marshalling only: every function here checks types, takes raw pointers
of torch tensors (device memory) or numpy arrays (host memory) and calls the
C entry point of the same name.  All arithmetic of the method runs in libsic's
CUDA kernels; there is no CPU fallback -- if the compiled library is missing,
`lib()` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsic.so")

SIC_OK, SIC_ERR_INVALID, SIC_ERR_NOT_PD, SIC_ERR_CUDA, SIC_ERR_OOM, SIC_ERR_TIMEOUT, SIC_ERR_UNSUPPORTED = range(7)
SIC_FP64, SIC_FP32_MIXED = 0, 1
SIC_OP_L, SIC_OP_LT, SIC_OP_LLT = 0, 1, 2

# every symbol include/sic.h declares
EXPORTS = [
    "sic_create", "sic_destroy", "sic_sync", "sic_last_error_unit", "sic_status_string", "sic_exhaustion_floor",
    "sic_prep_maximin", "sic_prep_candidates_columns", "sic_prep_groups", "sic_prep_candidates_groups",
    "sic_prep_candidates_targets", "sic_gp_predict",
    "sic_select_single_workspace", "sic_select_single", "sic_select_columns",
    "sic_select_aggregated_workspace", "sic_select_aggregated",
    "sic_select_columns_gain", "sic_select_aggregated_gain", "sic_allocate_global_workspace", "sic_allocate_global",
    "sic_side_state_fp64", "sic_prep_candidates_partial", "sic_select_partial", "sic_partial_columns",
    "sic_build_factor_partial", "sic_tune_build_factor", "sic_tune_select_aggregated", "sic_tune_save", "sic_tune_load", "sic_tune_count",
    "sic_tune_entry",
    "sic_factor_nnz_workspace", "sic_factor_nnz", "sic_factor_nnz_noalloc", "sic_build_factor_workspace",
    "sic_build_factor", "sic_prep_partition", "sic_factor_nnz_range", "sic_build_factor_range", "sic_sum_fixed",
    "sic_apply_factor_workspace", "sic_apply_factor",
    "sic_matern_matvec", "sic_pcg_workspace", "sic_pcg_solve", "sic_selftest_wait_timeout",
    "sic_selftest_fp64_math", "sic_selftest_matern_df", "sic_selftest_fixed_point",
    "sic_mlp_param_count", "sic_proposal_features", "sic_proposal_score",
    "sic_proposal_topk", "sic_proposal_labels", "sic_mlp_train_workspace", "sic_mlp_grads", "sic_adamw_step",
]


class SicError(RuntimeError):
    def __init__(self, code: int, where: str, unit: int = -1):
        self.code = code
        self.unit = unit
        super().__init__(f"{where}: {status_string(code)} (code {code}, unit {unit})")


class Kernel(C.Structure):
    """sic_kernel: Matern kernel, nu_x2 = 2 nu in {1, 3, 5}."""
    _fields_ = [("dim", C.c_int32), ("nu_x2", C.c_int32), ("length_scale", C.c_double),
                ("variance", C.c_double), ("nugget", C.c_double)]


def kernel(dim, nu_x2, length_scale, variance=1.0, nugget=0.0) -> Kernel:
    return Kernel(int(dim), int(nu_x2), float(length_scale), float(variance), float(nugget))


_lib = None


def lib():
    """Load libsic.so; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsic is not built ({LIB_PATH} missing); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, d, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_size_t
        pk = C.POINTER(Kernel)
        st = C.c_int
        sig = {
            "sic_create": (st, [C.POINTER(vp), C.c_int]),
            "sic_destroy": (None, [vp]),
            "sic_sync": (st, [vp, vp]),
            "sic_last_error_unit": (i64, [vp]),
            "sic_status_string": (C.c_char_p, [st]),
            "sic_exhaustion_floor": (d, [pk]),
            "sic_prep_maximin": (st, [vp, i64, i32, vp, vp, i32]),
            "sic_prep_candidates_columns": (st, [vp, i64, i32, i32, vp, vp, i32]),
            "sic_prep_candidates_targets": (st, [vp, i64, i32, i64, i32, vp, vp, i32]),
            "sic_gp_predict": (st, [vp, vp, i64, pk, vp, i64, vp, vp, i32, vp, vp, vp, vp]),
            "sic_prep_groups": (st, [vp, vp, i64, i32, i32, d, i32, i32, vp, vp, vp, i32]),
            "sic_prep_partition": (st, [vp, vp, i64, i32, i32, i32, vp]),
            "sic_factor_nnz_range": (st, [vp, vp, i64, vp, i64, i64, i64, vp, vp, sz, vp]),
            "sic_build_factor_range": (st, [vp, vp, i64, pk, vp, i64, i32, vp, vp, i32, i64, i64, vp, i64, vp, vp,
                                            vp, vp, vp, sz, vp]),
            "sic_sum_fixed": (st, [vp, vp, i64, vp, vp, sz, vp]),
            "sic_prep_candidates_groups": (st, [vp, i64, i32, vp, i64, i32, vp, vp, i32]),
            "sic_select_single_workspace": (st, [i64, i32, st, C.POINTER(sz)]),
            "sic_select_single": (st, [vp, vp, i64, vp, pk, i32, st, vp, vp, vp, vp, sz, vp]),
            "sic_select_columns": (st, [vp, vp, i64, pk, vp, i64, vp, vp, i32, i32, st, vp, vp, vp]),
            "sic_select_aggregated_workspace": (st, [vp, i64, i32, i32, i32, st, C.POINTER(sz)]),
            "sic_select_aggregated": (st, [vp, vp, i64, pk, vp, i64, vp, vp, i32, i32, i32, st, vp, vp, vp, sz,
                                           vp]),
            "sic_select_columns_gain": (st, [vp, vp, i64, pk, vp, i64, vp, vp, i32, i32, st, vp, vp, vp, vp]),
            "sic_select_aggregated_gain": (st, [vp, vp, i64, pk, vp, i64, vp, vp, i32, i32, i32, st, vp, vp, vp,
                                                vp, sz, vp]),
            "sic_allocate_global_workspace": (st, [i64, i32, C.POINTER(sz)]),
            "sic_side_state_fp64": (st, [vp, vp, i64, pk, vp, vp, i64, i32, vp, vp, i32, vp, vp, vp, vp]),
            "sic_prep_candidates_partial": (st, [vp, i64, i32, vp, vp, i64, i32, vp, vp, i32]),
            "sic_select_partial": (st, [vp, vp, i64, pk, vp, vp, i64, vp, vp, i32, i32, i32, st, vp, vp, vp, vp]),
            "sic_partial_columns": (st, [vp, i64, vp, vp, i64, vp, vp, i32, i32, vp, vp, vp]),
            "sic_build_factor_partial": (st, [vp, vp, i64, pk, vp, vp, i64, i32, vp, vp, i32, vp, vp, vp, vp, vp, vp,
                                              sz, vp]),
            "sic_allocate_global": (st, [vp, i64, vp, vp, vp, i32, i64, vp, vp, sz, vp]),
            "sic_factor_nnz_workspace": (st, [i64, C.POINTER(sz)]),
            "sic_factor_nnz": (st, [vp, vp, i64, vp, i64, vp, vp, sz, vp]),
            "sic_factor_nnz_noalloc": (st, [vp, vp, i64, vp, i64, vp, vp]),
            "sic_build_factor_workspace": (st, [i64, C.POINTER(sz)]),
            "sic_tune_build_factor": (st, [vp, vp, i64, pk, vp, i64, i32, vp, vp, i32, vp, vp, vp, vp, vp, vp, sz,
                                           vp, C.POINTER(i32)]),
            "sic_tune_select_aggregated": (st, [vp, vp, i64, pk, vp, i64, vp, vp, i32, i32, i32, st, vp, vp, vp, sz,
                                                vp, C.POINTER(i32)]),
            "sic_tune_save": (st, [vp, C.c_char_p]),
            "sic_tune_load": (st, [vp, C.c_char_p]),
            "sic_tune_count": (i32, [vp]),
            "sic_tune_entry": (st, [vp, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32),
                                    C.POINTER(C.c_float)]),
            "sic_build_factor": (st, [vp, vp, i64, pk, vp, i64, i32, vp, vp, i32, vp, vp, vp, vp, vp, vp, sz, vp]),
            "sic_apply_factor_workspace": (st, [i64, i32, st, C.POINTER(sz)]),
            "sic_apply_factor": (st, [vp, i64, vp, vp, vp, st, vp, vp, i32, vp, sz, vp]),
            "sic_matern_matvec": (st, [vp, vp, i64, pk, d, st, vp, vp, i32, vp]),
            "sic_selftest_wait_timeout": (st, [vp, i64, vp, vp]),
            "sic_selftest_fp64_math": (st, [vp, pk, vp, i64, vp, vp, vp, vp, vp]),
            "sic_selftest_matern_df": (st, [vp, pk, vp, vp, i64, vp, vp]),
            "sic_selftest_fixed_point": (st, [vp, vp, vp, i64, i32, vp, vp, vp, vp, vp]),
            "sic_pcg_workspace": (st, [i64, i32, C.POINTER(sz)]),
            "sic_pcg_solve": (st, [vp, vp, i64, pk, d, st, vp, vp, vp, vp, vp, i32, d, i32, vp, vp, vp, sz, vp]),
            "sic_mlp_param_count": (i32, []),
            "sic_proposal_features": (st, [vp, vp, i64, pk, vp, i64, vp, vp, vp, vp]),
            "sic_proposal_score": (st, [vp, vp, vp, i64, vp, vp]),
            "sic_proposal_topk": (st, [vp, vp, vp, vp, i64, i32, vp, vp, vp]),
            "sic_proposal_labels": (st, [vp, vp, vp, i64, vp, vp, i32, vp, vp]),
            "sic_mlp_train_workspace": (st, [i64, C.POINTER(sz)]),
            "sic_mlp_grads": (st, [vp, vp, vp, vp, i64, C.c_float, i32, vp, vp, vp, vp, sz, vp]),
            "sic_adamw_step": (st, [vp, vp, vp, vp, vp, i32, i32, C.c_float, C.c_float, C.c_float, C.c_float,
                                    C.c_float, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_string(code: int) -> str:
    try:
        return lib().sic_status_string(int(code)).decode()
    except Exception:
        return f"status {code}"


def _check(code: int, where: str, h=None):
    if code != SIC_OK:
        unit = lib().sic_last_error_unit(h.ptr) if h is not None else -1
        raise SicError(code, where, unit)


# ------------------------------------------------------------ marshalling --

def _dptr(t, dtype=None, name="tensor"):
    """Device pointer of a CUDA torch tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA torch tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _hptr(a, dtype, name="array"):
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        raise TypeError(f"{name} must be a C-contiguous numpy array of {dtype}")
    return C.c_void_p(a.ctypes.data)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------- handle --

class Handle:
    """Owns a sic_handle (device binding + status word)."""

    def __init__(self, device: int = 0):
        p = C.c_void_p()
        _check(lib().sic_create(C.byref(p), int(device)), "sic_create")
        self.ptr = p
        self.device = device

    def close(self):
        if self.ptr:
            lib().sic_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self, stream=None):
        """sic_sync: wait for the stream and raise the first kernel-recorded error."""
        _check(lib().sic_sync(self.ptr, _stream(stream)), "sic_sync", self)


def exhaustion_floor(kp: Kernel) -> float:
    return lib().sic_exhaustion_floor(C.byref(kp))


# ------------------------------------------------------------ host prep --

def prep_maximin(pts: np.ndarray, n_threads: int = 0):
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    n, dim = pts.shape
    order = np.empty(n, np.int64)
    ell2 = np.empty(n, np.float64)
    _check(lib().sic_prep_maximin(_hptr(pts, np.float64), n, dim, _hptr(order, np.int64), _hptr(ell2, np.float64),
                                  n_threads), "sic_prep_maximin")
    return order, ell2


def prep_candidates_columns(pts: np.ndarray, n_cand: int, n_threads: int = 0):
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    n, dim = pts.shape
    ptr = np.empty(n + 1, np.int64)
    idx = np.empty(max(1, n * n_cand), np.int32)
    _check(lib().sic_prep_candidates_columns(_hptr(pts, np.float64), n, dim, n_cand, _hptr(ptr, np.int64),
                                             _hptr(idx, np.int32), n_threads), "sic_prep_candidates_columns")
    return ptr, idx[:ptr[-1]].copy()


def prep_candidates_targets(pts: np.ndarray, n_targets: int, n_cand: int, n_threads: int = 0):
    """pts: targets first, then training points.  Returns (cand_ptr, cand_idx)."""
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    n, dim = pts.shape
    ptr = np.empty(n_targets + 1, np.int64)
    idx = np.empty(max(1, n_targets * n_cand), np.int32)
    _check(lib().sic_prep_candidates_targets(_hptr(pts, np.float64), n, dim, n_targets, n_cand,
                                             _hptr(ptr, np.int64), _hptr(idx, np.int32), n_threads),
           "sic_prep_candidates_targets")
    return ptr, idx[:ptr[-1]].copy()


def prep_groups(pts: np.ndarray, ell2: np.ndarray, K: int, lam: float = 1.5, mmin: int = 8, mmax: int = 64,
                n_threads: int = 0):
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    ell2 = np.ascontiguousarray(ell2, dtype=np.float64)
    n, dim = pts.shape
    members = np.empty(n, np.int64)
    gp = np.empty(n + 1, np.int64)
    ng = np.zeros(1, np.int64)
    _check(lib().sic_prep_groups(_hptr(pts, np.float64), _hptr(ell2, np.float64), n, dim, K, lam, mmin, mmax,
                                 _hptr(members, np.int64), _hptr(gp, np.int64), _hptr(ng, np.int64), n_threads),
           "sic_prep_groups")
    return members, gp[:ng[0] + 1].copy()


def prep_partition(cand_ptr: np.ndarray, grp_ptr, k: int, n_parts: int, max_cand: int = 0) -> np.ndarray:
    """sic_prep_partition: unit bounds of n_parts contiguous slices of near-equal cost."""
    cand_ptr = np.ascontiguousarray(cand_ptr, dtype=np.int64)
    gp = np.ascontiguousarray(grp_ptr, dtype=np.int64) if grp_ptr is not None else None
    bounds = np.empty(n_parts + 1, np.int64)
    _check(lib().sic_prep_partition(_hptr(cand_ptr, np.int64), _hptr(gp, np.int64) if gp is not None else None,
                                    len(cand_ptr) - 1, k, max_cand, n_parts, _hptr(bounds, np.int64)),
           "sic_prep_partition")
    return bounds


def prep_candidates_groups(pts: np.ndarray, grp_ptr: np.ndarray, n_cand: int, n_threads: int = 0):
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    grp_ptr = np.ascontiguousarray(grp_ptr, dtype=np.int64)
    n, dim = pts.shape
    ng = len(grp_ptr) - 1
    ptr = np.empty(ng + 1, np.int64)
    idx = np.empty(max(1, ng * n_cand), np.int32)
    _check(lib().sic_prep_candidates_groups(_hptr(pts, np.float64), n, dim, _hptr(grp_ptr, np.int64), ng, n_cand,
                                            _hptr(ptr, np.int64), _hptr(idx, np.int32), n_threads),
           "sic_prep_candidates_groups")
    return ptr, idx[:ptr[-1]].copy()


# ------------------------------------------------------------- selection --

def _ws(nbytes: int, device):
    import torch
    return torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device=device)


def select_single_workspace(n: int, k: int, prec: int) -> int:
    b = C.c_size_t()
    _check(lib().sic_select_single_workspace(n, k, prec, C.byref(b)), "sic_select_single_workspace")
    return b.value


def select_single(h: Handle, x_train, x_target, kp: Kernel, k: int, prec: int, out_idx, out_var, out_count, ws,
                  stream=None):
    import torch
    n = x_train.shape[0]
    _check(lib().sic_select_single(h.ptr, _dptr(x_train, torch.float64, "x_train"), n,
                                   _dptr(x_target, torch.float64, "x_target"), C.byref(kp), k, prec,
                                   _dptr(out_idx, torch.int32, "out_idx"), _dptr(out_var, torch.float64, "out_var"),
                                   _dptr(out_count, torch.int32, "out_count"), _dptr(ws), ws.numel(),
                                   _stream(stream)), "sic_select_single", h)


def select_columns(h: Handle, pts, kp: Kernel, cand_ptr, cand_idx, max_cand: int, k: int, prec: int, sel_idx,
                   sel_count, targets=None, stream=None, gain=None):
    """sic_select_columns, or sic_select_columns_gain when `gain` (n_cols x k FP64) is given."""
    import torch
    n = pts.shape[0]
    n_cols = targets.numel() if targets is not None else n
    args = [h.ptr, _dptr(pts, torch.float64, "pts"), n, C.byref(kp), _dptr(targets, torch.int32, "targets"), n_cols,
            _dptr(cand_ptr, torch.int64, "cand_ptr"), _dptr(cand_idx, torch.int32, "cand_idx"), max_cand, k, prec,
            _dptr(sel_idx, torch.int32, "sel_idx"), _dptr(sel_count, torch.int32, "sel_count")]
    if gain is None:
        _check(lib().sic_select_columns(*args, _stream(stream)), "sic_select_columns", h)
    else:
        _check(lib().sic_select_columns_gain(*args, _dptr(gain, torch.float64, "gain"), _stream(stream)),
               "sic_select_columns_gain", h)


def select_aggregated_workspace(h: Handle, n_grp: int, max_cand: int, max_m: int, k: int, prec: int) -> int:
    b = C.c_size_t()
    _check(lib().sic_select_aggregated_workspace(h.ptr, n_grp, max_cand, max_m, k, prec, C.byref(b)),
           "sic_select_aggregated_workspace")
    return b.value


def select_aggregated(h: Handle, pts, kp: Kernel, grp_ptr, cand_ptr, cand_idx, max_cand: int, max_m: int, k: int,
                      prec: int, sel_idx, sel_count, ws, stream=None, gain=None):
    """sic_select_aggregated, or sic_select_aggregated_gain when `gain` (n_grp x k FP64) is given."""
    import torch
    n = pts.shape[0]
    n_grp = grp_ptr.numel() - 1
    args = [h.ptr, _dptr(pts, torch.float64, "pts"), n, C.byref(kp), _dptr(grp_ptr, torch.int64, "grp_ptr"), n_grp,
            _dptr(cand_ptr, torch.int64, "cand_ptr"), _dptr(cand_idx, torch.int32, "cand_idx"), max_cand, max_m, k,
            prec, _dptr(sel_idx, torch.int32, "sel_idx"), _dptr(sel_count, torch.int32, "sel_count")]
    if gain is None:
        _check(lib().sic_select_aggregated(*args, _dptr(ws), ws.numel(), _stream(stream)), "sic_select_aggregated", h)
    else:
        _check(lib().sic_select_aggregated_gain(*args, _dptr(gain, torch.float64, "gain"), _dptr(ws), ws.numel(),
                                                _stream(stream)), "sic_select_aggregated_gain", h)


def prep_candidates_partial(pts: np.ndarray, members: np.ndarray, grp_ptr: np.ndarray, n_cand: int,
                            n_threads: int = 0):
    """Host: candidates of nonadjacent groups (sic_prep_candidates_partial) -> (cand_ptr, cand_idx)."""
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    members = np.ascontiguousarray(members, dtype=np.int64)
    grp_ptr = np.ascontiguousarray(grp_ptr, dtype=np.int64)
    n_grp = len(grp_ptr) - 1
    ptr = np.zeros(n_grp + 1, np.int64)
    idx = np.zeros(max(n_grp * n_cand, 1), np.int32)
    _check(lib().sic_prep_candidates_partial(_hptr(pts, np.float64), pts.shape[0], pts.shape[1],
                                             _hptr(members, np.int64), _hptr(grp_ptr, np.int64), n_grp, n_cand,
                                             _hptr(ptr, np.int64), _hptr(idx, np.int32), n_threads),
           "sic_prep_candidates_partial")
    return ptr, idx[:ptr[-1]].copy()


def select_partial(h: Handle, pts, kp: Kernel, grp_ptr, members, cand_ptr, cand_idx, max_cand: int, max_m: int,
                   k: int, prec: int, sel_idx, sel_count, gain=None, stream=None):
    """Partial selection for nonadjacent groups (sic_select_partial)."""
    import torch
    _check(lib().sic_select_partial(h.ptr, _dptr(pts, torch.float64, "pts"), pts.shape[0], C.byref(kp),
                                    _dptr(grp_ptr, torch.int64, "grp_ptr"), _dptr(members, torch.int64, "members"),
                                    grp_ptr.numel() - 1, _dptr(cand_ptr, torch.int64, "cand_ptr"),
                                    _dptr(cand_idx, torch.int32, "cand_idx"), max_cand, max_m, k, prec,
                                    _dptr(sel_idx, torch.int32, "sel_idx"), _dptr(sel_count, torch.int32, "sel_count"),
                                    _dptr(gain, torch.float64, "gain"), _stream(stream)), "sic_select_partial", h)


def partial_columns(h: Handle, n: int, grp_ptr, members, sel_idx, sel_count, k: int, kc: int, col_sel, col_count,
                    stream=None):
    """Single-column lists of a partial selection for the fill (sic_partial_columns)."""
    import torch
    _check(lib().sic_partial_columns(h.ptr, n, _dptr(grp_ptr, torch.int64, "grp_ptr"),
                                     _dptr(members, torch.int64, "members"), grp_ptr.numel() - 1,
                                     _dptr(sel_idx, torch.int32, "sel_idx"), _dptr(sel_count, torch.int32, "sel_count"),
                                     k, kc, _dptr(col_sel, torch.int32, "col_sel"),
                                     _dptr(col_count, torch.int32, "col_count"), _stream(stream)),
           "sic_partial_columns", h)


def tune_select_aggregated(h: Handle, pts, kp: Kernel, grp_ptr, cand_ptr, cand_idx, max_cand: int, max_m: int,
                           k: int, prec: int, sel_idx, sel_count, ws, stream=None) -> int:
    """sic_tune_select_aggregated: the selection with its launch plan tuned (kept in the handle)."""
    import torch
    n = pts.shape[0]
    choice = C.c_int32(0)
    _check(lib().sic_tune_select_aggregated(h.ptr, _dptr(pts, torch.float64, "pts"), n, C.byref(kp),
                                            _dptr(grp_ptr, torch.int64, "grp_ptr"), grp_ptr.numel() - 1,
                                            _dptr(cand_ptr, torch.int64, "cand_ptr"),
                                            _dptr(cand_idx, torch.int32, "cand_idx"), max_cand, max_m, k, prec,
                                            _dptr(sel_idx, torch.int32, "sel_idx"),
                                            _dptr(sel_count, torch.int32, "sel_count"), _dptr(ws), ws.numel(),
                                            _stream(stream), C.byref(choice)), "sic_tune_select_aggregated", h)
    return choice.value


def tune_build_factor(h: Handle, pts, kp: Kernel, grp_ptr, max_m: int, sel_idx, sel_count, k: int, col_ptr,
                      row_idx, val, logv, sum_logv, ws, stream=None) -> int:
    """sic_tune_build_factor: the fill with its group-size split tuned (and kept in the handle)."""
    import torch
    n = pts.shape[0]
    n_grp = grp_ptr.numel() - 1 if grp_ptr is not None else n
    best = C.c_int32(0)
    _check(lib().sic_tune_build_factor(h.ptr, _dptr(pts, torch.float64, "pts"), n, C.byref(kp),
                                       _dptr(grp_ptr, torch.int64, "grp_ptr"), n_grp, max_m,
                                       _dptr(sel_idx, torch.int32, "sel_idx"),
                                       _dptr(sel_count, torch.int32, "sel_count"), k,
                                       _dptr(col_ptr, torch.int64, "col_ptr"), _dptr(row_idx, torch.int32, "row_idx"),
                                       _dptr(val, torch.float64, "val"), _dptr(logv, torch.float64, "logv"),
                                       _dptr(sum_logv, torch.float64, "sum_logv"), _dptr(ws), ws.numel(),
                                       _stream(stream), C.byref(best)), "sic_tune_build_factor", h)
    return best.value


def tune_save(h: Handle, path: str):
    _check(lib().sic_tune_save(h.ptr, str(path).encode()), "sic_tune_save")


def tune_load(h: Handle, path: str):
    _check(lib().sic_tune_load(h.ptr, str(path).encode()), "sic_tune_load")


def tune_table(h: Handle):
    """The handle's tuned choices as a list of (op, a, b, value, ms)."""
    out = []
    for i in range(lib().sic_tune_count(h.ptr)):
        v = [C.c_int32() for _ in range(4)]
        ms = C.c_float()
        _check(lib().sic_tune_entry(h.ptr, i, *[C.byref(x) for x in v], C.byref(ms)), "sic_tune_entry")
        out.append((v[0].value, v[1].value, v[2].value, v[3].value, ms.value))
    return out


def build_factor_partial(h: Handle, pts, kp: Kernel, grp_ptr, members, max_m: int, sel_idx, sel_count, k: int,
                         col_ptr, row_idx, val, logv, sum_logv, ws, stream=None):
    """Aggregated FP64 fill of a partial-selection pattern (sic_build_factor_partial)."""
    import torch
    _check(lib().sic_build_factor_partial(h.ptr, _dptr(pts, torch.float64, "pts"), pts.shape[0], C.byref(kp),
                                          _dptr(grp_ptr, torch.int64, "grp_ptr"),
                                          _dptr(members, torch.int64, "members"), grp_ptr.numel() - 1, max_m,
                                          _dptr(sel_idx, torch.int32, "sel_idx"),
                                          _dptr(sel_count, torch.int32, "sel_count"), k,
                                          _dptr(col_ptr, torch.int64, "col_ptr"), _dptr(row_idx, torch.int32, "row_idx"),
                                          _dptr(val, torch.float64, "val"), _dptr(logv, torch.float64, "logv"),
                                          _dptr(sum_logv, torch.float64, "sum_logv"), _dptr(ws), ws.numel(),
                                          _stream(stream)), "sic_build_factor_partial", h)


def side_state_fp64(h: Handle, pts, kp: Kernel, sel_idx, sel_count, k: int, grp_ptr=None, max_m: int = 1,
                    targets=None, pvar=None, pvar_p=None, gain=None, stream=None):
    """FP64 conditional variances of the picks without / with the unit's targets and their
    exact decreases per nonzero (sic_side_state_fp64); outputs are n_units x k FP64."""
    import torch
    n = pts.shape[0]
    n_units = sel_count.numel()
    _check(lib().sic_side_state_fp64(h.ptr, _dptr(pts, torch.float64, "pts"), n, C.byref(kp),
                                     _dptr(grp_ptr, torch.int64, "grp_ptr"), _dptr(targets, torch.int32, "targets"),
                                     n_units, max_m, _dptr(sel_idx, torch.int32, "sel_idx"),
                                     _dptr(sel_count, torch.int32, "sel_count"), k,
                                     _dptr(pvar, torch.float64, "pvar"), _dptr(pvar_p, torch.float64, "pvar_p"),
                                     _dptr(gain, torch.float64, "gain"), _stream(stream)), "sic_side_state_fp64", h)


def allocate_global_workspace(n_units: int, k: int) -> int:
    b = C.c_size_t()
    _check(lib().sic_allocate_global_workspace(n_units, k, C.byref(b)), "sic_allocate_global_workspace")
    return b.value


def allocate_global(h: Handle, gain, sel_count, k: int, budget: int, out_count, ws, grp_ptr=None, stream=None):
    """Global greedy allocation of `budget` nonzeros (Section 5.4): out_count[u] leading picks of unit u."""
    import torch
    n_units = sel_count.numel()
    _check(lib().sic_allocate_global(h.ptr, n_units, _dptr(grp_ptr, torch.int64, "grp_ptr"),
                                     _dptr(gain, torch.float64, "gain"), _dptr(sel_count, torch.int32, "sel_count"),
                                     k, int(budget), _dptr(out_count, torch.int32, "out_count"), _dptr(ws),
                                     ws.numel(), _stream(stream)), "sic_allocate_global", h)


# ------------------------------------------------------------- the factor --

def factor_nnz_workspace(n: int) -> int:
    b = C.c_size_t()
    _check(lib().sic_factor_nnz_workspace(n, C.byref(b)), "sic_factor_nnz_workspace")
    return b.value


def factor_nnz(h: Handle, grp_ptr, sel_count, n: int, col_ptr, ws, stream=None):
    import torch
    n_grp = grp_ptr.numel() - 1 if grp_ptr is not None else n
    _check(lib().sic_factor_nnz(h.ptr, _dptr(grp_ptr, torch.int64, "grp_ptr"), n_grp,
                                _dptr(sel_count, torch.int32, "sel_count"), n, _dptr(col_ptr, torch.int64, "col_ptr"),
                                _dptr(ws), ws.numel(), _stream(stream)), "sic_factor_nnz", h)


def factor_nnz_noalloc(h: Handle, grp_ptr, sel_count, n: int, col_ptr, stream=None):
    """sic_factor_nnz without a workspace (static scratch inside libsic; see include/sic.h)."""
    import torch
    n_grp = grp_ptr.numel() - 1 if grp_ptr is not None else n
    _check(lib().sic_factor_nnz_noalloc(h.ptr, _dptr(grp_ptr, torch.int64, "grp_ptr"), n_grp,
                                        _dptr(sel_count, torch.int32, "sel_count"), n,
                                        _dptr(col_ptr, torch.int64, "col_ptr"), _stream(stream)),
           "sic_factor_nnz_noalloc", h)


def factor_nnz_range(h: Handle, grp_ptr, sel_count, col0: int, n_cols: int, base: int, col_ptr, ws, stream=None):
    """sic_factor_nnz_range: col_ptr[0 .. n_cols] of the slice's columns, starting at base."""
    import torch
    n_grp = grp_ptr.numel() - 1 if grp_ptr is not None else n_cols
    _check(lib().sic_factor_nnz_range(h.ptr, _dptr(grp_ptr, torch.int64, "grp_ptr"), n_grp,
                                      _dptr(sel_count, torch.int32, "sel_count"), col0, n_cols, base,
                                      _dptr(col_ptr, torch.int64, "col_ptr"), _dptr(ws), ws.numel(), _stream(stream)),
           "sic_factor_nnz_range", h)


def build_factor_range(h: Handle, pts, kp: Kernel, grp_ptr, max_m: int, sel_idx, sel_count, k: int, col0: int,
                       n_cols: int, col_ptr, base: int, row_idx, val, logv, sum_logv, ws, stream=None):
    """sic_build_factor_range: the fill of the slice of columns col0 .. col0 + n_cols - 1."""
    import torch
    n = pts.shape[0]
    n_grp = grp_ptr.numel() - 1 if grp_ptr is not None else n_cols
    _check(lib().sic_build_factor_range(h.ptr, _dptr(pts, torch.float64, "pts"), n, C.byref(kp),
                                        _dptr(grp_ptr, torch.int64, "grp_ptr"), n_grp, max_m,
                                        _dptr(sel_idx, torch.int32, "sel_idx"),
                                        _dptr(sel_count, torch.int32, "sel_count"), k, col0, n_cols,
                                        _dptr(col_ptr, torch.int64, "col_ptr"), base,
                                        _dptr(row_idx, torch.int32, "row_idx"), _dptr(val, torch.float64, "val"),
                                        _dptr(logv, torch.float64, "logv"), _dptr(sum_logv, torch.float64, "sum_logv"),
                                        _dptr(ws), ws.numel(), _stream(stream)), "sic_build_factor_range", h)


def sum_fixed(h: Handle, x, out, ws, stream=None):
    """sic_sum_fixed: out[0] = sum of x in the fill's fixed order."""
    import torch
    _check(lib().sic_sum_fixed(h.ptr, _dptr(x, torch.float64, "x"), x.numel(), _dptr(out, torch.float64, "out"),
                               _dptr(ws), ws.numel(), _stream(stream)), "sic_sum_fixed", h)


def build_factor_workspace(n: int) -> int:
    b = C.c_size_t()
    _check(lib().sic_build_factor_workspace(n, C.byref(b)), "sic_build_factor_workspace")
    return b.value


def build_factor(h: Handle, pts, kp: Kernel, grp_ptr, max_m: int, sel_idx, sel_count, k: int, col_ptr, row_idx, val,
                 logv, sum_logv, ws, stream=None):
    import torch
    n = pts.shape[0]
    n_grp = grp_ptr.numel() - 1 if grp_ptr is not None else n
    _check(lib().sic_build_factor(h.ptr, _dptr(pts, torch.float64, "pts"), n, C.byref(kp),
                                  _dptr(grp_ptr, torch.int64, "grp_ptr"), n_grp, max_m,
                                  _dptr(sel_idx, torch.int32, "sel_idx"), _dptr(sel_count, torch.int32, "sel_count"),
                                  k, _dptr(col_ptr, torch.int64, "col_ptr"), _dptr(row_idx, torch.int32, "row_idx"),
                                  _dptr(val, torch.float64, "val"), _dptr(logv, torch.float64, "logv"),
                                  _dptr(sum_logv, torch.float64, "sum_logv"), _dptr(ws), ws.numel(),
                                  _stream(stream)), "sic_build_factor", h)


def apply_factor_workspace(n: int, nrhs: int, op: int) -> int:
    b = C.c_size_t()
    _check(lib().sic_apply_factor_workspace(n, nrhs, op, C.byref(b)), "sic_apply_factor_workspace")
    return b.value


def apply_factor(h: Handle, col_ptr, row_idx, val, op: int, x, y, ws=None, stream=None):
    import torch
    n = col_ptr.numel() - 1
    nrhs = 1 if x.dim() == 1 else x.shape[1]
    _check(lib().sic_apply_factor(h.ptr, n, _dptr(col_ptr, torch.int64, "col_ptr"),
                                  _dptr(row_idx, torch.int32, "row_idx"), _dptr(val, torch.float64, "val"), op,
                                  _dptr(x, torch.float64, "x"), _dptr(y, torch.float64, "y"), nrhs, _dptr(ws),
                                  ws.numel() if ws is not None else 0, _stream(stream)), "sic_apply_factor", h)


# ------------------------------------------------------- learned proposal --

def mlp_param_count() -> int:
    return int(lib().sic_mlp_param_count())


def proposal_features(h: Handle, pts, kp: Kernel, grp_ptr, cand_ptr, cand_idx, feat, stream=None):
    import torch
    _check(lib().sic_proposal_features(h.ptr, _dptr(pts, torch.float64, "pts"), pts.shape[0], C.byref(kp),
                                       _dptr(grp_ptr, torch.int64, "grp_ptr"), grp_ptr.numel() - 1,
                                       _dptr(cand_ptr, torch.int64, "cand_ptr"),
                                       _dptr(cand_idx, torch.int32, "cand_idx"), _dptr(feat, torch.float32, "feat"),
                                       _stream(stream)), "sic_proposal_features", h)


def proposal_score(h: Handle, params, feat, score, stream=None):
    import torch
    rows = feat.shape[0]
    _check(lib().sic_proposal_score(h.ptr, _dptr(params, torch.float32, "params"), _dptr(feat, torch.float32, "feat"),
                                    rows, _dptr(score, torch.float32, "score"), _stream(stream)),
           "sic_proposal_score", h)


def proposal_topk(h: Handle, cand_ptr, cand_idx, score, top: int, out_ptr, out_idx, stream=None):
    import torch
    _check(lib().sic_proposal_topk(h.ptr, _dptr(cand_ptr, torch.int64, "cand_ptr"),
                                   _dptr(cand_idx, torch.int32, "cand_idx"), _dptr(score, torch.float32, "score"),
                                   cand_ptr.numel() - 1, top, _dptr(out_ptr, torch.int64, "out_ptr"),
                                   _dptr(out_idx, torch.int32, "out_idx"), _stream(stream)), "sic_proposal_topk", h)


def proposal_labels(h: Handle, cand_ptr, cand_idx, sel_idx, sel_count, k: int, label, stream=None):
    import torch
    _check(lib().sic_proposal_labels(h.ptr, _dptr(cand_ptr, torch.int64, "cand_ptr"),
                                     _dptr(cand_idx, torch.int32, "cand_idx"), cand_ptr.numel() - 1,
                                     _dptr(sel_idx, torch.int32, "sel_idx"), _dptr(sel_count, torch.int32, "sel_count"),
                                     k, _dptr(label, torch.float32, "label"), _stream(stream)),
           "sic_proposal_labels", h)


def mlp_train_workspace(batch: int) -> int:
    b = C.c_size_t()
    _check(lib().sic_mlp_train_workspace(batch, C.byref(b)), "sic_mlp_train_workspace")
    return b.value


def mlp_grads(h: Handle, params, feat, label, pos_weight: float, bf16: bool, grads, loss, ws, score=None,
              stream=None):
    import torch
    _check(lib().sic_mlp_grads(h.ptr, _dptr(params, torch.float32, "params"), _dptr(feat, torch.float32, "feat"),
                               _dptr(label, torch.float32, "label"), feat.shape[0], float(pos_weight), int(bf16),
                               _dptr(grads, torch.float32, "grads"), _dptr(loss, torch.float32, "loss"),
                               _dptr(score, torch.float32, "score"), _dptr(ws), ws.numel(), _stream(stream)),
           "sic_mlp_grads", h)


def adamw_step(h: Handle, params, m, v, grads, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0,
               stream=None):
    import torch
    _check(lib().sic_adamw_step(h.ptr, _dptr(params, torch.float32), _dptr(m, torch.float32), _dptr(v, torch.float32),
                                _dptr(grads, torch.float32), params.numel(), int(step), float(lr), float(beta1),
                                float(beta2), float(eps), float(wd), _stream(stream)), "sic_adamw_step", h)


# -------------------------------------------------------- preconditioning --

def matern_matvec(h: Handle, pts, kp: Kernel, shift: float, prec: int, x, y, stream=None):
    import torch
    nrhs = 1 if x.dim() == 1 else x.shape[1]
    _check(lib().sic_matern_matvec(h.ptr, _dptr(pts, torch.float64, "pts"), pts.shape[0], C.byref(kp), float(shift),
                                   prec, _dptr(x, torch.float64, "x"), _dptr(y, torch.float64, "y"), nrhs,
                                   _stream(stream)), "sic_matern_matvec", h)


def pcg_workspace(n: int, nrhs: int) -> int:
    b = C.c_size_t()
    _check(lib().sic_pcg_workspace(n, nrhs, C.byref(b)), "sic_pcg_workspace")
    return b.value


def pcg_solve(h: Handle, pts, kp: Kernel, shift: float, prec: int, factor, b, x, tol: float, max_iter: int, ws,
              stream=None):
    """factor = (col_ptr, row_idx, val) device tensors or None.  Returns (iters, relres) numpy arrays."""
    import torch
    nrhs = 1 if b.dim() == 1 else b.shape[1]
    iters = np.zeros(nrhs, np.int32)
    relres = np.zeros(nrhs, np.float64)
    cp, ri, vv = factor if factor is not None else (None, None, None)
    _check(lib().sic_pcg_solve(h.ptr, _dptr(pts, torch.float64, "pts"), pts.shape[0], C.byref(kp), float(shift), prec,
                               _dptr(cp, torch.int64, "col_ptr"), _dptr(ri, torch.int32, "row_idx"),
                               _dptr(vv, torch.float64, "val"), _dptr(b, torch.float64, "b"),
                               _dptr(x, torch.float64, "x"), nrhs, float(tol), int(max_iter), _hptr(iters, np.int32),
                               _hptr(relres, np.float64), _dptr(ws), ws.numel(), _stream(stream)), "sic_pcg_solve", h)
    return iters, relres


def selftest_wait_timeout(h: Handle, cap: int, out, stream=None):
    import torch
    _check(lib().sic_selftest_wait_timeout(h.ptr, int(cap), _dptr(out, torch.int32, "out"), _stream(stream)),
           "sic_selftest_wait_timeout", h)


def selftest_fp64_math(h: Handle, kp: Kernel, x, stream=None):
    """sqrt(x), 1/sqrt(x), exp(-x) and the Matern at squared distance x by the fill's FP64
    device routines; x is a CUDA float64 tensor, returns four tensors like it."""
    import torch
    x = x.contiguous()
    outs = [torch.empty_like(x) for _ in range(4)]
    _check(lib().sic_selftest_fp64_math(h.ptr, C.byref(kp), _dptr(x, torch.float64, "x"), x.numel(),
                                        *[_dptr(o, torch.float64, "out") for o in outs], _stream(stream)),
           "sic_selftest_fp64_math", h)
    return outs


def selftest_fixed_point(h: Handle, pa, pb, ga, gb, stream=None):
    """The fill's integer routines: squared distances between the rows of pa and pb (CUDA float64,
    n x dim) and dot products of the rows of ga and gb (n x 4), as the fill forms them."""
    import torch
    pa, pb, ga, gb = pa.contiguous(), pb.contiguous(), ga.contiguous(), gb.contiguous()
    n = pa.shape[0]
    d2 = torch.empty(n, dtype=torch.float64, device=pa.device)
    dot = torch.empty(n, dtype=torch.float64, device=pa.device)
    _check(lib().sic_selftest_fixed_point(h.ptr, _dptr(pa, torch.float64, "pa"), _dptr(pb, torch.float64, "pb"), n,
                                          pa.shape[1], _dptr(d2, torch.float64, "d2"), _dptr(ga, torch.float64, "ga"),
                                          _dptr(gb, torch.float64, "gb"), _dptr(dot, torch.float64, "dot"),
                                          _stream(stream)),
           "sic_selftest_fixed_point", h)
    return d2, dot


def selftest_matern_df(h: Handle, kp: Kernel, pa, pb, stream=None):
    """The fill's double-float Matern between the rows of pa and pb (CUDA float64, n x dim)."""
    import torch
    pa, pb = pa.contiguous(), pb.contiguous()
    out = torch.empty(pa.shape[0], dtype=torch.float64, device=pa.device)
    _check(lib().sic_selftest_matern_df(h.ptr, C.byref(kp), _dptr(pa, torch.float64, "pa"),
                                        _dptr(pb, torch.float64, "pb"), pa.shape[0],
                                        _dptr(out, torch.float64, "out"), _stream(stream)),
           "sic_selftest_matern_df", h)
    return out


def gp_predict(h: Handle, pts, kp: Kernel, targets, sel_idx, sel_count, k: int, y, mean, var, stream=None):
    """Posterior mean and variance at `targets` (CUDA tensors; targets may be None)."""
    import torch
    n_t = mean.numel()
    _check(lib().sic_gp_predict(h.ptr, _dptr(pts, torch.float64, "pts"), pts.shape[0], C.byref(kp),
                                None if targets is None else _dptr(targets, torch.int32, "targets"), n_t,
                                _dptr(sel_idx, torch.int32, "sel_idx"), _dptr(sel_count, torch.int32, "sel_count"),
                                int(k), _dptr(y, torch.float64, "y"), _dptr(mean, torch.float64, "mean"),
                                _dptr(var, torch.float64, "var"), _stream(stream)), "sic_gp_predict", h)
