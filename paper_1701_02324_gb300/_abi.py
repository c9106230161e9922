"""ctypes declarations of the C ABI in include/kf.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

KF_OK, KF_EINVAL, KF_ENOMEM, KF_ECUDA, KF_EILLCOND, KF_ENOTCONV, KF_ETIMEOUT, KF_EUNSUPPORTED = range(8)
KF_F32, KF_F64 = 0, 1
KF_PREC_FP64, KF_PREC_MIXED = 0, 1
KF_V_STORED, KF_V_RECOMPUTE = 0, 1

# Every entry point of include/kf.h: name -> (restype, argtypes).
_P, _I32, _I64, _U64, _D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double


class kf_alloc(ctypes.Structure):
    _fields_ = [("alloc", ctypes.c_void_p), ("free", ctypes.c_void_p), ("user", ctypes.c_void_p)]


class kf_opts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("n_samp", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("v_storage", ctypes.c_int32),
        ("sync_errors", ctypes.c_int32),
        ("refine_tol", ctypes.c_double),
        ("refine_max_iter", ctypes.c_int32),
        ("no_tensor_cores", ctypes.c_int32),
        ("fp64_operator", ctypes.c_int32),
        ("gmres_restart", ctypes.c_int32),
        ("no_cluster_kernels", ctypes.c_int32),
        ("tc_tile_n", ctypes.c_int32),
        ("zinv_max_nodes", ctypes.c_int32),
        ("hybrid_level", ctypes.c_int32),
        ("knn_kappa", ctypes.c_int32),
        ("knn_trees", ctypes.c_int32),
        ("knn_leaf", ctypes.c_int32),
        ("zoff_fused", ctypes.c_int32),
        ("w_recompute", ctypes.c_int32),
        ("tc_operator", ctypes.c_int32),
    ]


class kf_solve_info(ctypes.Structure):
    _fields_ = [("eps_r", ctypes.c_double), ("iters", ctypes.c_int32), ("status", ctypes.c_int32)]


SIGNATURES = {
    "kf_create": (_I32, [ctypes.POINTER(_P), _P]),
    "kf_destroy": (_I32, [_P]),
    "kf_status_string": (ctypes.c_char_p, [_I32]),
    "kf_last_error": (ctypes.c_char_p, [_P]),
    "kf_tree_build": (_I32, [_P, _P, _I32, _I64, _I32, _I32, _P, ctypes.POINTER(_P)]),
    "kf_tree_perm": (_I32, [_P, _P, _P]),
    "kf_tree_info": (_I32, [_P, _P, _P, _P, _P]),
    "kf_tree_free": (_I32, [_P]),
    "kf_factorize": (_I32, [_P, _D, _D, _D, _I32, _P, _P, ctypes.POINTER(_P)]),
    "kf_factor_status": (_I32, [_P, _P]),
    "kf_factor_free": (_I32, [_P]),
    "kf_solve": (_I32, [_P, _P, _P, _I64, _I64, _I32, _I32, _P, _P]),
    "kf_matvec": (_I32, [_P, _P, _P, _I64, _I64, _I32, _P]),
    "kf_grad": (_I32, [_P, _P, _P, _P, _P, _P, _I64, _I64, _P]),
    "kf_factor_ranks": (_I32, [_P, _P, _P]),
    "kf_factor_skeleton": (_I32, [_P, _I32, _P, _P]),
    "kf_factor_P": (_I32, [_P, _I32, _P, _P]),
    "kf_factor_Phat": (_I32, [_P, _I32, _P, _P]),
    "kf_factor_pivot_ratios": (_I32, [_P, _P, _P]),
    "kf_factor_knn": (_I32, [_P, _P, _P]),
    "kf_factor_near": (_I32, [_P, _I32, _P, _P, _P, _P]),
    "kf_factorize_with_ids": (_I32, [_P, _D, _D, _I32, _P, _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "kf_tree_perm_noalloc": (_I32, [_P, _I64, _I32, _I32, _P, _P, _P]),
    "kf_factorize_batched": (_I32, [_P, _I32, _P, _P, _P, _I32, _P, _P, _P]),
    "kf_solve_batched": (_I32, [_P, _I32, _P, _P, _P, _P, _I32, _P, _P]),
    "kf_autotune": (_I32, [_P, _D, _D, _D, _I32, _P, _P, _P, _P, _P]),
    "kf_test_tc_wait_probe": (_I32, [_I64]),
    "kf_launch_count": (_I64, []),
    "kf_profile_enable": (_I32, [_I32]),
    "kf_profile_read": (_I32, [_P, _P, _I32]),
    "kf_profile_timeline": (_I32, [_P, _P, _P, _P, _I64, _P]),
}

PHASES = ["tree", "sample", "eval_A", "qr", "leaf_assemble", "leaf_cholesky", "leaf_phat", "eval_V", "zoff", "z_lu",
          "z_solve_pc", "telescope", "solve_leaf", "solve_colsum", "solve_zsolve", "solve_rowupd", "matvec_leaf",
          "matvec_push", "misc", "qr_cluster", "qr_leaf", "matvec_colsum", "matvec_rowupd", "z_inv", "hybrid", "near"]

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libkf.so (building it in-tree first when asked).  Raises if the
    library cannot be built or loaded: there is no CPU fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise ImportError(f"libkf.so not found at {path}; run paper_1701_02324_gb300._build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class KFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


def status_name(s: int) -> str:
    return load().kf_status_string(int(s)).decode()


def check(status: int, ctx=None, allow=()):
    if status != KF_OK and status not in allow:
        msg = load().kf_last_error(ctx).decode(errors="replace")
        raise KFError(status, msg)
    return status
