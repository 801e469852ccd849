"""ctypes binding of liblya.so (include/lya.h).  Argument marshalling only.

The library is loaded from the package's ``_build`` directory.  There is no
fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int32, c_int64, c_size_t, c_uint64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblya.so")

LYA_OK = 0
LYA_ERR_INVALID_ARG = -1
LYA_ERR_UNSORTED = -2
LYA_ERR_NONFINITE = -3
LYA_ERR_NO_MEMORY = -4
LYA_ERR_CUDA = -5
LYA_ERR_TIMEOUT = -6
LYA_ERR_DEVICE_CHECK = -7
LYA_ERR_TOO_LARGE = -8

LYA_PREC_FP64 = 0
LYA_PREC_MIXED = 1
LYA_ETA_IDENTITY = 0
LYA_ETA_MEAN_SLOPE = 1


class LyaCatalog(ctypes.Structure):
    _fields_ = [("n_forests", c_int64), ("n_pix", c_int64), ("offsets", c_void_p), ("ra", c_void_p),
                ("dec", c_void_p), ("dist", c_void_p), ("loglam", c_void_p), ("delta", c_void_p),
                ("weight", c_void_p)]


class LyaBins(ctypes.Structure):
    _fields_ = [("n_par", c_int32), ("n_perp", c_int32), ("r_par_max", c_double),
                ("r_perp_max", c_double)]


class LyaBins3(ctypes.Structure):
    _fields_ = [("n_r", c_int32), ("n_theta", c_int32), ("n_alpha", c_int32), ("r_max", c_double)]


class LyaQuasars(ctypes.Structure):
    _fields_ = [("n", c_int64), ("ra", c_void_p), ("dec", c_void_p), ("dist", c_void_p), ("weight", c_void_p)]


H = c_void_p
CAT = POINTER(LyaCatalog)
QSO = POINTER(LyaQuasars)
BINS = POINTER(LyaBins)
BINS3 = POINTER(LyaBins3)

# name -> (restype, argtypes), one entry per declaration of include/lya.h
SIGNATURES = {
    "lya_create": (c_int, [POINTER(c_void_p)]),
    "lya_destroy": (c_int, [H]),
    "lya_last_error": (c_int, [H, c_char_p, c_size_t]),
    "lya_status_string": (c_char_p, [c_int]),
    "lya_sync_status": (c_int, [H, c_void_p]),
    "lya_pairs_build": (c_int, [H, CAT, BINS, POINTER(c_int64), c_void_p]),
    "lya_pairs_get": (c_int, [H, c_void_p, c_void_p, c_int64, POINTER(c_int64), c_void_p]),
    "lya_project": (c_int, [H, CAT, c_void_p, c_void_p]),
    "lya_xi": (c_int, [H, CAT, BINS, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lya_xi_pairs": (c_int, [H, CAT, BINS, c_int, c_void_p, c_void_p, c_int64, c_void_p, c_void_p,
                             c_void_p, c_void_p]),
    "lya_dmat": (c_int, [H, CAT, BINS, c_int, c_double, c_uint64, c_void_p, c_void_p, c_void_p]),
    "lya_dmat_batched": (c_int, [H, CAT, c_int32, BINS, c_int, c_double, c_uint64, c_void_p, c_void_p,
                                 c_void_p]),
    "lya_xi_backward": (c_int, [H, CAT, BINS, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_void_p]),
    "lya_xi_backward_full": (c_int, [H, CAT, BINS, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                     c_void_p, c_void_p]),
    "lya_xi_batched": (c_int, [H, CAT, c_int32, BINS, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lya_autotune": (c_int, [H, CAT, BINS, POINTER(c_int32), c_void_p]),
    "lya_last_launch": (c_int, [H, POINTER(c_int64), POINTER(c_int32), POINTER(c_int32),
                                POINTER(c_int32)]),
    "lya_pair_stats": (c_int, [H, CAT, BINS, c_double, c_uint64, POINTER(c_int64), POINTER(c_int64),
                               POINTER(c_double), c_void_p]),
    "lya_set_dmat_tiles": (c_int, [H, c_int32]),
    "lya_dmat_work": (c_int, [H, CAT, BINS, c_double, c_uint64, POINTER(c_int64), POINTER(c_int64),
                              POINTER(c_double), POINTER(c_double), c_void_p]),
    "lya_xi_subsamples": (c_int, [H, CAT, BINS, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lya_xi_covariance": (c_int, [H, c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p]),
    "lya_xi3": (c_int, [H, CAT, BINS3, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lya_xi_bin_means": (c_int, [H, CAT, BINS, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lya_xi_bin_means_z": (c_int, [H, CAT, BINS, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                   c_void_p, c_void_p]),
    "lya_xcf": (c_int, [H, CAT, QSO, c_void_p, BINS, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lya_xdmat": (c_int, [H, CAT, QSO, c_void_p, BINS, c_int, c_double, c_uint64, c_void_p, c_void_p,
                          c_void_p]),
    "lya_xi1d": (c_int, [H, CAT, c_int32, c_double, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lya_flip_tally": (c_int, [H, CAT, BINS, c_double, c_uint64, POINTER(c_int64), POINTER(c_int64),
                               POINTER(c_double), POINTER(c_double), c_void_p]),
    "lya_stage_ms": (c_int, [H, c_int32, POINTER(ctypes.c_float)]),
    "lya_xi_pairs_static": (c_int, [CAT, BINS, c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p,
                                    c_void_p]),
    "lya_kernel_launches": (c_int64, []),
    "lya_capture_begin": (c_int, [H, c_void_p]),
    "lya_capture_end": (c_int, [H, POINTER(c_void_p)]),
    "lya_graph_launch": (c_int, [c_void_p, c_void_p]),
    "lya_graph_destroy": (c_int, [c_void_p]),
}

_LIB = None


class LyaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{status_string(code)} ({code}): {msg}")
        self.code = code


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblya.so (once) and declare every entry point's signature."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"liblya.so not built ({path}); run __graft_entry__.build() or "
                           "python -m paper_2507_00129_gb300.build")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def status_string(code: int) -> str:
    try:
        return load().lya_status_string(code).decode()
    except Exception:  # library not loadable: still give a name
        return {0: "LYA_OK"}.get(code, f"status {code}")


def check(handle, code: int):
    if code != LYA_OK:
        buf = ctypes.create_string_buffer(512)
        if handle:
            load().lya_last_error(handle, buf, 512)
        raise LyaError(code, buf.value.decode(errors="replace"))
