"""ctypes declarations of the C ABI in include/pdscp.h.

Loading fails loudly when libpdscp.so has not been built: there is no CPU
fallback anywhere in the product path.
"""

import ctypes
import os

from .build import LIB

PDSCP_OK = 0
STATUS_NAMES = {
    0: "PDSCP_OK", 1: "PDSCP_ERR_INVALID_ARG", 2: "PDSCP_ERR_CUDA", 3: "PDSCP_ERR_TIMEOUT",
    4: "PDSCP_ERR_NOT_SEPARABLE", 5: "PDSCP_ERR_NOT_CONVERGED", 6: "PDSCP_ERR_NUMERIC",
    7: "PDSCP_ERR_NOT_IMPLEMENTED", 8: "PDSCP_ERR_WORKSPACE",
}
SES, SVM = 0, 1
F32, BF16 = 0, 1
RULES_NONE, RULES_PRACTICAL = 0, 1
MODE_PRACTICAL, MODE_THEORY, MODE_CERTIFIED, MODE_CORESET = 0, 1, 2, 3
OUT_RUNNING, OUT_SEPARATED, OUT_BEAT_ALPHA, OUT_STALLED = 0, 1, 2, 3
MAX_D = 1024

c_i32, c_i64, c_dbl, c_sz, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p


class StepOut(ctypes.Structure):
    """pdscp_step_out (72 bytes)."""
    _fields_ = [("oracle_value", c_dbl), ("objective", c_dbl), ("lower_bound", c_dbl),
                ("upper_bound", c_dbl), ("t", c_i64), ("failed", c_i32), ("stopped", c_i32),
                ("status", c_i32), ("outcome", c_i32), ("k", c_dbl), ("dual_bound", c_dbl)]


class Options(ctypes.Structure):
    """pdscp_options."""
    _fields_ = [("eps", c_dbl), ("delta", c_dbl), ("patience", c_i32), ("mode", c_i32),
                ("max_iters", c_i64), ("poll_every", c_i32), ("max_steps", c_i32), ("eta", c_dbl)]


class Report(ctypes.Structure):
    """pdscp_report."""
    _fields_ = [("value", c_dbl), ("lower_bound", c_dbl), ("upper_bound", c_dbl), ("D", c_dbl),
                ("search_L", c_dbl), ("search_U", c_dbl), ("iters", c_i64),
                ("search_steps", c_i32), ("status", c_i32)]


assert ctypes.sizeof(StepOut) == 72

# name -> (restype, argtypes); every entry point declared in include/pdscp.h
SIGNATURES = {
    "pdscp_version": (c_i32, []),
    "pdscp_polytope_distance": (c_i32, [c_vp, c_i32, c_vp, c_i32, c_i32, c_dbl, c_i32, c_vp, c_vp, c_vp]),
    "pdscp_meb_dual": (c_i32, [c_vp, c_i32, c_i32, c_dbl, c_i32, c_vp, c_vp, c_vp, c_vp]),
    "pdscp_last_error": (ctypes.c_char_p, []),
    "pdscp_workspace_size": (c_i32, [c_i32, c_i64, c_i32, ctypes.POINTER(c_sz)]),
    "pdscp_state_size": (c_i32, [c_i32, c_i32, ctypes.POINTER(c_sz)]),
    "pdscp_bounds": (c_i32, [c_i32, c_vp, c_i32, c_vp, c_i64, c_i32, c_vp, c_sz, c_vp, c_vp]),
    "mwu_state_init": (c_i32, [c_i32, c_vp, c_i32, c_i64, c_i32, c_i32, c_dbl, c_i32, c_vp, c_vp, c_sz, c_vp]),
    "mwu_step": (c_i32, [c_i32, c_vp, c_i32, c_vp, c_vp, c_i64, c_i32, c_dbl, c_dbl, c_dbl, c_i32,
                         c_vp, c_vp, c_sz, c_vp, c_vp]),
    "mwu_run": (c_i32, [c_i32, c_vp, c_i32, c_vp, c_vp, c_i64, c_i32, c_dbl, c_dbl, c_dbl, c_i64, c_vp, c_vp, c_sz,
                        c_vp, c_vp]),
    "mwu_step_noalloc": (c_i32, [c_i32, c_vp, c_i32, c_vp, c_vp, c_i64, c_i32, c_dbl, c_dbl, c_dbl, c_i32,
                                 c_vp, c_vp, c_vp]),
    "mwu_state_read": (c_i32, [c_i32, c_i32, c_vp, c_vp, c_vp, c_vp]),
    "mwu_state_set": (c_i32, [c_i32, c_vp, c_i32, c_vp, c_vp, c_i64, c_i32, c_i64, c_vp, c_dbl, c_vp, c_vp,
                              c_sz, c_vp]),
    "ses_solve": (c_i32, [c_vp, c_i32, c_vp, c_i64, c_i32, ctypes.POINTER(Options), c_vp, c_sz, c_vp,
                          c_vp, ctypes.POINTER(Report)]),
    "svm_solve": (c_i32, [c_vp, c_i32, c_vp, c_i64, c_i32, ctypes.POINTER(Options), c_vp, c_sz, c_vp,
                          c_vp, ctypes.POINTER(Report)]),
    "ses_batch_workspace_size": (c_i32, [c_i32, c_vp, c_vp, c_i32, ctypes.POINTER(c_sz)]),
    "ses_batch_init": (c_i32, [c_i32, c_vp, c_i32, c_i64, c_vp, c_vp, c_vp, c_i32, c_vp, c_sz, c_vp]),
    "ses_batch_step": (c_i32, [c_i32, c_vp, c_i32, c_vp, c_vp, c_vp, c_sz, c_vp, c_vp]),
    "ses_batch_read": (c_i32, [c_i32, c_vp, c_vp, c_vp, c_vp]),
    "ses_batch_solve_init": (c_i32, [c_i32, c_vp, c_i32, c_i64, c_vp, c_vp, c_vp, c_i32, c_vp, c_vp, c_sz, c_vp]),
    "ses_batch_solve_run": (c_i32, [c_i32, c_vp, c_vp, c_sz, c_i32, c_i64, c_vp, ctypes.POINTER(c_i64),
                                    ctypes.POINTER(c_i32)]),
    "ses_batch_solve_read": (c_i32, [c_i32, c_vp, c_dbl, c_vp, c_vp, c_vp]),
    "svm_batch_workspace_size": (c_i32, [c_i32, c_vp, c_vp, c_i32, ctypes.POINTER(c_sz)]),
    "svm_batch_init": (c_i32, [c_i32, c_vp, c_i32, c_i64, c_vp, c_vp, c_vp, c_vp, c_i64, c_vp, c_i32, c_vp, c_sz,
                               c_vp]),
    "svm_batch_step": (c_i32, [c_i32, c_vp, c_i32, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp, c_vp]),
    "svm_batch_read": (c_i32, [c_i32, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "svm_batch_solve_init": (c_i32, [c_i32, c_vp, c_i32, c_i64, c_vp, c_vp, c_vp, c_vp, c_i64, c_vp, c_i32, c_vp,
                                     c_vp, c_sz, c_vp]),
    "svm_batch_solve_run": (c_i32, [c_i32, c_vp, c_vp, c_vp, c_sz, c_i32, c_i64, c_vp, ctypes.POINTER(c_i64),
                                    ctypes.POINTER(c_i32)]),
    "svm_batch_solve_read": (c_i32, [c_i32, c_vp, c_dbl, c_vp, c_vp, c_vp]),
    "ses_batch_autotune": (c_i32, [c_i32, c_vp, c_i32, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp,
                                   ctypes.POINTER(c_i32), ctypes.POINTER(ctypes.c_float), ctypes.POINTER(c_i32),
                                   ctypes.POINTER(c_i32)]),
    "ses_batch_set_launch": (c_i32, [c_i32, c_vp, c_vp, c_i32, c_i32, c_vp]),
    "mwu_shard_row_width": (c_i32, [c_i32, c_i32, ctypes.POINTER(c_i32)]),
    "mwu_shard_init": (c_i32, [c_i32, c_vp, c_i32, c_i32, c_i32, c_dbl, c_i32, c_vp, c_vp, c_sz, c_vp]),
    "mwu_shard_partial": (c_i32, [c_i32, c_vp, c_i32, c_vp, c_vp, c_i64, c_i32, c_i32, c_dbl, c_dbl, c_dbl,
                                  c_i32, c_vp, c_vp, c_sz, c_vp, c_vp]),
    "mwu_shard_finish": (c_i32, [c_i32, c_vp, c_i32, c_vp, c_i32, c_vp, c_i32, c_dbl, c_dbl, c_dbl, c_i32,
                                 c_vp, c_vp, c_vp]),
    "ses_multi_state_stride": (c_i32, [c_i32, ctypes.POINTER(c_sz)]),
    "ses_multi_workspace_size": (c_i32, [c_i32, c_i32, ctypes.POINTER(c_sz)]),
    "ses_multi_step": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp, c_vp]),
    "mwu_backward_workspace_size": (c_i32, [c_i32, c_i64, c_i32, c_i64, ctypes.POINTER(c_sz)]),
    "mwu_backward": (c_i32, [c_i32, c_vp, c_i32, c_vp, c_vp, c_i64, c_i32, c_dbl, c_dbl, c_dbl, c_i64, c_vp,
                             c_vp, c_sz, c_vp, c_vp, c_vp]),
}

_lib = None


class PdscpError(RuntimeError):
    """A C-ABI call returned a status other than PDSCP_OK."""

    def __init__(self, status, fn, msg):
        self.status = status
        super().__init__(f"{fn}: {STATUS_NAMES.get(status, status)}: {msg}")


def load(path=None):
    """Load libpdscp.so (built in-tree by ``paper_2405_09157_gb300.build``)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB
    if not os.path.exists(p):
        raise ImportError(f"libpdscp.so not found at {p}: build it first with "
                          "`python -m paper_2405_09157_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def check(status, fn):
    if status != PDSCP_OK:
        msg = load().pdscp_last_error()
        raise PdscpError(status, fn, msg.decode() if msg else "")
    return status
