"""ctypes mirror of include/qaoa.h.

Loads ``_lib/libqaoa_gb300.so`` (built in-tree by ``build.py``).  There is no
fallback: if the library is missing or cannot be loaded, every entry point
raises.
"""

from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

c_int, c_int64, c_double, c_void_p = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p

QAOA_OK, QAOA_ERR_INVALID, QAOA_ERR_OOM, QAOA_ERR_CUDA, QAOA_ERR_TIMEOUT, QAOA_ERR_UNSUPPORTED = range(6)
STATUS_NAMES = {0: "QAOA_OK", 1: "QAOA_ERR_INVALID", 2: "QAOA_ERR_OOM", 3: "QAOA_ERR_CUDA",
                4: "QAOA_ERR_TIMEOUT", 5: "QAOA_ERR_UNSUPPORTED"}

QAOA_COST_F32, QAOA_COST_U8 = 0, 1
QAOA_PROBLEM_MAXCUT, QAOA_PROBLEM_WMAXCUT, QAOA_PROBLEM_SK, QAOA_PROBLEM_DKS, QAOA_PROBLEM_KVC = 0, 1, 2, 3, 4
QAOA_MIXER_X, QAOA_MIXER_EIGEN, QAOA_MIXER_X_MA, QAOA_MIXER_X_GENERAL, QAOA_MIXER_EIGEN_SYM = 0, 1, 2, 3, 4
QAOA_MIXER_GROVER = 5
QAOA_XY_RING, QAOA_XY_CLIQUE = 0, 1
QAOA_GEMM_FP32_SIMT, QAOA_GEMM_3XTF32, QAOA_GEMM_BF16X3 = 0, 1, 2
QAOA_CKPT_NONE, QAOA_CKPT_ROUND, QAOA_CKPT_PASS = 0, 1, 2


class QaoaProblem(ctypes.Structure):
    _fields_ = [("kind", c_int), ("n", c_int), ("k", c_int), ("m", c_int),
                ("edges", c_void_p), ("weights", c_void_p), ("J", c_void_p)]


class QaoaMixer(ctypes.Structure):
    _fields_ = [("kind", c_int), ("n", c_int), ("dim", c_int64), ("d_V", c_void_p),
                ("d_lambda", c_void_p), ("gemm_precision", c_int), ("k", c_int), ("id", ctypes.c_uint64)]


class QaoaJob(ctypes.Structure):
    _fields_ = [("d_cost", c_void_p), ("cost_dtype", c_int), ("mixer", ctypes.POINTER(QaoaMixer)),
                ("p", c_int), ("n_sets", c_int), ("d_angles", c_void_p), ("d_E", c_void_p),
                ("d_grad", c_void_p), ("d_init", c_void_p)]


class QaoaHostJob(ctypes.Structure):
    _fields_ = [("d_cost", c_void_p), ("cost_dtype", c_int), ("mixer", ctypes.POINTER(QaoaMixer)),
                ("p", c_int), ("n_sets", c_int), ("h_angles", c_void_p), ("h_E", c_void_p),
                ("h_grad", c_void_p), ("d_init", c_void_p)]


class QaoaXTune(ctypes.Structure):
    _fields_ = [("n", c_int), ("cost_dtype", c_int), ("cmin", c_int), ("split", c_int),
                ("nbuf_bwd_contig", c_int), ("nbuf_bwd_gather", c_int), ("ms", c_double)]


class QaoaKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", c_int64), ("total_ms", c_double),
                ("algo_bytes", c_double), ("algo_flops", c_double)]


#: Every symbol include/qaoa.h declares, with its ctypes signature.
SIGNATURES = {
    "qaoa_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_void_p]),
    "qaoa_destroy": (None, [c_void_p]),
    "qaoa_last_error": (ctypes.c_char_p, [c_void_p]),
    "qaoa_scratch_bytes": (c_int64, [c_void_p]),
    "qaoa_cost_precompute": (c_int, [c_void_p, ctypes.POINTER(QaoaProblem), c_void_p, c_int, c_int64]),
    "qaoa_dicke_states": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int64]),
    "qaoa_ring_hamiltonian": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int64]),
    "qaoa_clique_hamiltonian": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int64]),
    "qaoa_expectation": (c_int, [c_void_p, c_void_p, c_int, ctypes.POINTER(QaoaMixer), c_void_p, c_int,
                                 c_void_p, c_void_p]),
    "qaoa_gradient": (c_int, [c_void_p, c_void_p, c_int, ctypes.POINTER(QaoaMixer), c_void_p, c_int,
                              c_void_p, c_void_p, c_void_p, c_int]),
    "qaoa_expectation_batched": (c_int, [c_void_p, c_int, ctypes.POINTER(QaoaJob), c_int]),
    "qaoa_expectation_batched_host": (c_int, [c_void_p, c_int, ctypes.POINTER(QaoaHostJob), c_int]),
    "qaoa_set_profiling": (c_int, [c_void_p, c_int]),
    "qaoa_kernel_stats": (c_int, [c_void_p, ctypes.POINTER(QaoaKernelStat), c_int]),
    "qaoa_reset_stats": (None, [c_void_p]),
    "qaoa_launch_count": (c_int64, [c_void_p]),
    "qaoa_gradient_small_noalloc": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                            c_void_p]),
    "qaoa_set_checkpointing": (c_int, [c_void_p, c_int]),
    "qaoa_set_state_limit": (c_int, [c_void_p, c_int64]),
    "qaoa_x_mixer_weights": (c_int, [c_int, c_int, c_void_p, c_void_p]),
    "qaoa_xy_block_hamiltonians": (c_int, [c_int, c_int, c_int, ctypes.POINTER(c_int), c_void_p, c_void_p]),
    "qaoa_check_bounded_wait": (c_int, [c_void_p]),
    "qaoa_cost_degeneracy": (c_int, [c_void_p, ctypes.POINTER(QaoaProblem), c_void_p, c_int]),
    "qaoa_grover_batched": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "qaoa_pass_schedule": (c_int, [c_int, c_int, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int), c_int]),
    "qaoa_autotune_x": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, ctypes.POINTER(QaoaXTune)]),
    "qaoa_set_xtune": (c_int, [c_void_p, ctypes.POINTER(QaoaXTune)]),
    "qaoa_get_xtune": (c_int, [c_void_p, c_int, c_int, ctypes.POINTER(QaoaXTune)]),
}

_lock = threading.Lock()
_lib = None


class QAOAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load (building first if needed) the CUDA library; raises on failure."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB_PATH):
            raise ImportError(f"CUDA library not built: {_build.LIB_PATH}")
        lib = ctypes.CDLL(_build.LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib
