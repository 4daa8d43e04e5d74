"""ctypes binding of the engine's C ABI (include/lbm.h), same names, marshalling only.

Every computation runs in the CUDA library ``liblbm_gb300.so``; this module
only converts arguments.  Importing it without the built library raises:
there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (POINTER, Structure, c_char_p, c_double, c_int, c_int32, c_int64, c_size_t,
                    c_uint32, c_uint8, c_void_p)

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm_gb300.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ESTATE, LBM_ENONFINITE, LBM_ETIMEOUT = \
    0, -1, -2, -3, -4, -5, -6
LBM_D2Q9, LBM_D2Q21 = 9, 21
LBM_FP64, LBM_FP32, LBM_FP16S, LBM_BF16S = 0, 1, 2, 3
LBM_PSI_EXP, LBM_PSI_EOS = 0, 1
STORAGE = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16s": LBM_FP16S, "bf16s": LBM_BF16S}
LBM_ROUND_STOCHASTIC, LBM_ROUND_NEAREST = 0, 1
ROUNDING = {"stochastic": LBM_ROUND_STOCHASTIC, "nearest": LBM_ROUND_NEAREST}
ERRNAMES = {LBM_EINVAL: "LBM_EINVAL", LBM_ENOMEM: "LBM_ENOMEM", LBM_ECUDA: "LBM_ECUDA",
            LBM_ESTATE: "LBM_ESTATE", LBM_ENONFINITE: "LBM_ENONFINITE",
            LBM_ETIMEOUT: "LBM_ETIMEOUT"}


class lbm_params(Structure):
    _fields_ = [
        ("nx", c_int32), ("ny", c_int32), ("lattice", c_int32), ("storage", c_int32),
        ("psi_kind", c_int32), ("project", c_int32),
        ("tau", c_double), ("G", c_double), ("rho0", c_double),
        ("eos_theta_v", c_double), ("eos_theta_u", c_double), ("eos_theta_l", c_double),
        ("eos_rho1", c_double), ("eos_rho2", c_double),
        ("body_force", c_double * 2), ("shift_rho", c_double),
        ("check_every", c_int32), ("tile_rows", c_int32),
        ("rounding", c_int32), ("reserved", c_int32),
    ]


ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_void_p)


class lbm_allocator(Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", c_void_p)]


class lbm_layout(Structure):
    _fields_ = [
        ("bytes_per_node", c_int64), ("pitch", c_int64), ("strip_width", c_int32),
        ("tile_rows", c_int32), ("grid_x", c_int32), ("grid_y", c_int32), ("stages", c_int32),
        ("ghost_x", c_int32), ("ghost_y", c_int32), ("device_bytes", c_int64),
    ]


# Every symbol declared in include/lbm.h, with its ctypes signature.
_DP = POINTER(c_double)
SIGNATURES = {
    "lbm_params_default": (c_int, [POINTER(lbm_params)]),
    "lbm_create": (c_int, [POINTER(lbm_params), POINTER(lbm_allocator), c_void_p, POINTER(c_void_p)]),
    "lbm_set_stream": (c_int, [c_void_p, c_void_p]),
    "lbm_set_wall": (c_int, [c_void_p, _DP, _DP, _DP, c_double, c_double, c_double, _DP]),
    "lbm_set_populations": (c_int, [c_void_p, _DP]),
    "lbm_set_equilibrium": (c_int, [c_void_p, _DP, _DP, _DP, _DP]),
    "lbm_step": (c_int, [c_void_p, c_int64]),
    "lbm_moments": (c_int, [c_void_p, _DP, _DP, _DP]),
    "lbm_moments_device": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "lbm_get_populations": (c_int, [c_void_p, _DP]),
    "lbm_totals": (c_int, [c_void_p, _DP]),
    "lbm_steps_done": (c_int, [c_void_p, POINTER(c_int64)]),
    "lbm_get_clock": (c_int, [c_void_p, POINTER(c_int64), POINTER(c_uint32), _DP]),
    "lbm_set_clock": (c_int, [c_void_p, c_int64, c_uint32]),
    "lbm_sync": (c_int, [c_void_p]),
    "lbm_destroy": (c_int, [c_void_p]),
    "lbm_last_error": (c_char_p, [c_void_p]),
    "lbm_get_layout": (c_int, [c_void_p, POINTER(lbm_layout)]),
    "lbm_debug_stall_next_step": (c_int, [c_void_p, c_int32]),
    "lbm_wall_gaussian_filter": (c_int, [c_int32, c_int32, c_int32, POINTER(c_uint8), c_int32,
                                         c_int32, _DP, _DP, _DP]),
    "lbm_wall_core_tail": (c_int, [c_int32, c_int32, _DP, _DP, c_double, c_double, c_double,
                                   c_double, c_double, _DP, _DP, _DP]),
    "lbm_reduce3_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
    "lbm_batch_create": (c_int, [POINTER(lbm_allocator), c_void_p, POINTER(c_void_p)]),
    "lbm_batch_add": (c_int, [c_void_p, c_void_p]),
    "lbm_batch_remove": (c_int, [c_void_p, c_void_p]),
    "lbm_batch_size": (c_int, [c_void_p, POINTER(c_int32)]),
    "lbm_batch_launches_per_step": (c_int, [c_void_p, POINTER(c_int32)]),
    "lbm_batch_set_tiling": (c_int, [c_void_p, c_int32, c_int32]),
    "lbm_batch_use_tuned": (c_int, [c_void_p, POINTER(c_int32)]),
    "lbm_batch_step": (c_int, [c_void_p, c_int64]),
    "lbm_batch_autotune": (c_int, [c_void_p, c_int32, POINTER(c_int32), POINTER(c_int32),
                                   POINTER(c_double)]),
    "lbm_batch_destroy": (c_int, [c_void_p]),
    "lbm_batch_last_error": (c_char_p, [c_void_p]),
}


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRNAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build the CUDA engine first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(rc: int, ctx=None):
    if rc != LBM_OK:
        msg = load().lbm_last_error(ctx)
        raise LbmError(rc, msg.decode() if msg else "")


def check_batch(rc: int, batch=None):
    if rc != LBM_OK:
        msg = load().lbm_batch_last_error(batch)
        raise LbmError(rc, msg.decode() if msg else "")


def dptr(a):
    """ctypes double* of a C-contiguous float64 numpy array (None -> NULL)."""
    if a is None:
        return None
    return a.ctypes.data_as(_DP)
