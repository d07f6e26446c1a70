"""ctypes declarations of the C ABI in ``include/mpsano.h`` (argument marshalling only).

The shared library is built in-tree by ``paper_2607_10280_b300.build``.  Loading
fails loudly when it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpsano.so")

MPS_OK = 0
STATUS_NAMES = {0: "MPS_OK", 1: "MPS_ERR_INVALID_ARG", 2: "MPS_ERR_OOM", 3: "MPS_ERR_CUDA",
                4: "MPS_ERR_TIMEOUT", 5: "MPS_ERR_UNSUPPORTED", 6: "MPS_ERR_NOT_READY",
                7: "MPS_ERR_DEVICE"}
PRECISION = {"fp64": 0, "mixed": 1, "mixed_orth64": 2, "mixed_fast": 3}
ANSATZ = {"ladder": 0, "paper": 1}
PAIR_SET = {"hv": 0, "hvd": 1}
PAULI_KERNEL = {"column": 0, "sweep": 1, "auto": 2}


class MpsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class mps_circuit(ctypes.Structure):
    _fields_ = [
        ("ansatz", ctypes.c_int32),
        ("L", ctypes.c_int32),
        ("L_per_image", ctypes.POINTER(ctypes.c_int32)),
        ("params", ctypes.c_void_p),
        ("params_n", ctypes.c_int32),
    ]


class ano_adam(ctypes.Structure):
    _fields_ = [("lr_abd", ctypes.c_float), ("lr_linear", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("mse_weight", ctypes.c_float)]


_c = ctypes
SIGNATURES = {
    "mps_create_batch": (_c.c_int, [_c.c_int32, _c.POINTER(_c.c_int32), _c.POINTER(_c.c_int32), _c.c_int32,
                                    _c.c_int32, _c.c_void_p, _c.POINTER(_c.c_void_p)]),
    "mps_destroy_batch": (_c.c_int, [_c.c_void_p]),
    "mps_reserve": (_c.c_int, [_c.c_void_p, _c.c_int32]),
    "mps_reshape_batch": (_c.c_int, [_c.c_void_p, _c.c_int32, _c.POINTER(_c.c_int32), _c.POINTER(_c.c_int32),
                                     _c.c_int32]),
    "mps_apply_circuit": (_c.c_int, [_c.c_void_p, _c.c_void_p, _c.POINTER(mps_circuit)]),
    "mps_pauli_cache": (_c.c_int, [_c.c_void_p, _c.c_int32, _c.c_void_p, _c.POINTER(_c.c_int64)]),
    "ano_features": (_c.c_int, [_c.c_void_p, _c.c_int32, _c.c_int64, _c.c_int32, _c.c_void_p, _c.c_void_p,
                                _c.c_void_p, _c.c_int32, _c.c_void_p, _c.c_void_p, _c.c_void_p]),
    "mps_sync": (_c.c_int, [_c.c_void_p]),
    "ano_status": (_c.c_int, []),
    "ano_train_workspace_floats": (_c.c_int64, [_c.c_int64, _c.c_int32, _c.c_int32]),
    "ano_train_step": (_c.c_int, [_c.c_void_p, _c.c_int32, _c.c_int64, _c.c_int32, _c.c_void_p, _c.c_void_p,
                                  _c.c_void_p, _c.c_int32, _c.c_void_p, _c.c_void_p, _c.c_int32,
                                  _c.POINTER(ano_adam), _c.c_void_p, _c.c_void_p, _c.c_void_p]),
    "mps_last_error": (_c.c_char_p, []),
    "mps_pair_count": (_c.c_int64, [_c.c_int32, _c.c_int32]),
    "mps_bond_dims": (_c.c_int, [_c.c_void_p, _c.POINTER(_c.c_int32)]),
    "mps_discarded_weight": (_c.c_int, [_c.c_void_p, _c.POINTER(_c.c_double)]),
    "mps_launch_count": (_c.c_uint64, []),
    "mps_plan_image": (_c.c_int, [_c.c_int32, _c.c_int32, _c.c_int32, _c.c_int32, _c.c_int32, _c.c_int32,
                                  _c.POINTER(_c.c_int32)]),
    "mps_set_launch_shape": (_c.c_int, [_c.c_void_p, _c.c_int32, _c.c_int32, _c.c_int32]),
    "mps_set_timing": (_c.c_int, [_c.c_void_p, _c.c_int32]),
    "mps_set_layer_pipeline": (_c.c_int, [_c.c_void_p, _c.c_int32]),
    "mps_set_half_structure": (_c.c_int, [_c.c_void_p, _c.c_int32]),
    "mps_set_block_truncation": (_c.c_int, [_c.c_void_p, _c.c_int32]),
    "mps_set_real_arithmetic": (_c.c_int, [_c.c_void_p, _c.c_int32]),
    "mps_set_pauli_sweep": (_c.c_int, [_c.c_void_p, _c.c_int32]),
    "mps_kernel_times": (_c.c_int, [_c.c_void_p, _c.POINTER(_c.c_double), _c.POINTER(_c.c_int64)]),
    "mps_pauli_cache_noalloc": (_c.c_int, [_c.c_int32, _c.c_int32, _c.c_int32, _c.c_int32, _c.c_void_p,
                                           _c.c_void_p, _c.c_int32, _c.c_void_p, _c.c_void_p, _c.c_void_p]),
}
KERNEL_KINDS = ("circuit", "renv", "pauli")

_lib = None


def lib() -> ctypes.CDLL:
    """Load the CUDA library (once).  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_2607_10280_b300.build` "
                               "(the CUDA library is required; there is no CPU path)")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def check(status: int) -> None:
    if status != MPS_OK:
        raise MpsError(status, lib().mps_last_error().decode())
