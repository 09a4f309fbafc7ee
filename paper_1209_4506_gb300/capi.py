"""ctypes declarations of the C ABI in include/hartree.h (argument marshalling only).

Every function keeps its C name.  Pointers are passed as integers (device or
host addresses), streams as the integer value of a cudaStream_t.  The library
is loaded from the package's ``_lib`` directory; if it is missing it is built
from ``csrc`` with nvcc, and if that fails the import fails -- there is no
other implementation to fall back on.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

HARTREE_FP64 = 0
HARTREE_FP32 = 1
HARTREE_FP32_TC_SPLIT = 2

HARTREE_OK = 0
HARTREE_ERR_INVALID = 1
HARTREE_ERR_UNSUPPORTED_SIZE = 2
HARTREE_ERR_CUDA = 3
HARTREE_ERR_OOM = 4
HARTREE_ERR_TIMEOUT = 5
HARTREE_ERR_NOT_CAPTURABLE = 6

HARTREE_FLAG_TC_BF16 = 1
HARTREE_FLAG_FUSED_SPLAT = 2

# Every symbol the public header declares (the CPU tests check the exports).
EXPORTED = (
    "hartree_plan_create",
    "hartree_plan_destroy",
    "hartree_plan_workspace_bytes",
    "hartree_atoms_reorder",
    "hartree_atoms_reorder_device",
    "hartree_splat",
    "hartree_solve_density",
    "hartree_solve",
    "hartree_forces",
    "hartree_step",
    "hartree_step_host",
    "hartree_solve_pass",
    "hartree_splat_pass",
    "hartree_plan_fused_splat",
    "hartree_plan_launch_count",
    "hartree_solve_density_noalloc",
    "hartree_plan_autotune",
    "hartree_plan_set_variants",
    "hartree_plan_device_status",
    "hartree_batch_create",
    "hartree_batch_destroy",
    "hartree_batch_offsets",
    "hartree_solve_batched",
    "hartree_batch_device_status",
    "hartree_batch_fault_inject",
    "hartree_status_string",
    "hartree_last_error",
)


class hartree_desc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("cell", ctypes.c_double * 3),
        ("sigma", ctypes.c_double),
        ("cutoff_sigmas", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("atoms_per_leaf", ctypes.c_int),
        ("max_atoms", ctypes.c_int),
        ("flags", ctypes.c_uint),
    ]


class HartreeError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[{status}] {message}")
        self.status = status


_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_i = ctypes.c_int


def lib():
    """The loaded libhartree_gb300.so (built on first use if absent)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                path = _build.build()
            L = ctypes.CDLL(path)
            L.hartree_plan_create.argtypes = [ctypes.POINTER(hartree_desc), ctypes.POINTER(_vp)]
            L.hartree_plan_destroy.argtypes = [_vp]
            L.hartree_plan_destroy.restype = None
            L.hartree_plan_workspace_bytes.argtypes = [_vp]
            L.hartree_plan_workspace_bytes.restype = ctypes.c_ulonglong
            L.hartree_atoms_reorder.argtypes = [_vp, _vp, _i, _i, _vp, _vp]
            L.hartree_atoms_reorder_device.argtypes = [_vp, _vp, _vp, _i, _i, _vp, _vp, _vp]
            L.hartree_splat.argtypes = [_vp, _vp, _vp, _i, _vp, _vp]
            L.hartree_solve_density.argtypes = [_vp, _vp, _vp, _vp, _vp]
            L.hartree_solve.argtypes = [_vp, _vp, _vp, _i, _vp, _vp, _vp, _vp]
            L.hartree_forces.argtypes = [_vp, _vp, _vp, _i, _vp, _vp, _vp, _vp]
            L.hartree_step.argtypes = [_vp, _vp, _vp, _i, _vp, _vp, _vp, _vp, _vp, _vp]
            L.hartree_step_host.argtypes = [_vp, _vp, _vp, _i, _vp, _vp, _vp]
            L.hartree_solve_pass.argtypes = [_vp, _i, _vp, _vp, _vp]
            L.hartree_splat_pass.argtypes = [_vp, _vp, _vp, _i, _vp]
            L.hartree_plan_fused_splat.argtypes = [_vp]
            L.hartree_plan_launch_count.argtypes = [_vp]
            L.hartree_plan_launch_count.restype = ctypes.c_ulonglong
            L.hartree_solve_density_noalloc.argtypes = [ctypes.POINTER(hartree_desc), _vp, _vp, _vp, _vp]
            L.hartree_plan_autotune.argtypes = [_vp, _vp, _vp]
            L.hartree_plan_set_variants.argtypes = [_vp, _vp]
            L.hartree_plan_device_status.argtypes = [_vp]
            L.hartree_batch_create.argtypes = [ctypes.POINTER(hartree_desc), _vp, _i, ctypes.POINTER(_vp)]
            L.hartree_batch_destroy.argtypes = [_vp]
            L.hartree_batch_destroy.restype = None
            L.hartree_batch_offsets.argtypes = [_vp, _vp, _vp]
            L.hartree_solve_batched.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
            L.hartree_batch_device_status.argtypes = [_vp]
            L.hartree_batch_fault_inject.argtypes = [_vp, _i, _i, ctypes.c_uint]
            L.hartree_status_string.argtypes = [_i]
            L.hartree_status_string.restype = ctypes.c_char_p
            L.hartree_last_error.argtypes = []
            L.hartree_last_error.restype = ctypes.c_char_p
            _lib = L
    return _lib


def check(status: int) -> None:
    if status != HARTREE_OK:
        L = lib()
        raise HartreeError(status, f"{L.hartree_status_string(status).decode()}: {L.hartree_last_error().decode()}")


def _call(name):
    def f(*args):
        return getattr(lib(), name)(*args)

    f.__name__ = name
    return f


hartree_plan_create = _call("hartree_plan_create")
hartree_plan_destroy = _call("hartree_plan_destroy")
hartree_plan_workspace_bytes = _call("hartree_plan_workspace_bytes")
hartree_atoms_reorder = _call("hartree_atoms_reorder")
hartree_atoms_reorder_device = _call("hartree_atoms_reorder_device")
hartree_splat = _call("hartree_splat")
hartree_solve_density = _call("hartree_solve_density")
hartree_solve = _call("hartree_solve")
hartree_forces = _call("hartree_forces")
hartree_step = _call("hartree_step")
hartree_step_host = _call("hartree_step_host")
hartree_solve_pass = _call("hartree_solve_pass")
hartree_splat_pass = _call("hartree_splat_pass")
hartree_plan_fused_splat = _call("hartree_plan_fused_splat")
hartree_plan_launch_count = _call("hartree_plan_launch_count")
hartree_solve_density_noalloc = _call("hartree_solve_density_noalloc")
hartree_plan_autotune = _call("hartree_plan_autotune")
hartree_plan_set_variants = _call("hartree_plan_set_variants")
hartree_plan_device_status = _call("hartree_plan_device_status")
hartree_status_string = _call("hartree_status_string")
hartree_last_error = _call("hartree_last_error")
hartree_batch_create = _call("hartree_batch_create")
hartree_batch_destroy = _call("hartree_batch_destroy")
hartree_batch_offsets = _call("hartree_batch_offsets")
hartree_solve_batched = _call("hartree_solve_batched")
hartree_batch_device_status = _call("hartree_batch_device_status")
hartree_batch_fault_inject = _call("hartree_batch_fault_inject")
