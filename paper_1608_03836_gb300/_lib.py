"""ctypes loader for libwadg.so (the C ABI declared in include/wadg.h)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwadg.so")

c_int, c_int64, c_double, c_void_p = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
P_double = ctypes.POINTER(ctypes.c_double)
P_int64 = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes); must match include/wadg.h
SIGNATURES = {
    "wadg_version": (c_int, []),
    "wadg_mesh_create": (c_int, [c_int, c_int64, P_double, c_int64, P_int64, P_double, ctypes.POINTER(c_void_p)]),
    "wadg_mesh_create_rule": (c_int, [c_int, c_int64, P_double, c_int64, P_int64, P_double, c_int, P_double,
                                      ctypes.POINTER(c_void_p)]),
    "wadg_set_operators": (c_int, [c_void_p, c_int, c_int, c_double, c_double, P_double]),
    "wadg_device_status": (c_int, [c_void_p, c_void_p]),
    "wadg_selftest_bounded_wait": (c_int, [c_void_p, ctypes.c_uint32, c_void_p]),
    "wadg_mesh_info": (c_int, [c_void_p, P_int64]),
    "wadg_volume_points": (c_int, [c_void_p, P_double]),
    "wadg_reference_rules": (c_int, [c_int, P_double, P_double, P_double, P_double]),
    "wadg_project": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "wadg_rhs": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "wadg_step": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_double, c_int, c_void_p, c_void_p]),
    "wadg_set_formulation": (c_int, [c_void_p, c_int]),
    "wadg_set_conservation": (c_int, [c_void_p, c_int]),
    "wadg_set_compensation": (c_int, [c_void_p, c_int]),
    "wadg_compensation_carry": (c_int, [c_void_p, c_void_p, c_int, c_void_p]),
    "wadg_set_planar_split": (c_int, [c_void_p, c_int]),
    "wadg_planar_info": (c_int, [c_void_p, c_void_p]),
    "wadg_step_host": (c_int, [c_void_p, c_void_p, c_void_p, ctypes.c_double, ctypes.c_double, c_int, c_void_p]),
    "wadg_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_double, c_double, c_void_p,
                           ctypes.POINTER(c_int), c_void_p]),
    "wadg_set_sources": (c_int, [c_void_p, P_double, c_double, c_double]),
    "wadg_set_receivers": (c_int, [c_void_p, c_int, P_double]),
    "wadg_energy": (c_int, [c_void_p, c_void_p, P_double, c_void_p]),
    "wadg_energy_noalloc": (c_int, [c_void_p, c_void_p, P_double, c_void_p]),
    "wadg_l2_error": (c_int, [c_void_p, c_void_p, c_void_p, c_int, P_double, c_void_p]),
    "wadg_rhs_adjoint": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "wadg_step_record": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_double, c_void_p, c_void_p, c_void_p]),
    "wadg_step_adjoint": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_void_p]),
    "wadg_receivers_adjoint": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "wadg_segment_adjoint": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_double, c_int, c_void_p, c_void_p,
                                     c_void_p, c_void_p, c_void_p, c_void_p]),
    "wadg_batch_create": (c_int, [ctypes.POINTER(c_void_p), c_int, ctypes.POINTER(c_void_p)]),
    "wadg_batch_info": (c_int, [c_void_p, P_int64]),
    "wadg_batch_set_grid": (c_int, [c_void_p, c_int]),
    "wadg_batch_set_rule": (c_int, [c_void_p, c_int]),
    "wadg_batch_autotune": (c_int, [c_void_p, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                    ctypes.POINTER(c_int), c_void_p]),
    "wadg_batch_step": (c_int, [c_void_p, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), c_double, c_double,
                                c_int, c_void_p]),
    "wadg_batch_solve": (c_int, [c_void_p, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), c_double, c_double,
                                 c_double, ctypes.POINTER(c_int), c_void_p]),
    "wadg_batch_destroy": (None, [c_void_p]),
    "wadg_batch_last_error": (ctypes.c_char_p, [c_void_p]),
    "wadg_mesh_destroy": (None, [c_void_p]),
    "wadg_status_string": (ctypes.c_char_p, [c_int]),
    "wadg_last_error": (ctypes.c_char_p, [c_void_p]),
}


class WadgError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: status {status} ({status_name(status)}){': ' + detail if detail else ''}")


_lib = None


def load() -> ctypes.CDLL:
    """Load the in-tree library; raises ImportError when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_1608_03836_gb300/build.py` "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_name(status: int) -> str:
    try:
        return load().wadg_status_string(status).decode()
    except Exception:  # pragma: no cover - only while the library is missing
        return "?"
