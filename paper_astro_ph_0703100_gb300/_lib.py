"""ctypes view of libcunbody.so (the C ABI of include/cunbody.h).

Loading fails loudly when the library has not been built: there is no
fallback path.
"""

from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcunbody.so")

c_i64 = ctypes.c_int64
c_i32 = ctypes.c_int32
c_f32 = ctypes.c_float
c_f64 = ctypes.c_double
c_size = ctypes.c_size_t
c_int = ctypes.c_int
vp = ctypes.c_void_p


class cn_tune(ctypes.Structure):
    _fields_ = [
        ("i_per_thread", c_i32),
        ("threads", c_i32),
        ("j_tile", c_i32),
        ("stages", c_i32),
        ("ctas_per_sm", c_i32),
        ("chunk_units", c_i32),
        ("j_lanes", c_i32),
    ]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


# name -> (restype, argtypes); the order of the declarations in include/cunbody.h
SIGNATURES = {
    "cn_force": (c_int, [c_i64, vp, c_i64, vp, c_f32, vp, vp, vp]),
    "cn_force_ws": (c_int, [c_i64, vp, c_i64, vp, c_f32, vp, vp, vp, c_size, vp]),
    "cn_force_dd": (c_int, [c_i64, vp, c_i64, vp, c_f32, vp, vp, vp]),
    "cn_force_dd_ws": (c_int, [c_i64, vp, c_i64, vp, c_f32, vp, vp, vp, c_size, vp]),
    "cn_workspace_bytes": (c_size, [c_int, c_i64, c_i64]),
    "cn_force_noalloc": (c_int, [c_i64, vp, c_i64, vp, c_f32, vp, vp, vp]),
    "cn_force_symmetric": (c_int, [c_i64, vp, c_f32, vp, vp, vp]),
    "cn_force_eps_i": (c_int, [c_i64, vp, c_i64, vp, vp, vp, vp]),
    "cn_batch_plan_create": (c_int, [c_i32, vp, vp, vp, c_int, ctypes.POINTER(vp)]),
    "cn_batch_plan_destroy": (c_int, [vp]),
    "cn_batch_plan_workspace_bytes": (c_size, [vp]),
    "cn_batch_plan_info": (c_int, [vp, ctypes.POINTER(c_i64), ctypes.POINTER(c_f64)]),
    "cn_force_batched": (c_int, [vp, vp, vp, vp, vp, c_size, vp]),
    "cn_batch_plan_capture": (c_int, [vp, vp, vp, vp, vp, c_size, vp]),
    "cn_batch_plan_launch": (c_int, [vp, vp]),
    "cn_list_plan_create": (c_int, [c_i32, vp, vp, vp, vp, vp, c_int, ctypes.POINTER(vp)]),
    "cn_list_plan_create_indexed": (c_int, [c_i32, vp, vp, vp, vp, vp, c_i64, c_i64, vp, c_int, ctypes.POINTER(vp)]),
    "cn_force_lists": (c_int, [vp, vp, vp, vp, vp, vp, c_size, vp]),
    "cn_list_plan_capture": (c_int, [vp, vp, vp, vp, vp, vp, c_size, vp]),
    "cn_force_adjoint": (c_int, [c_i64, vp, c_f32, vp, vp, vp, vp]),
    "cn_force_jerk": (c_int, [c_i64, vp, vp, c_i64, vp, vp, c_f32, vp, vp, vp, vp]),
    "cn_potential_energy": (c_int, [c_i64, vp, vp, vp, vp]),
    "cn_potential_energy_dd": (c_int, [c_i64, vp, vp, vp, vp]),
    "cn_force_host": (c_int, [c_i64, vp, c_i64, vp, c_f32, vp, vp, vp]),
    "cn_force_host_f64": (c_int, [vp, vp, vp, c_f64, vp, c_int, c_int]),
    "cn_tune_get": (c_int, [c_int, c_i64, c_i64, ctypes.POINTER(cn_tune)]),
    "cn_tune_set": (c_int, [c_int, c_i64, c_i64, ctypes.POINTER(cn_tune)]),
    "cn_tune_save": (c_int, [ctypes.c_char_p]),
    "cn_tune_load": (c_int, [ctypes.c_char_p, ctypes.POINTER(c_i32)]),
    "cn_autotune": (c_int, [c_int, c_i64, vp, c_i64, vp, c_f32, vp, vp, c_int, vp, ctypes.POINTER(cn_tune)]),
    "cn_autotune_batched": (c_int, [c_i32, vp, vp, vp, vp, vp, c_int, vp, ctypes.POINTER(cn_tune)]),
    "cn_get_device_status": (c_int, [vp]),
    "cn_set_wait_limit_ns": (c_int, [ctypes.c_uint64]),
    "cn_debug_timeout_probe": (c_int, [vp]),
    "cn_probe_peaks": (c_int, [vp, ctypes.POINTER(c_f64)]),
    "cn_status_string": (ctypes.c_char_p, [c_int]),
    "cn_last_error_message": (ctypes.c_char_p, []),
    "cn_version": (ctypes.c_char_p, []),
}

STATUS = {
    0: "CN_OK",
    1: "CN_ERR_INVALID_ARG",
    2: "CN_ERR_MISALIGNED",
    3: "CN_ERR_CUDA",
    4: "CN_ERR_TIMEOUT",
    5: "CN_ERR_UNSUPPORTED_DEVICE",
    6: "CN_ERR_WORKSPACE",
    7: "CN_ERR_HOST",
}

_lock = threading.Lock()
_lib = None


class CunbodyError(RuntimeError):
    """A libcunbody call returned a status other than CN_OK."""

    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        self.code = STATUS.get(status, f"status {status}")
        super().__init__(f"{where}: {self.code}: {detail}")


def load(path: str | None = None):
    """Load libcunbody.so (and declare its signatures); raises if it is missing.
    CUNBODY_LIB, when set, names another build of the library to load (for
    instance the bounds-checked libcunbody_debug.so)."""
    global _lib
    if _lib is not None:  # loaded: no lock on the per-call path
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or os.environ.get("CUNBODY_LIB") or LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(
                f"libcunbody.so is not built ({path} missing): run "
                "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(status: int, where: str) -> None:
    if status != 0:
        msg = load().cn_last_error_message()
        raise CunbodyError(status, where, msg.decode() if msg else "")
