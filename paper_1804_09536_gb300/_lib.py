"""ctypes binding of the C ABI in include/tfft.h (argument marshalling only).

Every function of the header is bound under the same name; a non-zero status
raises ``TfftError`` with the library's own message.  The shared library is
the in-tree ``libtfft.so`` built by ``paper_1804_09536_gb300.build``; if it is
missing, loading raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtfft.so")

TFFT_FORWARD = -1
TFFT_BACKWARD = 1
TFFT_C2C = 0
TFFT_R2C = 1
TFFT_BATCH_PERSISTENT = 0
TFFT_BATCH_STREAMS = 1
TFFT_FP32 = 0
TFFT_TC_BF16X3 = 1
TFFT_TC_FP16X3 = 2
TFFT_NORM_FORWARD = 0
TFFT_NORM_BACKWARD = 4
TFFT_NO_TMA = 8
TFFT_NO_GRAPH = 16
TFFT_MODE_FUSED = 0
TFFT_MODE_UNFUSED = 1
TFFT_MODE_PACKED = 2

STATUS = {0: "TFFT_OK", 1: "TFFT_EINVAL", 2: "TFFT_EUNSUPPORTED", 3: "TFFT_EALIGN",
          4: "TFFT_EWORKSPACE", 5: "TFFT_ECUDA", 6: "TFFT_ESTATE"}

_i64p = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p

# name -> argument types (all return int status unless listed in _RESTYPE)
SIGNATURES = {
    "tfft_status_string": [ctypes.c_int],
    "tfft_last_error": [],
    "tfft_version": [],
    "tfft_decompose": [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _i64p, _i64p],
    "tfft_plan_create": [ctypes.POINTER(_vp), ctypes.c_int, _i64p, ctypes.c_int,
                         ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "tfft_plan_destroy": [_vp],
    "tfft_plan_num_stages": [_vp, ctypes.POINTER(ctypes.c_int)],
    "tfft_plan_num_ranks": [_vp, ctypes.POINTER(ctypes.c_int)],
    "tfft_plan_stage_axis": [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "tfft_plan_stage_elems": [_vp, ctypes.c_int, ctypes.c_int, _i64p],
    "tfft_plan_local_box": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64p, _i64p, _i64p],
    "tfft_plan_state_bytes": [_vp, ctypes.POINTER(ctypes.c_size_t)],
    "tfft_plan_bind": [_vp, _vp, ctypes.c_size_t, _vp],
    "tfft_plan_workspace_bytes": [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)],
    "tfft_redistribute": [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp],
    "tfft_partial": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp],
    "tfft_execute": [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, ctypes.c_size_t, _vp],
    "tfft_plan_num_launches": [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "tfft_plan_set_launch_events": [_vp, ctypes.POINTER(_vp), ctypes.c_int],
    "tfft_adjoint": [_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_size_t, _vp, _vp],
    "tfft_weighted_energy": [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp],
    "tfft_weighted_energy_grad": [_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_size_t, _vp, _vp],
    "tfft_host_space_bytes": [_vp, ctypes.POINTER(ctypes.c_size_t)],
    "tfft_execute_host": [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.POINTER(_vp),
                          ctypes.POINTER(_vp), _vp, ctypes.c_size_t, _vp],
    "tfft_weight_scale": [_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_double, _vp, _vp],
    "tfft_batch_create": [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_vp), ctypes.c_int],
    "tfft_batch_destroy": [_vp],
    "tfft_batch_state_bytes": [_vp, ctypes.POINTER(ctypes.c_size_t)],
    "tfft_batch_bind": [_vp, _vp, ctypes.c_size_t, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                        ctypes.POINTER(_vp), _vp],
    "tfft_batch_execute": [_vp, _vp],
    "tfft_batch_autotune": [_vp, ctypes.c_int, _vp],
    "tfft_batch_num_items": [_vp, _i64p, ctypes.POINTER(ctypes.c_int)],
    "tfft_batch_variant": [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "tfft_batch_segment": [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "tfft_batch_set_variant": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp],
    "tfft_batch_set_wait_limit": [_vp, ctypes.c_longlong],
    "tfft_batch_set_executor": [_vp, ctypes.c_int, ctypes.c_int],
    "tfft_batch_executor": [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "tfft_plan_set_wait_limit": [_vp, ctypes.c_uint32],
    "tfft_batch_device_status": [_vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int, _vp],
    "tfft_execute_noalloc": [_vp, ctypes.c_int, _vp, _vp, _vp],
    "tfft_plan_device_status": [_vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int, _vp],
    "tfft_plan_copy_tasks": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64p, ctypes.c_int64, _i64p],
    "tfft_plan_launch_info": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_char_p,
                              ctypes.c_int, _i64p],
}
_RESTYPE = {"tfft_status_string": ctypes.c_char_p, "tfft_last_error": ctypes.c_char_p}


class TfftError(RuntimeError):
    def __init__(self, status, func, msg):
        self.status = status
        super().__init__(f"{func} -> {STATUS.get(status, status)}: {msg}")


_lib = None


def load(path: str = LIB_PATH):
    """Load libtfft.so and declare its prototypes.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with paper_1804_09536_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = _RESTYPE.get(name, ctypes.c_int)
    _lib = lib
    return lib


def call(name, *args):
    """Call an ABI function; raise TfftError on a non-zero status."""
    lib = load()
    rc = getattr(lib, name)(*args)
    if rc != 0:
        msg = lib.tfft_last_error()
        raise TfftError(rc, name, msg.decode() if msg else "")
    return rc
