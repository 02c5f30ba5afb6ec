"""ctypes binding of libsc_level.so (the C ABI of include/sc_level.h,
include/sc_bboxset.h, include/sc_hierarchy.h and include/sc_dist.h).  Argument marshalling only: every computation runs
in the library.  There is no fallback -- if the library is missing or fails
to load, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# SC_LEVEL_LIB selects another build of the library (the checked build)
LIB_PATH = os.environ.get("SC_LEVEL_LIB") or os.path.join(HERE, "libsc_level.so")

SC_OK, SC_EINVAL, SC_ENOMEM, SC_ECUDA, SC_EDEVICE, SC_ENOTSUP = 0, -1, -2, -3, -4, -5
SC_ARITH_FP64, SC_ARITH_FIXED = 0, 1
SC_STAGING_REGISTERS, SC_STAGING_SHARED = 0, 1
SC_MODE_GRAPH, SC_MODE_PER_BOX, SC_MODE_BATCHED, SC_MODE_TIMED = 0, 1, 2, 3
SC_SET_UNION, SC_SET_INTERSECTION, SC_SET_DIFFERENCE, SC_SET_XOR = 0, 1, 2, 3
SC_PASS_ONE_ROLE, SC_PASS_WARP_SPECIALISED = 0, 1
SC_DIST_GREEDY, SC_DIST_BISECT = 0, 1
SC_DIST_STATE, SC_DIST_STAGE = 0, 1
(SC_KERNEL_STAGE, SC_KERNEL_GATHER, SC_KERNEL_STAGE_RECORD, SC_KERNEL_ADJ_A, SC_KERNEL_ADJ_B,
 SC_KERNEL_ADJ_C, SC_KERNEL_PAIR_A, SC_KERNEL_PAIR_B) = range(8)

_i32, _i64, _u32, _dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double
_vp = ctypes.c_void_p
_p64 = ctypes.POINTER(ctypes.c_int64)


class ScBox(ctypes.Structure):
    _fields_ = [("lo", _i64 * 3), ("hi", _i64 * 3), ("domain", _i32), ("reserved", _i32)]


class ScDomain(ctypes.Structure):
    _fields_ = [("lo", _i64 * 3), ("hi", _i64 * 3), ("h", _dbl), ("periodic", _u32),
                ("reserved", _u32)]


class ScCopy(ctypes.Structure):
    _fields_ = [("src_box", _i32), ("dst_box", _i32), ("src_lo", _i64 * 3),
                ("dst_lo", _i64 * 3), ("ext", _i64 * 3)]


class ScTile(ctypes.Structure):
    _fields_ = [("tile_x", _i32), ("tile_y", _i32), ("tile_z", _i32), ("reserved", _i32)]


class ScError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("sc error %d: %s" % (code, msg))
        self.code = code


_SIGS = {
    "sc_level_create": (_i32, [ctypes.POINTER(ScBox), _i32, ctypes.POINTER(ScDomain), _i32,
                               _i32, ctypes.POINTER(_vp)]),
    "sc_level_destroy": (None, [_vp]),
    "sc_level_field_size": (_i32, [_vp, _p64]),
    "sc_level_box_layout": (_i32, [_vp, _i32, _p64, _p64, _p64]),
    "sc_level_num_boxes": (_i32, [_vp, ctypes.POINTER(_i32)]),
    "sc_level_exchange_list": (_i32, [_vp, ctypes.POINTER(ScCopy), _i64, _p64]),
    "sc_level_work_items": (_i32, [_vp, ctypes.POINTER(ctypes.c_int32), _i64, _p64]),
    "sc_level_set_arith": (_i32, [_vp, _i32]),
    "sc_level_set_tuning": (_i32, [_vp, _i32, ctypes.POINTER(ScTile), _i32]),
    "sc_level_size_classes": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "sc_level_get_tuning": (_i32, [_vp, _i32, ctypes.POINTER(ScTile)]),
    "sc_level_set_fusion": (_i32, [_vp, _i32]),
    "sc_level_get_fusion": (_i32, [_vp, ctypes.POINTER(_i32)]),
    "sc_level_set_staging": (_i32, [_vp, _i32]),
    "sc_level_get_staging": (_i32, [_vp, ctypes.POINTER(_i32)]),
    "sc_level_autotune": (_i32, [_vp, _i32, _dbl, _dbl, ctypes.c_char_p, _vp]),
    "sc_level_set_pass_kernel": (_i32, [_vp, _i32]),
    "sc_level_get_pass_kernel": (_i32, [_vp, ctypes.POINTER(_i32)]),
    "sc_level_arm_wait_test": (_i32, [_vp]),
    "sc_level_fill_ghosts": (_i32, [_vp, _vp, _vp]),
    "sc_level_apply_laplacian": (_i32, [_vp, _vp, _vp, _vp]),
    "sc_level_rk4_step": (_i32, [_vp, _vp, _vp, _vp, ctypes.POINTER(_dbl), _i32, _i32, _i32,
                                 _vp]),
    "sc_level_rk4_step_host": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_dbl), _i32,
                                      _i32, _vp]),
    "sc_level_misfit": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "sc_level_grad": (_i32, [_vp, _vp, _vp, _vp, ctypes.POINTER(_dbl), _i32, _i32, _i32, _vp,
                             _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sc_level_forward_tape": (_i32, [_vp, _vp, _vp, _vp, ctypes.POINTER(_dbl), _i32, _i32, _i32,
                                     _vp, _vp, _vp]),
    "sc_level_backward_tape": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sc_level_sync": (_i32, [_vp, _vp]),
    "sc_level_launch_count": (_i32, [_vp, _p64]),
    "sc_level_kernel_times": (_i32, [_vp, ctypes.POINTER(_dbl), _p64, ctypes.POINTER(_dbl),
                                     _p64]),
    "sc_level_kernel_time": (_i32, [_vp, _i32, ctypes.POINTER(_dbl), _p64]),
    "sc_level_set_profiling": (_i32, [_vp, _i32]),
    "sc_box_rk4_step_noalloc": (_i32, [_vp, _vp, _vp, _i32, _i32, _i32, _dbl, _dbl, _i32, _vp]),
    "sc_last_error": (ctypes.c_char_p, []),
    "sc_bboxset_op": (_i32, [_i32, _p64, _i64, _p64, _i64, _p64, _i64, _p64]),
    "sc_bboxset_derivative": (_i32, [_p64, _i64, _p64, _i64, _p64]),
    "sc_bboxset_expand_shift": (_i32, [_p64, _i64, _p64, _p64, _p64, _p64, _i64, _p64]),
    "sc_bboxset_size": (_i32, [_p64, _i64, _p64]),
    "sc_bboxset_coarsen": (_i32, [_p64, _i64, _i64, _p64, _i64, _p64]),
    "sc_hierarchy_create": (_i32, [_vp, _vp, _i32, _i32, ctypes.POINTER(_vp)]),
    "sc_hierarchy_destroy": (None, [_vp]),
    "sc_hierarchy_counts": (_i32, [_vp, _p64, _p64]),
    "sc_hierarchy_prolongation_points": (_i32, [_vp, _p64, _i64, _p64]),
    "sc_hierarchy_restriction_points": (_i32, [_vp, _p64, _i64, _p64]),
    "sc_hierarchy_prolongate": (_i32, [_vp, _vp, _vp, _vp, _vp, _dbl, _vp, _vp, _vp]),
    "sc_hierarchy_restrict": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "sc_hierarchy_step": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _dbl, _i32, _i32, _vp]),
    "sc_dist_partition": (_i32, [ctypes.POINTER(ScBox), _i32, _i32, _i32,
                                 ctypes.POINTER(_i32)]),
    "sc_dist_create": (_i32, [ctypes.POINTER(ScBox), _i32, ctypes.POINTER(ScDomain), _i32, _i32,
                              ctypes.POINTER(_i32), _i32, _i32, ctypes.POINTER(_vp)]),
    "sc_dist_info": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                            ctypes.POINTER(_i32)]),
    "sc_dist_global_box": (_i32, [_vp, _i32, ctypes.POINTER(_i32)]),
    "sc_dist_buffer_sizes": (_i32, [_vp, _p64, _p64]),
    "sc_dist_peer": (_i32, [_vp, _i32, ctypes.POINTER(_i32), _p64, _p64, _p64, _p64]),
    "sc_dist_list": (_i32, [_vp, _i32, _i32, ctypes.POINTER(ScCopy), _i64, _p64]),
    "sc_dist_pack": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp]),
    "sc_dist_unpack": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp]),
    "sc_dist_rk4_begin": (_i32, [_vp, _vp, _vp, _vp, ctypes.POINTER(_dbl), _i32, _vp]),
    "sc_dist_rk4_pass": (_i32, [_vp, _vp, _vp, _i32, _vp]),
}

_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library.  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    "libsc_level.so is missing: build it with "
                    "`python -m paper_1308_1343_gb300.build` (there is no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def declared_symbols():
    return list(_SIGS)


def check(rc: int) -> None:
    if rc != SC_OK:
        msg = lib().sc_last_error()
        raise ScError(rc, msg.decode() if msg else "")
