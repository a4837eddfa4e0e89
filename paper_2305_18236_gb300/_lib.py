"""ctypes binding of the C ABI in ``include/gemm.h``.

Argument marshalling only: every function here forwards plain pointers,
sizes and a CUDA stream handle to ``libgb300gemm.so``; all arithmetic runs
in the library's CUDA kernels.  There is no fallback: if the library is not
built, or the device is not an sm_103 GPU, calls raise.
"""
import ctypes
import os

from . import build as _build

OP_N, OP_T = 0, 1
MODE_F32_SIMT, MODE_BF16, MODE_BF16X3 = 0, 1, 2
MODES = {"f32_simt": MODE_F32_SIMT, "simt": MODE_F32_SIMT, "bf16": MODE_BF16,
         "bf16x3": MODE_BF16X3}

LOWER, UPPER = 0, 1
UPLOS = {"lower": LOWER, "upper": UPPER}
LAYOUT_AUTO, LAYOUT_K_MAJOR, LAYOUT_AS_STORED = 0, 1, 2
LAYOUTS = {"auto": LAYOUT_AUTO, "k_major": LAYOUT_K_MAJOR, "as_stored": LAYOUT_AS_STORED}
SPLIT_AUTO, SPLIT_PREPASS, SPLIT_IN_KERNEL, SPLIT_IN_KERNEL_A, SPLIT_IN_KERNEL_B = 0, 1, 2, 3, 4
SPLIT_PLACES = {"auto": SPLIT_AUTO, "prepass": SPLIT_PREPASS, "in_kernel": SPLIT_IN_KERNEL,
                "in_kernel_a": SPLIT_IN_KERNEL_A, "in_kernel_b": SPLIT_IN_KERNEL_B}
SPLITK_AUTO, SPLITK_LAUNCH = 0, 1
SPLITK_REDUCES = {"auto": SPLITK_AUTO, "launch": SPLITK_LAUNCH}

GEMM_OK = 0
GEMM_ERR_ARG = -1
GEMM_ERR_ALIGN = -2
GEMM_ERR_WORKSPACE = -3
GEMM_ERR_CUDA = -4
GEMM_ERR_TIMEOUT = -5
GEMM_ERR_UNSUPPORTED = -6
GEMM_ERR_DEVICE = -7

GROUPED_AUTOTUNE, GROUPED_GRAPH = 1, 2

_i32, _i64, _f32, _vp, _sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p, ctypes.c_size_t


class gemm_config_t(ctypes.Structure):
    _fields_ = [("bn", _i32), ("bk", _i32), ("stages", _i32), ("split_k", _i32),
                ("raster_group", _i32), ("max_ctas", _i32), ("promote_k", _i32),
                ("cta_group", _i32), ("wait_poll_limit", _i64), ("operand_layout", _i32),
                ("split_place", _i32), ("splitk_reduce", _i32)]


class gemm_problem_t(ctypes.Structure):
    _fields_ = [("M", _i64), ("N", _i64), ("K", _i64), ("lda", _i64), ("ldb", _i64),
                ("ldc", _i64), ("A", _vp), ("B", _vp), ("C", _vp), ("alpha", _f32),
                ("beta", _f32), ("transA", _i32), ("transB", _i32)]


# name -> (restype, argtypes), mirroring include/gemm.h
_SIGS = {
    "gemm_create": (ctypes.c_int, [ctypes.POINTER(_vp)]),
    "gemm_destroy": (ctypes.c_int, [_vp]),
    "gemm_set_config": (ctypes.c_int, [_vp, ctypes.POINTER(gemm_config_t)]),
    "gemm_workspace_size": (_sz, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64, _i64, _i64]),
    "gemm_set_workspace": (ctypes.c_int, [_vp, _vp, _sz]),
    "gemm": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _i64, _i64, _i64, _f32, _vp, _i64,
                            _vp, _i64, _f32, _vp, _i64, ctypes.c_int, _vp]),
    "gemm_bf16": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _i64, _i64, _i64, _f32, _vp,
                                 _i64, _vp, _i64, _f32, _vp, _i64, _vp]),
    "gemm_split_bf16": (ctypes.c_int, [_vp, ctypes.c_int, _i64, _i64, _vp, _i64, _vp, _vp, _i64,
                                       _vp]),
    "gemm_from_host": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _i64, _i64, _i64, _f32,
                                      _vp, _i64, _vp, _i64, _f32, _vp, _i64, ctypes.c_int, _vp]),
    "gemm_grouped": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(gemm_problem_t), _i32, _vp]),
    "gemm_grouped_plan_create": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(gemm_problem_t),
                                                _i32, ctypes.c_uint32, _vp, ctypes.POINTER(_vp)]),
    "gemm_grouped_plan_run": (ctypes.c_int, [_vp, _vp]),
    "gemm_grouped_plan_config": (ctypes.c_int, [_vp, ctypes.POINTER(gemm_config_t),
                                                ctypes.POINTER(ctypes.c_double)]),
    "gemm_grouped_plan_destroy": (ctypes.c_int, [_vp]),
    "gemm_backward": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _i64, _i64, _i64, _vp, _i64,
                                     _vp, _i64, _vp, _i64, _vp, _i64, _vp, _i64, ctypes.c_int,
                                     _vp]),
    "gemm_syr2k": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _i64, _i64, _f32, _vp, _i64,
                                  _vp, _i64, _f32, _vp, _i64, ctypes.c_int, _vp]),
    "gemm_syr2k_workspace_size": (_sz, [_vp, ctypes.c_int, ctypes.c_int, _i64, _i64]),
    "gemm_profile_enable": (ctypes.c_int, [_vp, ctypes.c_int]),
    "gemm_profile_read": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int)]),
    "gemm_profile_read_each": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_int)]),
    "gemm_bf16x3_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _i64, _i64, _i64, _f32,
                                           _vp, _i64, _vp, _i64, _f32, _vp, _i64, _vp]),
    "gemm_bf16x3_noalloc_check": (ctypes.c_int, [_vp]),
    "gemm_sync": (ctypes.c_int, [_vp, _vp]),
    "gemm_last_error_arg": (ctypes.c_int, [_vp]),
    "gemm_get_last_error_arg": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "gemm_last_launch_count": (ctypes.c_int, [_vp]),
    "gemm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}

EXPORTED = tuple(_SIGS)

_LIB = None


class GemmError(RuntimeError):
    def __init__(self, status, func, arg=0):
        self.status = status
        self.arg = arg
        msg = "%s: %s" % (func, status_string(status) if _LIB else status)
        if status == GEMM_ERR_ARG:
            msg += " (argument %d)" % arg
        super().__init__(msg)


def library_path():
    return _build.LIB


def load():
    """Load the built library (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("CUDA library %s is not built; run "
                               "paper_2305_18236_gb300.build.build() (needs nvcc)" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def status_string(status):
    return load().gemm_status_string(int(status)).decode()


def check(status, func, handle=None):
    if status != GEMM_OK:
        arg = load().gemm_last_error_arg(handle) if handle else 0
        raise GemmError(status, func, arg)
    return status
