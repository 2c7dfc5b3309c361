"""ctypes view of libfcfs.so (include/fcfs.h).  No compute happens here."""
import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfcfs.so")

STATUS = {0: "FCFS_OK", 1: "FCFS_EINVAL", 2: "FCFS_EINVAL_DATA", 3: "FCFS_EWORKSPACE",
          4: "FCFS_ECUDA", 5: "FCFS_ETIMEOUT", 6: "FCFS_EUNSUPPORTED"}
PREC = {"fp32": 0, "split_f16": 1}
FLAG_VALIDATE = 1

_p = C.c_void_p
_i32, _i64, _u32, _u64, _sz = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_size_t

SIGNATURES = {
    "fcfs_version": (C.c_int, []),
    "fcfs_status_string": (C.c_char_p, [C.c_int]),
    "fcfs_launch_count": (_u64, []),
    "fcfs_workspace_size": (_sz, [_i64, _i32, _i32, _i32]),
    "fcfs_forward": (C.c_int, [_p, _p, _p, _i64, _i32, _i32, _i32, _u32, _p, _p, _p, _sz, _p]),
    "fcfs_adjoint_workspace_size": (_sz, [_i64, _i32, _i32, _i32]),
    "fcfs_adjoint": (C.c_int, [_p, _p, _p, _i64, _i32, _i32, _i32, _p, _p, _p, _p, _sz, _p]),
    "fcfs_edge_chain": (C.c_int, [_p, _p, _p, _p, _p, _i64, _p, _p]),
    "fcfs_batch_workspace_size": (_sz, [_i64, _i32, _i32, _i32, _i32]),
    "fcfs_batch": (C.c_int, [_p, _p, _p, _p, _i32, _i64, _i32, _i32, _i32, _u32, _p, _p, _p, _sz, _p]),
    "fcfs_cosine_workspace_size": (_sz, [_i64, _i32, _i32, _i32]),
    "fcfs_cosine": (C.c_int, [_p, _p, _p, _i64, _i32, _i32, _i32, _u32, _p, _p, _p, _sz, _p]),
    "fcfs_haar_workspace_size": (_sz, [_i64, _i32, _i32]),
    "fcfs_haar": (C.c_int, [_p, _p, _p, _i64, _i32, _i32, _u32, _p, _p, _sz, _p]),
    "fcfs_get_status": (C.c_int, [_p, _p]),
    "fcfs_forward_noalloc": (C.c_int, [_p, _p, _p, _i64, _i32, _i32, _i32, _u32, _p, _p, _p]),
    "fcfs_noalloc_status": (C.c_int, [_p]),
    "fcfs_plan_create": (C.c_int, [C.POINTER(_p), _i32, _i64, _i32, _i32, _i32, _i32]),
    "fcfs_plan_destroy": (None, [_p]),
    "fcfs_plan_set": (C.c_int, [_p, _i32, _i64]),
    "fcfs_plan_get": (_i64, [_p, _i32]),
    "fcfs_plan_workspace_size": (_sz, [_p]),
    "fcfs_plan_forward": (C.c_int, [_p, _p, _p, _p, _i64, _u32, _p, _p, _p, _sz, _p]),
    "fcfs_plan_batch": (C.c_int, [_p, _p, _p, _p, _p, _i64, _p, _p, _p, _sz, _p]),
    "fcfs_plan_adjoint": (C.c_int, [_p, _p, _p, _p, _i64, _p, _p, _p, _p, _sz, _p]),
    "fcfs_debug_set_splits": (None, [_i32]),
    "fcfs_debug_set_fuse": (None, [_i32]),
    "fcfs_debug_set_pair": (None, [_i32]),
    "fcfs_debug_set_barrier_extra": (None, [_i32]),
    "fcfs_debug_set_hybrid": (None, [_i32]),
    "fcfs_debug_set_overlap": (None, [_i32]),
    "fcfs_forward_grouped": (_i32, [_i64, _i32, _i32, _i32]),
    "fcfs_adjoint_grouped": (_i32, [_i64, _i32, _i32, _i32]),
    "fcfs_profile_enable": (None, [_i32]),
    "fcfs_set_batch_unit_chunks": (None, [_i32]),
    "fcfs_profile_read": (_i32, [C.POINTER(C.c_float), _i32]),
    "fcfs_kernel_timing_enable": (None, [_i32]),
    "fcfs_kernel_timing_count": (_i32, []),
    "fcfs_kernel_timing_name": (C.c_char_p, [_i32]),
    "fcfs_kernel_timing_ms": (C.c_float, [_i32]),
}

_lib = None


class FCFSError(RuntimeError):
    def __init__(self, fn, code):
        self.code = code
        self.name = STATUS.get(code, str(code))
        super().__init__("%s returned %s" % (fn, self.name))


def load():
    """The loaded library; raises if it was not built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libfcfs.so is not built (run paper_1010_5562_gb300.build.build()); "
                               "the FCFS transform has no CPU fallback")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(fn, code):
    if code != 0:
        raise FCFSError(fn, code)
