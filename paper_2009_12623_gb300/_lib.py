"""ctypes binding of libfwi.so (include/fwi.h).  Argument marshalling only.

The library is loaded from this package directory.  There is no fallback: if
``libfwi.so`` is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfwi.so")

FWI_OK, FWI_ERR_ARG, FWI_ERR_CAPACITY, FWI_ERR_CORRUPT = 0, -1, -2, -3
FWI_ERR_NONFINITE, FWI_ERR_CUDA, FWI_ERR_TIMEOUT, FWI_ERR_NOMEM = -4, -5, -6, -7
FWI_CKPT_FULL, FWI_CKPT_EVERY_K, FWI_CKPT_BINOMIAL, FWI_CKPT_SUBSAMPLE = 1, 2, 3, 4
FWI_ACT_ADVANCE, FWI_ACT_STORE, FWI_ACT_RESTORE, FWI_ACT_RECOMPUTE, FWI_ACT_ADJOINT, FWI_ACT_FREE = (
    1, 2, 3, 4, 5, 6)

#: every symbol include/fwi.h declares
EXPORTS = [
    "fwi_ckpt_schedule", "fwi_ckpt_store_create", "fwi_ckpt_store_destroy", "fwi_ckpt_store_stats",
    "fwi_ckpt_store_slot_bytes", "fwi_ckpt_store_slot_zero_blocks",
    "fwi_forward", "fwi_gradient", "fwi_gradient_host", "zfp_max_compressed_bytes",
    "zfp_compress_fixed_accuracy", "zfp_decompress", "fwi_misfit", "fwi_dot_f64",
    "fwi_status_string", "fwi_kernel_launch_count", "fwi_profile_enable", "fwi_profile_reset",
    "fwi_profile_read", "zfp_compress_fixed_accuracy_noalloc", "fwi_forward_store",
    "fwi_adjoint_store", "fwi_batch_create", "fwi_batch_destroy", "fwi_batch_gradient",
    "fwi_batch_forward", "fwi_batch_adjoint", "fwi_batch_get_stats", "fwi_selftest_bounded_wait",
    "fwi_selftest_damped_quotient",
]
KERNEL_CLASSES = ["stencil_forward", "stencil_adjoint", "zfp_encode", "zfp_decode", "other"]


class FwiError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        super().__init__(f"{fn} failed: {status} ({status_string(status)})")


class Geometry(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("h", C.c_double),
                ("dt", C.c_double), ("nt", C.c_int), ("nbl", C.c_int),
                ("sponge_R", C.c_double), ("vmax", C.c_double)]


class Policy(C.Structure):
    _fields_ = [("mode", C.c_int), ("k_or_snaps", C.c_int), ("atol", C.c_double)]


class Action(C.Structure):
    _fields_ = [("kind", C.c_int), ("step", C.c_int), ("arg", C.c_int)]


class StoreStats(C.Structure):
    _fields_ = [("capacity_bytes", C.c_size_t), ("used_bytes", C.c_size_t),
                ("raw_bytes", C.c_size_t), ("n_checkpoints", C.c_int), ("overflowed", C.c_int)]


class Shot(C.Structure):
    _fields_ = [("x0", C.c_int), ("y0", C.c_int), ("z0", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
                ("nz", C.c_int), ("nt", C.c_int), ("src_i", C.c_int), ("src_j", C.c_int),
                ("src_k", C.c_int), ("rec_first", C.c_int), ("nrec", C.c_int),
                ("wavelet_first", C.c_longlong), ("obs_first", C.c_longlong)]


class BatchStats(C.Structure):
    _fields_ = [("nshots", C.c_int), ("max_nt", C.c_int), ("zc", C.c_int), ("ctas", C.c_int),
                ("zc_adjoint", C.c_int), ("ctas_adjoint", C.c_int), ("tuned", C.c_int),
                ("graph_nodes", C.c_int), ("launches_per_call", C.c_uint64), ("arena_bytes", C.c_size_t),
                ("used_bytes", C.c_size_t), ("raw_bytes", C.c_size_t), ("device_bytes", C.c_size_t)]


FWI_BATCH_GRAPH = 1
FWI_BATCH_TUNE = 2

_lock = threading.Lock()
_lib = None


def load() -> C.CDLL:
    """Load libfwi.so (raises if it is absent: there is no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfwi.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, fp, ip, dp = C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)
        gp, pp = C.POINTER(Geometry), C.POINTER(Policy)
        L.fwi_ckpt_schedule.argtypes = [C.c_int, pp, C.POINTER(Action), C.c_size_t, C.POINTER(C.c_size_t)]
        L.fwi_ckpt_store_create.argtypes = [C.c_size_t, C.POINTER(C.c_void_p)]
        L.fwi_ckpt_store_destroy.argtypes = [vp]
        L.fwi_ckpt_store_stats.argtypes = [vp, C.POINTER(StoreStats)]
        L.fwi_ckpt_store_slot_bytes.argtypes = [vp, C.POINTER(C.c_ulonglong), C.c_int, C.POINTER(C.c_int)]
        L.fwi_ckpt_store_slot_zero_blocks.argtypes = L.fwi_ckpt_store_slot_bytes.argtypes
        L.fwi_forward.argtypes = [gp, fp, vp, C.c_int, C.c_int, C.c_int, ip, C.c_int, fp,
                                  fp, fp, fp, fp, vp]
        L.fwi_gradient.argtypes = [gp, fp, vp, C.c_int, C.c_int, C.c_int, ip, C.c_int, fp, fp, dp,
                                   vp, pp, vp]
        L.fwi_gradient_host.argtypes = L.fwi_gradient.argtypes
        L.fwi_forward_store.argtypes = [gp, fp, vp, C.c_int, C.c_int, C.c_int, ip, C.c_int, fp, vp, pp, vp]
        L.fwi_adjoint_store.argtypes = [gp, fp, vp, C.c_int, C.c_int, C.c_int, ip, C.c_int, fp, fp, vp, pp,
                                        vp]
        L.zfp_max_compressed_bytes.argtypes = [C.c_int, C.c_int, C.c_int]
        L.zfp_max_compressed_bytes.restype = C.c_size_t
        L.zfp_compress_fixed_accuracy.argtypes = [fp, C.c_int, C.c_int, C.c_int, C.c_double, vp,
                                                  C.c_size_t, C.POINTER(C.c_size_t), vp]
        L.zfp_compress_fixed_accuracy_noalloc.argtypes = L.zfp_compress_fixed_accuracy.argtypes
        L.zfp_decompress.argtypes = [vp, C.c_size_t, fp, C.c_int, C.c_int, C.c_int, vp]
        L.fwi_misfit.argtypes = [fp, fp, C.c_size_t, fp, dp, vp]
        L.fwi_dot_f64.argtypes = [fp, fp, C.c_size_t, dp, vp]
        L.fwi_status_string.argtypes = [C.c_int]
        L.fwi_status_string.restype = C.c_char_p
        L.fwi_kernel_launch_count.argtypes = []
        L.fwi_kernel_launch_count.restype = C.c_uint64
        L.fwi_profile_enable.argtypes = [C.c_int]
        L.fwi_profile_reset.argtypes = []
        L.fwi_profile_read.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_uint64), C.c_int]
        L.fwi_batch_create.argtypes = [gp, C.c_int, C.POINTER(Shot), ip, pp, C.c_size_t, C.c_int,
                                       C.POINTER(C.c_void_p)]
        L.fwi_batch_destroy.argtypes = [vp]
        L.fwi_batch_gradient.argtypes = [vp, fp, vp, fp, fp, dp, vp]
        L.fwi_batch_forward.argtypes = [vp, fp, vp, fp, vp]
        L.fwi_batch_adjoint.argtypes = [vp, fp, vp, fp, fp, vp]
        L.fwi_batch_get_stats.argtypes = [vp, C.POINTER(BatchStats)]
        L.fwi_selftest_bounded_wait.argtypes = [C.c_longlong, vp]
        L.fwi_selftest_damped_quotient.argtypes = [vp, vp, vp, C.c_longlong, vp]
        _lib = L
        return L


def status_string(status: int) -> str:
    return load().fwi_status_string(status).decode()


def check(fn: str, status: int) -> None:
    if status != FWI_OK:
        raise FwiError(fn, status)
