"""Python binding of the libfwi C ABI (include/fwi.h), one wrapper per entry point.

Marshalling only: tensors are checked for device, dtype and contiguity, and
their pointers and the current CUDA stream are handed to the library.  Every
arithmetic step runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import (FWI_CKPT_BINOMIAL, FWI_CKPT_EVERY_K, FWI_CKPT_FULL, FWI_CKPT_SUBSAMPLE,  # noqa: F401
                   FwiError, check)


@dataclass
class Geometry:
    """Grid [nz][ny][nx] with spacing h (m), nt steps of dt (s), an nbl-cell
    absorbing layer (reflection target sponge_R, reference velocity vmax)."""
    nx: int
    ny: int
    nz: int
    h: float
    dt: float
    nt: int
    nbl: int
    vmax: float
    sponge_R: float = 1e-3

    def cstruct(self) -> _lib.Geometry:
        return _lib.Geometry(self.nx, self.ny, self.nz, self.h, self.dt, self.nt, self.nbl,
                             self.sponge_R, self.vmax)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _dev(t: torch.Tensor, dtype, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA {dtype} tensor")
    return t.data_ptr()


def _opt(t, dtype, name):
    return None if t is None else _dev(t, dtype, name)


def _host_f32(a) -> np.ndarray:
    if isinstance(a, torch.Tensor):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=np.float32)


def kernel_launch_count() -> int:
    return int(_lib.load().fwi_kernel_launch_count())


def profile_enable(on: bool = True) -> None:
    check("fwi_profile_enable", _lib.load().fwi_profile_enable(1 if on else 0))


def profile_reset() -> None:
    check("fwi_profile_reset", _lib.load().fwi_profile_reset())


def profile_read() -> dict:
    """{kernel class: (device ms, launches)} since the last reset."""
    n = len(_lib.KERNEL_CLASSES)
    ms = (C.c_double * n)()
    cnt = (C.c_uint64 * n)()
    check("fwi_profile_read", _lib.load().fwi_profile_read(ms, cnt, n))
    return {k: (ms[i], int(cnt[i])) for i, k in enumerate(_lib.KERNEL_CLASSES)}


def ckpt_schedule(nt: int, mode: int, k: int = 1, atol: float = 0.0):
    L = _lib.load()
    pol = _lib.Policy(mode, k, atol)
    n = C.c_size_t(0)
    st = L.fwi_ckpt_schedule(nt, C.byref(pol), None, 0, C.byref(n))
    if st not in (0, _lib.FWI_ERR_CAPACITY):
        check("fwi_ckpt_schedule", st)
    acts = (_lib.Action * max(n.value, 1))()
    check("fwi_ckpt_schedule", L.fwi_ckpt_schedule(nt, C.byref(pol), acts, n.value, C.byref(n)))
    return [(a.kind, a.step, a.arg) for a in acts[: n.value]]


class CheckpointStore:
    """Device arena for compressed checkpoints (fwi_ckpt_store_*)."""

    def __init__(self, capacity_bytes: int):
        self._h = C.c_void_p()
        check("fwi_ckpt_store_create",
              _lib.load().fwi_ckpt_store_create(int(capacity_bytes), C.byref(self._h)))
        self.capacity = int(capacity_bytes)

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("store is closed")
        return self._h

    def stats(self) -> dict:
        s = _lib.StoreStats()
        check("fwi_ckpt_store_stats", _lib.load().fwi_ckpt_store_stats(self.handle, C.byref(s)))
        return {"capacity_bytes": s.capacity_bytes, "used_bytes": s.used_bytes,
                "raw_bytes": s.raw_bytes, "n_checkpoints": s.n_checkpoints,
                "overflowed": bool(s.overflowed)}

    def close(self):
        if self._h:
            _lib.load().fwi_ckpt_store_destroy(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def forward(geom: Geometry, m: torch.Tensor, wavelet, src, rec: torch.Tensor,
            u_prev_init: torch.Tensor | None = None, u_cur_init: torch.Tensor | None = None,
            return_state: bool = False):
    """fwi_forward: records d[n, r] = u^{n+1} at receiver r (FP32, device)."""
    w = _host_f32(wavelet)
    nrec = rec.shape[0]
    d = torch.empty((geom.nt, nrec), dtype=torch.float32, device=m.device)
    up = torch.empty(geom.shape, dtype=torch.float32, device=m.device) if return_state else None
    ul = torch.empty(geom.shape, dtype=torch.float32, device=m.device) if return_state else None
    g = geom.cstruct()
    st = _lib.load().fwi_forward(
        C.byref(g), _dev(m, torch.float32, "m"), w.ctypes.data, int(src[0]), int(src[1]), int(src[2]),
        _dev(rec, torch.int32, "rec"), nrec, _dev(d, torch.float32, "d"),
        _opt(u_prev_init, torch.float32, "u_prev_init"), _opt(u_cur_init, torch.float32, "u_cur_init"),
        _opt(up, torch.float32, "u_prev_out"), _opt(ul, torch.float32, "u_last_out"), _stream())
    check("fwi_forward", st)
    return (d, up, ul) if return_state else d


def gradient(geom: Geometry, m: torch.Tensor, wavelet, src, rec: torch.Tensor,
             d_obs: torch.Tensor, store: CheckpointStore, mode: int = FWI_CKPT_FULL, k: int = 1,
             atol: float = 0.0, grad: torch.Tensor | None = None):
    """fwi_gradient: returns (grad += dPhi/dm, Phi)."""
    w = _host_f32(wavelet)
    if grad is None:
        grad = torch.zeros(geom.shape, dtype=torch.float32, device=m.device)
    pol = _lib.Policy(mode, k, atol)
    phi = C.c_double(0.0)
    g = geom.cstruct()
    st = _lib.load().fwi_gradient(
        C.byref(g), _dev(m, torch.float32, "m"), w.ctypes.data, int(src[0]), int(src[1]), int(src[2]),
        _dev(rec, torch.int32, "rec"), rec.shape[0], _dev(d_obs, torch.float32, "d_obs"),
        _dev(grad, torch.float32, "grad"), C.byref(phi), store.handle, C.byref(pol), _stream())
    check("fwi_gradient", st)
    return grad, phi.value


def forward_store(geom: Geometry, m: torch.Tensor, wavelet, src, rec: torch.Tensor,
                  store: CheckpointStore, mode: int = FWI_CKPT_FULL, k: int = 1, atol: float = 0.0):
    """fwi_forward_store: records (nt, nrec), checkpoints kept in `store`."""
    w = _host_f32(wavelet)
    nrec = rec.shape[0]
    d = torch.empty((geom.nt, nrec), dtype=torch.float32, device=m.device)
    pol = _lib.Policy(mode, k, atol)
    g = geom.cstruct()
    st = _lib.load().fwi_forward_store(
        C.byref(g), _dev(m, torch.float32, "m"), w.ctypes.data, int(src[0]), int(src[1]), int(src[2]),
        _dev(rec, torch.int32, "rec"), nrec, _dev(d, torch.float32, "d"), store.handle, C.byref(pol),
        _stream())
    check("fwi_forward_store", st)
    return d


def adjoint_store(geom: Geometry, m: torch.Tensor, wavelet, src, rec: torch.Tensor,
                  resid: torch.Tensor, store: CheckpointStore, mode: int = FWI_CKPT_FULL, k: int = 1,
                  atol: float = 0.0, grad: torch.Tensor | None = None):
    """fwi_adjoint_store: grad += J^T resid from the checkpoints in `store`."""
    w = _host_f32(wavelet)
    if grad is None:
        grad = torch.zeros(geom.shape, dtype=torch.float32, device=m.device)
    pol = _lib.Policy(mode, k, atol)
    g = geom.cstruct()
    st = _lib.load().fwi_adjoint_store(
        C.byref(g), _dev(m, torch.float32, "m"), w.ctypes.data, int(src[0]), int(src[1]), int(src[2]),
        _dev(rec, torch.int32, "rec"), rec.shape[0], _dev(resid, torch.float32, "resid"),
        _dev(grad, torch.float32, "grad"), store.handle, C.byref(pol), _stream())
    check("fwi_adjoint_store", st)
    return grad


def gradient_host(geom: Geometry, m: np.ndarray, wavelet, src, rec: np.ndarray, d_obs: np.ndarray,
                  store: CheckpointStore, mode: int = FWI_CKPT_FULL, k: int = 1, atol: float = 0.0,
                  grad: np.ndarray | torch.Tensor | None = None):
    """fwi_gradient_host: host arrays in, host gradient out (copies inside the call).
    Arrays may be numpy or (pinned) CPU torch tensors."""
    def hp(a, dtype):
        if isinstance(a, torch.Tensor):
            assert a.device.type == "cpu" and a.is_contiguous() and a.dtype == dtype
            return a.data_ptr(), a
        arr = np.ascontiguousarray(a, dtype={torch.float32: np.float32, torch.int32: np.int32}[dtype])
        return arr.ctypes.data, arr
    w = _host_f32(wavelet)
    if grad is None:
        grad = np.zeros((geom.nz, geom.ny, geom.nx), dtype=np.float32)
    pm, _m = hp(m, torch.float32)
    pr, _r = hp(rec, torch.int32)
    po, _o = hp(d_obs, torch.float32)
    pg, _g = hp(grad, torch.float32)
    pol = _lib.Policy(mode, k, atol)
    phi = C.c_double(0.0)
    g = geom.cstruct()
    nrec = int(np.prod(_r.shape)) // 3
    st = _lib.load().fwi_gradient_host(C.byref(g), pm, w.ctypes.data, int(src[0]), int(src[1]),
                                       int(src[2]), pr, nrec, po, pg, C.byref(phi), store.handle,
                                       C.byref(pol), _stream())
    check("fwi_gradient_host", st)
    return _g, phi.value


def zfp_max_compressed_bytes(nx: int, ny: int, nz: int) -> int:
    return int(_lib.load().zfp_max_compressed_bytes(nx, ny, nz))


def zfp_compress(field: torch.Tensor, atol: float, out: torch.Tensor | None = None):
    """zfp_compress_fixed_accuracy: returns the stream as a CUDA uint8 tensor."""
    nz, ny, nx = field.shape
    cap = zfp_max_compressed_bytes(nx, ny, nz)
    if out is None:
        out = torch.empty(cap, dtype=torch.uint8, device=field.device)
    n = C.c_size_t(0)
    st = _lib.load().zfp_compress_fixed_accuracy(_dev(field, torch.float32, "field"), nx, ny, nz,
                                                 float(atol), _dev(out, torch.uint8, "out"),
                                                 out.numel(), C.byref(n), _stream())
    check("zfp_compress_fixed_accuracy", st)
    return out[: n.value]


def zfp_compress_status(field: torch.Tensor, atol: float, capacity: int):
    """Raw status variant (for error-path tests): (status, nbytes, out)."""
    nz, ny, nx = field.shape
    out = torch.zeros(max(capacity, 1), dtype=torch.uint8, device=field.device)
    n = C.c_size_t(0)
    st = _lib.load().zfp_compress_fixed_accuracy(field.data_ptr(), nx, ny, nz, float(atol),
                                                 out.data_ptr(), capacity, C.byref(n), _stream())
    return st, n.value, out


def zfp_decompress(stream: torch.Tensor, shape, out: torch.Tensor | None = None):
    nz, ny, nx = shape
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=stream.device)
    st = _lib.load().zfp_decompress(_dev(stream, torch.uint8, "stream"), stream.numel(),
                                    _dev(out, torch.float32, "out"), nx, ny, nz, _stream())
    check("zfp_decompress", st)
    return out


def zfp_decompress_status(stream: torch.Tensor, nbytes: int, shape):
    nz, ny, nx = shape
    out = torch.zeros(shape, dtype=torch.float32, device=stream.device)
    st = _lib.load().zfp_decompress(stream.data_ptr(), nbytes, out.data_ptr(), nx, ny, nz, _stream())
    return st, out


def misfit(d_sim: torch.Tensor, d_obs: torch.Tensor):
    """fwi_misfit: (residual, 1/2 sum residual^2 in FP64)."""
    r = torch.empty_like(d_sim)
    phi = C.c_double(0.0)
    check("fwi_misfit", _lib.load().fwi_misfit(_dev(d_sim, torch.float32, "d_sim"),
                                               _dev(d_obs, torch.float32, "d_obs"), d_sim.numel(),
                                               _dev(r, torch.float32, "resid"), C.byref(phi),
                                               _stream()))
    return r, phi.value


def dot_f64(a: torch.Tensor, b: torch.Tensor) -> float:
    out = C.c_double(0.0)
    check("fwi_dot_f64", _lib.load().fwi_dot_f64(_dev(a, torch.float32, "a"), _dev(b, torch.float32, "b"),
                                                 a.numel(), C.byref(out), _stream()))
    return out.value
