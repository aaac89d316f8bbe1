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

    def slot_bytes(self) -> np.ndarray:
        """fwi_ckpt_store_slot_bytes: bytes of each checkpoint slot of the last
        forward sweep, in slot order (full history: u^1, u^2, ...)."""
        L = _lib.load()
        n = C.c_int(0)
        check("fwi_ckpt_store_slot_bytes", L.fwi_ckpt_store_slot_bytes(self.handle, None, 0, C.byref(n)))
        out = np.zeros(max(1, n.value), dtype=np.uint64)
        check("fwi_ckpt_store_slot_bytes", L.fwi_ckpt_store_slot_bytes(
            self.handle, out.ctypes.data_as(C.POINTER(C.c_ulonglong)), n.value, C.byref(n)))
        return out[:n.value]

    def slot_zero_blocks(self) -> np.ndarray:
        """fwi_ckpt_store_slot_zero_blocks: blocks each compressed slot codes as
        zero (decoded exactly 0, skipped by the full-history reverse sweep)."""
        L = _lib.load()
        n = C.c_int(0)
        check("fwi_ckpt_store_slot_zero_blocks",
              L.fwi_ckpt_store_slot_zero_blocks(self.handle, None, 0, C.byref(n)))
        out = np.zeros(max(1, n.value), dtype=np.uint64)
        check("fwi_ckpt_store_slot_zero_blocks", L.fwi_ckpt_store_slot_zero_blocks(
            self.handle, out.ctypes.data_as(C.POINTER(C.c_ulonglong)), n.value, C.byref(n)))
        return out[:n.value]

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


# ---- batched shots ------------------------------------------------------------

@dataclass
class ShotSpec:
    """One shot of a survey on its aperture: the nx*ny*nz window at (x0, y0, z0)
    of the model grid (absorbing layer inside the window), record length nt
    steps, source cell `src` and receiver cells `rec` ((nrec, 3) int32, i j k)
    in model-grid coordinates."""
    x0: int
    y0: int
    z0: int
    nx: int
    ny: int
    nz: int
    nt: int
    src: tuple
    rec: np.ndarray

    @property
    def window(self):
        return (slice(self.z0, self.z0 + self.nz), slice(self.y0, self.y0 + self.ny),
                slice(self.x0, self.x0 + self.nx))

    def local_geometry(self, geom: Geometry) -> Geometry:
        return Geometry(nx=self.nx, ny=self.ny, nz=self.nz, h=geom.h, dt=geom.dt, nt=self.nt, nbl=geom.nbl,
                        vmax=geom.vmax, sponge_R=geom.sponge_R)


def _concat_host(parts) -> np.ndarray:
    return np.ascontiguousarray(np.concatenate([_host_f32(p).ravel() for p in parts]), dtype=np.float32)


class Batch:
    """fwi_batch plan: all shots of a survey advanced together (one persistent
    stencil launch per time step over the tiles of every active shot).
    `graph` captures a whole call as a CUDA graph replayed on later calls
    with the same tensors; `tune` times launch shapes on the first call.
    Records, observed data and residuals are flat float32 tensors with each
    shot's (nt, nrec) block at `offsets[s]` (see `split`)."""

    def __init__(self, geom: Geometry, shots: list, mode: int = FWI_CKPT_EVERY_K, k: int = 10,
                 atol: float = 0.0, arena_bytes: int = 1 << 30, graph: bool = False, tune: bool = False,
                 device=None):
        self.geom, self.shots = geom, list(shots)
        self.mode, self.k, self.atol = mode, k, atol
        n = len(self.shots)
        arr = (_lib.Shot * max(n, 1))()
        wf = of = rf = 0
        self.offsets, self.wavelet_offsets = [], []
        for i, s in enumerate(self.shots):
            nrec = int(len(s.rec))
            arr[i] = _lib.Shot(s.x0, s.y0, s.z0, s.nx, s.ny, s.nz, s.nt, int(s.src[0]), int(s.src[1]),
                               int(s.src[2]), rf, nrec, wf, of)
            self.offsets.append(of)
            self.wavelet_offsets.append(wf)
            wf += s.nt
            of += s.nt * nrec
            rf += nrec
        self.n_obs, self.n_wavelet = of, wf
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        recs = [np.asarray(s.rec, np.int32).reshape(-1, 3) for s in self.shots]
        rec = torch.from_numpy(np.ascontiguousarray(np.concatenate(recs) if rf else np.zeros((1, 3), np.int32)))
        self.rec = rec.to(dev)
        self.device = dev
        pol = _lib.Policy(mode, k, atol)
        self.graph = graph
        self._staged = {}
        flags = (_lib.FWI_BATCH_GRAPH if graph else 0) | (_lib.FWI_BATCH_TUNE if tune else 0)
        h = C.c_void_p()
        g = geom.cstruct()
        torch.cuda.synchronize(dev)
        check("fwi_batch_create", _lib.load().fwi_batch_create(C.byref(g), n, arr, self.rec.data_ptr(),
                                                                C.byref(pol), arena_bytes, flags, C.byref(h)))
        self._h = h

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("batch plan is closed")
        return self._h

    def split(self, flat: torch.Tensor) -> list:
        """Per-shot (nt, nrec) views of a flat records / data tensor."""
        return [flat[o:o + s.nt * len(s.rec)].view(s.nt, len(s.rec)) for o, s in zip(self.offsets, self.shots)]

    def concat(self, parts) -> torch.Tensor:
        """Flat device tensor from per-shot (nt, nrec) blocks."""
        return torch.cat([torch.as_tensor(p, dtype=torch.float32).reshape(-1) for p in parts]).to(self.device)

    def _wavelets(self, wavelets) -> np.ndarray:
        w = _concat_host(wavelets) if isinstance(wavelets, (list, tuple)) else _host_f32(wavelets).ravel()
        if w.size < self.n_wavelet:
            raise ValueError("wavelets shorter than the shots' record lengths")
        return np.ascontiguousarray(w)

    def _stage(self, name: str, src: torch.Tensor | None, shape) -> torch.Tensor:
        """Plan-owned tensor (same storage on every call, so that a captured
        graph is replayed), filled from src when given."""
        t = self._staged.get(name)
        if t is None:
            t = torch.empty(shape, dtype=torch.float32, device=self.device)
            self._staged[name] = t
        if src is not None:
            t.copy_(src.reshape(t.shape))
        return t

    def gradient(self, m: torch.Tensor, wavelets, d_obs: torch.Tensor, grad: torch.Tensor | None = None):
        """fwi_batch_gradient: (grad += sum_s dPhi_s/dm, misfits (nshots,) FP64)."""
        w = self._wavelets(wavelets)
        if grad is None:
            grad = torch.zeros(self.geom.shape, dtype=torch.float32, device=m.device)
        phi = (C.c_double * max(len(self.shots), 1))()
        g = grad
        if self.graph:  # graph replay needs the same device pointers on every call
            m = self._stage("m", m, self.geom.shape)
            d_obs = self._stage("obs", d_obs, (max(self.n_obs, 1),))
            g = self._stage("grad", None, self.geom.shape).zero_()
        st = _lib.load().fwi_batch_gradient(self.handle, _dev(m, torch.float32, "m"), w.ctypes.data,
                                            _dev(d_obs, torch.float32, "d_obs"), _dev(g, torch.float32, "grad"),
                                            phi, _stream())
        check("fwi_batch_gradient", st)
        if g is not grad:
            grad += g
        return grad, np.array(phi[: len(self.shots)])

    def forward(self, m: torch.Tensor, wavelets, out: torch.Tensor | None = None) -> torch.Tensor:
        """fwi_batch_forward: flat records of all shots; checkpoints kept in the plan."""
        w = self._wavelets(wavelets)
        if out is None:
            out = torch.empty(max(self.n_obs, 1), dtype=torch.float32, device=m.device)
        d = out
        if self.graph:
            m = self._stage("m", m, self.geom.shape)
            d = self._stage("d", None, (max(self.n_obs, 1),))
        st = _lib.load().fwi_batch_forward(self.handle, _dev(m, torch.float32, "m"), w.ctypes.data,
                                           _dev(d, torch.float32, "d"), _stream())
        check("fwi_batch_forward", st)
        if d is not out:
            out.copy_(d)
        return out[: self.n_obs]

    def adjoint(self, m: torch.Tensor, wavelets, resid: torch.Tensor, grad: torch.Tensor | None = None):
        """fwi_batch_adjoint: grad += sum_s J_s^T resid_s from the plan's checkpoints."""
        w = self._wavelets(wavelets)
        if grad is None:
            grad = torch.zeros(self.geom.shape, dtype=torch.float32, device=m.device)
        g = grad
        if self.graph:
            m = self._stage("m", m, self.geom.shape)
            resid = self._stage("resid", resid, (max(self.n_obs, 1),))
            g = self._stage("grad", None, self.geom.shape).zero_()
        st = _lib.load().fwi_batch_adjoint(self.handle, _dev(m, torch.float32, "m"), w.ctypes.data,
                                           _dev(resid, torch.float32, "resid"), _dev(g, torch.float32, "grad"),
                                           _stream())
        check("fwi_batch_adjoint", st)
        if g is not grad:
            grad += g
        return grad

    def stats(self) -> dict:
        s = _lib.BatchStats()
        check("fwi_batch_get_stats", _lib.load().fwi_batch_get_stats(self.handle, C.byref(s)))
        return {f: getattr(s, f) for f, _ in _lib.BatchStats._fields_}

    def close(self):
        if self._h:
            _lib.load().fwi_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gradient_per_shot(geom: Geometry, m: torch.Tensor, shots: list, wavelets, d_obs: list,
                      store: CheckpointStore, mode: int = FWI_CKPT_FULL, k: int = 1, atol: float = 0.0,
                      grad: torch.Tensor | None = None):
    """One fwi_gradient call per shot on its window of the model (the plain,
    one-shot-per-launch-sequence path): returns (grad += sum_s dPhi_s/dm,
    misfits).  The window copy of m and the stacking add are tensor copies."""
    if grad is None:
        grad = torch.zeros(geom.shape, dtype=torch.float32, device=m.device)
    phis = []
    for i, s in enumerate(shots):
        lg = s.local_geometry(geom)
        mw = m[s.window].contiguous()
        origin = torch.tensor([s.x0, s.y0, s.z0], dtype=torch.int32, device=m.device)
        rec = (torch.as_tensor(np.asarray(s.rec, np.int32), device=m.device) - origin).contiguous()
        src = (s.src[0] - s.x0, s.src[1] - s.y0, s.src[2] - s.z0)
        g, phi = gradient(lg, mw, wavelets[i], src, rec, d_obs[i], store, mode=mode, k=k, atol=atol)
        grad[s.window] += g
        phis.append(phi)
    return grad, np.array(phis)


def selftest_bounded_wait(polls: int = 1000) -> int:
    """fwi_selftest_bounded_wait: status of a kernel whose bounded wait is made
    to run out (FWI_ERR_TIMEOUT when the mechanism works)."""
    return _lib.load().fwi_selftest_bounded_wait(int(polls), _stream())


def selftest_damped_quotient(num: torch.Tensor, den: torch.Tensor) -> torch.Tensor:
    """fwi_selftest_damped_quotient: num / den as the stencil kernels divide by
    the damping factor 1 + eta (den in [1, 2^126))."""
    if num.shape != den.shape:
        raise ValueError("num and den must have one shape")
    out = torch.empty_like(num)
    check("fwi_selftest_damped_quotient", _lib.load().fwi_selftest_damped_quotient(
        _dev(num, torch.float32, "num"), _dev(den, torch.float32, "den"), _dev(out, torch.float32, "out"),
        num.numel(), _stream()))
    return out
