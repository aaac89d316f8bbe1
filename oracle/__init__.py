"""Oracle for the checkpointed FWI gradient with lossy checkpoint compression.

TEST INFRASTRUCTURE ONLY: a plain, slow FP64 CPU restatement of what the GPU
library computes (Kukreja et al., "Lossy Checkpoint Compression in Full
Waveform Inversion", Sec. 2 Eq. (1)-(4), Sec. 1.3-1.4).  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm
may import this package.  It shares no code with ``paper_2009_12623_gb300``;
the C sources here are compiled into ``liboracle.so`` by :func:`build`.

Parity status per function is given in ``oracle/oracle.h``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# ORACLE_LIBRARY names a separately built copy of the oracle (the planted-
# mistake tests build mutated copies and run the pins against them).
_LIB_PATH = os.environ.get("ORACLE_LIBRARY") or os.path.join(_HERE, "liboracle.so")
_SOURCES = ["fwi_oracle.c", "zfp_oracle.c"]
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_CAPACITY, ERR_CORRUPT, ERR_NONFINITE = 0, -1, -2, -3, -4
CKPT_FULL, CKPT_EVERY_K, CKPT_BINOMIAL, CKPT_SUBSAMPLE = 1, 2, 3, 4
ACT_ADVANCE, ACT_STORE, ACT_RESTORE, ACT_RECOMPUTE, ACT_ADJOINT, ACT_FREE = 1, 2, 3, 4, 5, 6


def build(force: bool = False) -> str:
    """Compile the oracle's C sources into ``oracle/liboracle.so`` (gcc, OpenMP)."""
    if os.environ.get("ORACLE_LIBRARY"):
        return _LIB_PATH  # built elsewhere, used as it is
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    hdr = os.path.join(_HERE, "oracle.h")
    if not force and os.path.exists(_LIB_PATH):
        t = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= t for s in srcs + [hdr]):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
           "-Wno-unknown-pragmas", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Geometry(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("h", C.c_double),
                ("dt", C.c_double), ("nt", C.c_int), ("nbl", C.c_int),
                ("sponge_R", C.c_double), ("vmax", C.c_double)]


class Policy(C.Structure):
    _fields_ = [("mode", C.c_int), ("k", C.c_int), ("atol", C.c_double)]


class Action(C.Structure):
    _fields_ = [("kind", C.c_int), ("step", C.c_int), ("arg", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            dp, fp, ip, u8p = (C.POINTER(C.c_double), C.POINTER(C.c_float),
                               C.POINTER(C.c_int), C.POINTER(C.c_uint8))
            gp = C.POINTER(Geometry)
            L.oracle_sponge_profile.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, dp]
            L.oracle_laplacian.argtypes = [gp, dp, dp]
            L.oracle_forward.argtypes = [gp, dp, dp, dp, C.c_int, C.c_int, C.c_int, ip, C.c_int, dp,
                                         dp, dp, dp, dp]
            L.oracle_adjoint_trace.argtypes = [gp, dp, dp, dp, ip, C.c_int, C.c_int, C.c_int,
                                               C.c_int, dp]
            L.oracle_gradient.argtypes = [gp, dp, dp, dp, C.c_int, C.c_int, C.c_int, ip, C.c_int,
                                          dp, C.POINTER(Policy), dp, dp, dp, dp]
            L.oracle_ckpt_schedule.argtypes = [C.c_int, C.POINTER(Policy), C.POINTER(Action),
                                               C.c_size_t, C.POINTER(C.c_size_t)]
            L.oracle_zfp_max_bytes.argtypes = [C.c_int, C.c_int, C.c_int]
            L.oracle_zfp_max_bytes.restype = C.c_size_t
            L.oracle_zfp_compress.argtypes = [fp, C.c_int, C.c_int, C.c_int, C.c_double, u8p,
                                              C.c_size_t, C.POINTER(C.c_size_t)]
            L.oracle_zfp_decompress.argtypes = [u8p, C.c_size_t, fp, C.c_int, C.c_int, C.c_int]
            L.oracle_zfp_minexp.argtypes = [C.c_double]
            L.oracle_zfp_encode_block.argtypes = [fp, C.c_int, C.POINTER(C.c_uint64), C.c_int]
            L.oracle_zfp_decode_block.argtypes = [C.POINTER(C.c_uint64), C.c_int, C.c_int, fp]
            L.oracle_zfp_fwd_xform.argtypes = [C.POINTER(C.c_int32)]
            L.oracle_zfp_inv_xform.argtypes = [C.POINTER(C.c_int32)]
            L.oracle_zfp_fwd_lift4.argtypes = [C.POINTER(C.c_int32), C.c_int]
            L.oracle_zfp_inv_lift4.argtypes = [C.POINTER(C.c_int32), C.c_int]
            L.oracle_zfp_perm.argtypes = [ip]
            L.oracle_zfp_block_quantise.argtypes = [fp, C.c_int, C.POINTER(C.c_int32), ip, ip]
            L.oracle_num_threads.restype = C.c_int
            L.oracle_binomial_cost.argtypes = [C.c_int, C.c_int]
            L.oracle_gradient_batch.argtypes = [gp, dp, C.c_int, C.POINTER(Shot), dp, ip, dp,
                                                C.POINTER(Policy), dp, dp]
            L.oracle_binomial_cost.restype = C.c_longlong
            _lib = L
    return _lib


def _p(a, ct):
    return None if a is None else a.ctypes.data_as(C.POINTER(ct))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def geometry(nx, ny, nz, h, dt, nt, nbl, sponge_R=1e-3, vmax=None) -> Geometry:
    return Geometry(nx, ny, nz, h, dt, nt, nbl, sponge_R, vmax if vmax is not None else 0.0)


def _geom(g) -> Geometry:
    if isinstance(g, Geometry):
        return g
    return Geometry(g.nx, g.ny, g.nz, g.h, g.dt, g.nt, g.nbl, g.sponge_R, g.vmax)


def num_threads() -> int:
    return lib().oracle_num_threads()


def sponge_profile(n, nbl, h, vmax, R=1e-3):
    out = np.zeros(n)
    lib().oracle_sponge_profile(n, nbl, h, vmax, R, _p(out, C.c_double))
    return out


def laplacian(g, u):
    g = _geom(g)
    u = _f64(u)
    out = np.zeros_like(u)
    lib().oracle_laplacian(C.byref(g), _p(u, C.c_double), _p(out, C.c_double))
    return out


def forward(g, m, wavelet, src, rec, m0=None, u_prev_init=None, u_cur_init=None,
            return_state=False):
    """Records d[n, r] = u^{n+1}[rec_r], n = 0..nt-1 (FP64)."""
    g = _geom(g)
    m, m0, w = _f64(m), _f64(m0), _f64(wavelet)
    rec = np.ascontiguousarray(rec, dtype=np.int32).reshape(-1, 3)
    out = np.zeros((g.nt, len(rec)))
    ub = np.zeros_like(m) if return_state else None
    ul = np.zeros_like(m) if return_state else None
    st = lib().oracle_forward(C.byref(g), _p(m, C.c_double), _p(m0, C.c_double), _p(w, C.c_double),
                              int(src[0]), int(src[1]), int(src[2]), _p(rec, C.c_int), len(rec),
                              _p(out, C.c_double), _p(_f64(u_prev_init), C.c_double),
                              _p(_f64(u_cur_init), C.c_double), _p(ub, C.c_double),
                              _p(ul, C.c_double))
    if st:
        raise RuntimeError(f"oracle_forward failed: {st}")
    return (out, ub, ul) if return_state else out


def adjoint_trace(g, m, resid, rec, src, m0=None):
    g = _geom(g)
    m, m0, r = _f64(m), _f64(m0), _f64(resid)
    rec = np.ascontiguousarray(rec, dtype=np.int32).reshape(-1, 3)
    out = np.zeros(g.nt)
    st = lib().oracle_adjoint_trace(C.byref(g), _p(m, C.c_double), _p(m0, C.c_double),
                                    _p(r, C.c_double), _p(rec, C.c_int), len(rec), int(src[0]),
                                    int(src[1]), int(src[2]), _p(out, C.c_double))
    if st:
        raise RuntimeError(f"oracle_adjoint_trace failed: {st}")
    return out


def gradient(g, m, wavelet, src, rec, d_obs, mode=CKPT_FULL, k=1, atol=0.0, m0=None):
    """Returns (grad, misfit, d_sim, checkpoint_bytes), all FP64."""
    g = _geom(g)
    m, m0, w, dobs = _f64(m), _f64(m0), _f64(wavelet), _f64(d_obs)
    rec = np.ascontiguousarray(rec, dtype=np.int32).reshape(-1, 3)
    grad = np.zeros_like(m)
    phi = C.c_double(0.0)
    dsim = np.zeros((g.nt, len(rec)))
    nbytes = C.c_double(0.0)
    pol = Policy(mode, k, atol)
    st = lib().oracle_gradient(C.byref(g), _p(m, C.c_double), _p(m0, C.c_double), _p(w, C.c_double),
                               int(src[0]), int(src[1]), int(src[2]), _p(rec, C.c_int), len(rec),
                               _p(dobs, C.c_double), C.byref(pol), _p(grad, C.c_double),
                               C.byref(phi), _p(dsim, C.c_double), C.byref(nbytes))
    if st:
        raise RuntimeError(f"oracle_gradient failed: {st}")
    return grad, phi.value, dsim, nbytes.value


class Shot(C.Structure):
    _fields_ = [("x0", C.c_int), ("y0", C.c_int), ("z0", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
                ("nz", C.c_int), ("nt", C.c_int), ("src_i", C.c_int), ("src_j", C.c_int),
                ("src_k", C.c_int), ("rec_first", C.c_int), ("nrec", C.c_int),
                ("wavelet_first", C.c_longlong), ("obs_first", C.c_longlong)]


def gradient_batch(g, m, shots, wavelets, recs, d_obs, mode=CKPT_FULL, k=1, atol=0.0):
    """Stacked gradient of a survey.  shots: sequence of (x0, y0, z0, nx, ny,
    nz, nt, (si, sj, sk)) in model-grid cells; wavelets[s]: (nt,) samples;
    recs[s]: (nrec, 3) receiver cells (model grid); d_obs[s]: (nt, nrec).
    Returns (grad on the model grid, misfit per shot), FP64."""
    g = _geom(g)
    m = _f64(m)
    arr = (Shot * max(len(shots), 1))()
    wf = of = rf = 0
    for i, (x0, y0, z0, nx, ny, nz, nt, src) in enumerate(shots):
        nrec = len(recs[i])
        arr[i] = Shot(x0, y0, z0, nx, ny, nz, nt, int(src[0]), int(src[1]), int(src[2]), rf, nrec, wf, of)
        wf += nt
        of += nt * nrec
        rf += nrec
    w = _f64(np.concatenate([np.asarray(x, np.float64).ravel() for x in wavelets]) if shots else np.zeros(1))
    rr = np.ascontiguousarray(np.concatenate([np.asarray(r, np.int32).reshape(-1, 3) for r in recs])
                              if rf else np.zeros((1, 3)), dtype=np.int32)
    dob = _f64(np.concatenate([np.asarray(d, np.float64).ravel() for d in d_obs]) if of else np.zeros(1))
    grad = np.zeros_like(m)
    phi = np.zeros(max(len(shots), 1))
    pol = Policy(mode, k, atol)
    st = lib().oracle_gradient_batch(C.byref(g), _p(m, C.c_double), len(shots), arr, _p(w, C.c_double),
                                     _p(rr, C.c_int), _p(dob, C.c_double), C.byref(pol),
                                     _p(grad, C.c_double), _p(phi, C.c_double))
    if st:
        raise RuntimeError(f"oracle_gradient_batch failed: {st}")
    return grad, phi[: len(shots)]


def binomial_cost(n, s):
    return int(lib().oracle_binomial_cost(n, s))


def ckpt_schedule(nt, mode, k=1, atol=0.0):
    pol = Policy(mode, k, atol)
    n = C.c_size_t(0)
    lib().oracle_ckpt_schedule(nt, C.byref(pol), None, 0, C.byref(n))
    acts = (Action * max(n.value, 1))()
    st = lib().oracle_ckpt_schedule(nt, C.byref(pol), acts, n.value, C.byref(n))
    if st:
        raise RuntimeError(f"oracle_ckpt_schedule failed: {st}")
    return [(a.kind, a.step, a.arg) for a in acts[: n.value]]


# ---- codec ----------------------------------------------------------------

def zfp_max_bytes(nx, ny, nz) -> int:
    return int(lib().oracle_zfp_max_bytes(nx, ny, nz))


def zfp_compress(field, atol) -> bytes:
    f = np.ascontiguousarray(field, dtype=np.float32)
    nz, ny, nx = f.shape
    cap = zfp_max_bytes(nx, ny, nz)
    out = np.zeros(cap, dtype=np.uint8)
    used = C.c_size_t(0)
    st = lib().oracle_zfp_compress(_p(f, C.c_float), nx, ny, nz, float(atol), _p(out, C.c_uint8),
                                   cap, C.byref(used))
    if st:
        raise ValueError(f"oracle_zfp_compress failed: {st}")
    return out[: used.value].tobytes()


def zfp_decompress_status(stream: bytes, shape):
    nz, ny, nx = shape
    buf = np.frombuffer(stream, dtype=np.uint8).copy()
    out = np.zeros(shape, dtype=np.float32)
    st = lib().oracle_zfp_decompress(_p(buf, C.c_uint8), len(buf), _p(out, C.c_float), nx, ny, nz)
    return st, out


def zfp_decompress(stream: bytes, shape):
    st, out = zfp_decompress_status(stream, shape)
    if st:
        raise ValueError(f"oracle_zfp_decompress failed: {st}")
    return out


def zfp_minexp(atol) -> int:
    return lib().oracle_zfp_minexp(float(atol))


def zfp_encode_block(v, minexp):
    v = np.ascontiguousarray(v, dtype=np.float32).reshape(64)
    words = np.zeros(40, dtype=np.uint64)
    n = lib().oracle_zfp_encode_block(_p(v, C.c_float), int(minexp), _p(words, C.c_uint64), 40)
    if n < 0:
        raise ValueError(f"encode failed: {n}")
    return words, n


def zfp_decode_block(words, nbits, minexp):
    w = np.ascontiguousarray(words, dtype=np.uint64)
    out = np.zeros(64, dtype=np.float32)
    n = lib().oracle_zfp_decode_block(_p(w, C.c_uint64), int(nbits), int(minexp), _p(out, C.c_float))
    if n < 0:
        raise ValueError(f"decode failed: {n}")
    return out, n


def zfp_fwd_xform(q):
    a = np.ascontiguousarray(q, dtype=np.int32).reshape(64).copy()
    lib().oracle_zfp_fwd_xform(_p(a, C.c_int32))
    return a


def zfp_inv_xform(q):
    a = np.ascontiguousarray(q, dtype=np.int32).reshape(64).copy()
    lib().oracle_zfp_inv_xform(_p(a, C.c_int32))
    return a


def zfp_lift4(x, inverse=False):
    a = np.ascontiguousarray(x, dtype=np.int32).reshape(4).copy()
    (lib().oracle_zfp_inv_lift4 if inverse else lib().oracle_zfp_fwd_lift4)(_p(a, C.c_int32), 1)
    return a


def zfp_perm():
    p = np.zeros(64, dtype=np.int32)
    lib().oracle_zfp_perm(_p(p, C.c_int))
    return p


def zfp_block_quantise(v, minexp):
    v = np.ascontiguousarray(v, dtype=np.float32).reshape(64)
    q = np.zeros(64, dtype=np.int32)
    emax, planes = C.c_int(0), C.c_int(0)
    st = lib().oracle_zfp_block_quantise(_p(v, C.c_float), int(minexp), _p(q, C.c_int32),
                                         C.byref(emax), C.byref(planes))
    if st:
        raise ValueError(f"quantise failed: {st}")
    return q, emax.value, planes.value
