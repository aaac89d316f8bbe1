"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method itself (no stencil, damping,
adjoint, imaging or codec step): only input construction -- velocity models,
source wavelet samples, acquisition geometry and test wavefields.  Both the
GPU path and the CPU oracle receive the arrays it returns.

The paper's experiments use the SEG/EAGE Overthrust model, which is not
available here; the layered model below stands in for it (Sec. 3, "Reference
Problem": 287 x 881 x 881 points including a 40-point absorbing layer, 4000 ms
at dt = 1.75 ms, 8 Hz Ricker source just under the water surface, smoothed
starting model).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .api import Geometry, ShotSpec


def ricker(t, f: float, t0: float):
    """Ricker wavelet (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2), tau = t - t0."""
    a = (np.pi * f * (np.asarray(t, dtype=np.float64) - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def wavelet(nt: int, dt: float, f: float, t0: float | None = None) -> np.ndarray:
    """Source samples q^n = ricker(n dt) with delay t0 = 1.5/f (default)."""
    t0 = 1.5 / f if t0 is None else t0
    return ricker(np.arange(nt) * dt, f, t0).astype(np.float32)


def slowness2(v: np.ndarray) -> np.ndarray:
    """Squared slowness m = 1/c^2 (the model the PDE is written in)."""
    v = np.asarray(v, dtype=np.float64)
    return (1.0 / (v * v)).astype(np.float32)


@dataclass
class Shot:
    name: str
    geom: Geometry
    f: float
    src: tuple
    rec: np.ndarray       # (nrec, 3) int32 (i, j, k)
    v_true: np.ndarray    # (nz, ny, nx) float32, generates d_obs
    v0: np.ndarray        # (nz, ny, nx) float32, model where the gradient is taken

    @property
    def wavelet(self) -> np.ndarray:
        return wavelet(self.geom.nt, self.geom.dt, self.f)


def two_layer_shot(n: int = 64, nt: int = 200, h: float = 10.0, dt: float = 1e-3, nbl: int = 10,
                   f: float = 10.0) -> Shot:
    """Plain checkpointed-gradient case: n^3 grid at h, 1500 m/s over 2500 m/s
    at z = n/2, true model with a +10% Gaussian blob (sigma 5 cells) at the
    centre, source at (n/2, n/2, 4), receivers along x at y = n/2, z = 4."""
    z = np.arange(n)[:, None, None]
    v0 = np.where(z < n // 2, 1500.0, 2500.0) * np.ones((n, n, n))
    zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    c = n // 2
    blob = np.exp(-((xx - c) ** 2 + (yy - c) ** 2 + (zz - c) ** 2) / (2.0 * 5.0 ** 2))
    v_true = v0 * (1.0 + 0.1 * blob)
    rec = np.stack([np.arange(n), np.full(n, c), np.full(n, 4)], axis=1).astype(np.int32)
    geom = Geometry(nx=n, ny=n, nz=n, h=h, dt=dt, nt=nt, nbl=nbl, vmax=float(v_true.max()))
    return Shot("two_layer", geom, f, (c, c, 4), rec, v_true.astype(np.float32), v0.astype(np.float32))


def layered_velocity(nx: int, ny: int, nz: int, seed: int = 0, nlayers: int = 12,
                     vmin: float = 1500.0, vmax: float = 6000.0, water: int = 50,
                     fault_shift: int = 20) -> np.ndarray:
    """Layered model: a water layer of `water` cells, then nlayers layers with
    velocities rising from vmin to vmax, interfaces undulating as
    zbar_k + A_k sin(2 pi x / lx_k + phi_k) sin(2 pi y / ly_k + psi_k), and two
    planar dipping thrust faults whose hanging walls are lifted by
    fault_shift cells.  Built slab by slab in z to bound host memory."""
    rng = np.random.default_rng(seed)
    vel = np.linspace(vmin, vmax, nlayers + 1)[1:] if nlayers > 0 else np.array([])
    vel = np.concatenate([[vmin], vel]).astype(np.float32)
    zbar = np.linspace(water, nz - 1, nlayers + 1)[:-1] + rng.uniform(-2, 2, nlayers)
    zbar[0] = water
    amp = rng.uniform(2.0, 0.04 * nz + 2.0, nlayers)
    amp[0] = 0.0
    lx = rng.uniform(0.3, 1.2, nlayers) * nx
    ly = rng.uniform(0.3, 1.2, nlayers) * ny
    phx = rng.uniform(0, 2 * np.pi, nlayers)
    phy = rng.uniform(0, 2 * np.pi, nlayers)
    x = np.arange(nx, dtype=np.float32)[None, :]
    y = np.arange(ny, dtype=np.float32)[:, None]
    surfaces = [(zbar[k] + amp[k] * np.sin(2 * np.pi * x / lx[k] + phx[k])
                 * np.sin(2 * np.pi * y / ly[k] + phy[k])).astype(np.float32) for k in range(nlayers)]
    # faults: planes through (xf, zf) dipping along x (and slightly along y)
    faults = []
    for _ in range(2):
        xf = rng.uniform(0.25, 0.75) * nx
        zf = rng.uniform(0.4, 0.8) * nz
        dip = np.tan(np.deg2rad(rng.uniform(25, 45))) * rng.choice([-1.0, 1.0])
        sy = rng.uniform(-0.2, 0.2)
        faults.append((xf, zf, dip, sy))
    out = np.empty((nz, ny, nx), dtype=np.float32)
    for z0 in range(0, nz, 16):
        z1 = min(nz, z0 + 16)
        zz = np.arange(z0, z1, dtype=np.float32)[:, None, None]
        zeff = np.broadcast_to(zz, (z1 - z0, ny, nx)).copy()
        for xf, zf, dip, sy in faults:
            side = (x[None] - xf - sy * (y[None] - ny / 2)) + dip * (zz - zf)
            zeff = np.where((side > 0) & (zz > water), zeff + fault_shift, zeff)
        idx = np.zeros((z1 - z0, ny, nx), dtype=np.int32)
        for s in surfaces:
            idx += (zeff >= s[None]).astype(np.int32)
        idx = np.where(zz < water, 0, np.maximum(idx, 1))
        out[z0:z1] = vel[idx]
    return out


def add_anomalies(v: np.ndarray, seed: int = 0, n: int = 3, amplitude: float = 0.08,
                  sigma_frac: float = 0.08) -> np.ndarray:
    """v * (1 + sum_j a_j exp(-|x - x_j|^2 / 2 s^2)) with n Gaussian anomalies of
    amplitude +-`amplitude` (alternating sign), centres uniform in the middle
    half of the model, width s = sigma_frac * min(nx, ny, nz) cells."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = v.shape
    s = sigma_frac * min(nx, ny, nz)
    z = np.arange(nz, dtype=np.float32)[:, None, None]
    y = np.arange(ny, dtype=np.float32)[None, :, None]
    x = np.arange(nx, dtype=np.float32)[None, None, :]
    out = np.ones_like(v, dtype=np.float32)
    for j in range(n):
        cz, cy, cx = (rng.uniform(0.25, 0.75) * d for d in (nz, ny, nx))
        a = amplitude * (1 if j % 2 == 0 else -1)
        out += a * np.exp(-((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) / (2 * s * s)).astype(np.float32)
    return (v * out).astype(np.float32)


def smooth(v: np.ndarray, sigma_cells: float) -> np.ndarray:
    """Gaussian-smoothed copy (the paper's starting model, Sec. 3)."""
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(v.astype(np.float32), sigma=sigma_cells, mode="nearest").astype(np.float32)


def overthrust_like_shot(nx: int = 881, ny: int = 881, nz: int = 287, nt: int = 2286,
                         h: float = 25.0, dt: float = 1.75e-3, nbl: int = 40, f: float = 8.0,
                         seed: int = 0, rec_stride: int = 2, smooth_cells: float = 6.0,
                         src_xy=None) -> Shot:
    """Overthrust-shaped single shot: layered model (1500-6000 m/s), source near
    the surface centre at depth nbl+2, receivers on every rec_stride-th (x, y)
    node of that plane."""
    v_true = layered_velocity(nx, ny, nz, seed=seed, water=min(nbl + 10, nz // 3))
    v0 = smooth(v_true, smooth_cells)
    zr = min(nbl + 2, nz - 1)
    xs = np.arange(0, nx, rec_stride)
    ys = np.arange(0, ny, rec_stride)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    rec = np.stack([X.ravel(), Y.ravel(), np.full(X.size, zr)], axis=1).astype(np.int32)
    sx, sy = src_xy if src_xy is not None else (nx // 2, ny // 2)
    geom = Geometry(nx=nx, ny=ny, nz=nz, h=h, dt=dt, nt=nt, nbl=nbl, vmax=float(v_true.max()))
    return Shot("overthrust_like", geom, f, (int(sx), int(sy), zr), rec, v_true, v0)


def wavefield_snapshot(shot: Shot, t: float, planes) -> np.ndarray:
    """Analytic stand-in for the shot's wavefield at time t on the given
    z-planes (float32, (len(planes), ny, nx)): the direct wave and the
    reflections from every layer interface of the velocity column under the
    source, each a spherical Ricker front h^3 q(t - r/c) / (4 pi r) from the
    source or its mirror image across the interface (amplitude scaled by the
    normal-incidence reflection coefficient, speed the mean velocity above
    the interface).  A seeded, reproducible input shaped like a propagated
    state, for timing the codec on the same data anywhere."""
    g = shot.geom
    sx, sy, sz = shot.src
    col = shot.v_true[:, sy, sx].astype(np.float64)
    fronts = [(float(sz), float(col[sz]), 1.0)]
    for zk in np.nonzero(np.diff(col))[0] + 1:
        if zk <= sz:
            continue
        r = (col[zk] - col[zk - 1]) / (col[zk] + col[zk - 1])
        fronts.append((2.0 * zk - sz, float(col[sz:zk].mean()), float(r)))
    x = (np.arange(g.nx) - sx)[None, :] * g.h
    y = (np.arange(g.ny) - sy)[:, None] * g.h
    rxy2 = x * x + y * y
    t0 = 1.5 / shot.f
    out = np.zeros((len(planes), g.ny, g.nx), np.float32)
    for i, z in enumerate(planes):
        acc = np.zeros(g.ny * g.nx)
        for zi, c, a in fronts:
            r = np.sqrt(rxy2 + ((z - zi) * g.h) ** 2).ravel()
            near = np.nonzero(np.abs(t - r / c - t0) < 3.0 / shot.f)[0]   # the front's support
            rr = r[near]
            acc[near] += a * g.h ** 3 / (4 * np.pi * np.maximum(rr, g.h)) * ricker(t - rr / c, shot.f, t0)
        out[i] = acc.reshape(g.ny, g.nx)
    return out


def shells_field(n: int = 512, seed: int = 0, nshell: int = 8, f: float = 15.0, h: float = 10.0,
                 c: float = 1500.0, rmin: float = 50.0, rmax: float = 200.0,
                 noise: float = 1e-7) -> np.ndarray:
    """Codec benchmark snapshot: sum of nshell spherical Ricker shells
    A_j ricker((r - R_j) h / c) with A_j ~ N(0,1), centres uniform in the cube,
    R_j ~ U(rmin, rmax) cells, plus noise * N(0,1)."""
    rng = np.random.default_rng(seed)
    A = rng.normal(size=nshell)
    C0 = rng.uniform(0, n, size=(nshell, 3))
    R = rng.uniform(rmin, rmax, size=nshell)
    out = np.empty((n, n, n), dtype=np.float32)
    y = np.arange(n, dtype=np.float32)[:, None]
    x = np.arange(n, dtype=np.float32)[None, :]
    for z0 in range(0, n, 32):
        z1 = min(n, z0 + 32)
        z = np.arange(z0, z1, dtype=np.float32)[:, None, None]
        acc = np.zeros((z1 - z0, n, n), dtype=np.float32)
        for j in range(nshell):
            r = np.sqrt((x - C0[j, 0]) ** 2 + (y - C0[j, 1]) ** 2 + (z - C0[j, 2]) ** 2)
            acc += (A[j] * ricker((r - R[j]) * h / c, f, 0.0)).astype(np.float32)
        out[z0:z1] = acc
    out += (noise * rng.normal(size=out.shape)).astype(np.float32)
    return out


@dataclass
class Survey:
    """Many shots over one model: `geom` is the model grid (nt = the longest
    record), each ShotSpec gives a shot's aperture, record length, source
    and receivers."""
    geom: Geometry
    f: float
    v_true: np.ndarray
    v0: np.ndarray
    shots: list

    def wavelets(self) -> list:
        return [wavelet(s.nt, self.geom.dt, self.f) for s in self.shots]


def batch_survey(nx: int = 600, ny: int = 600, nz: int = 200, nshots: int = 32, h: float = 20.0,
                 dt: float = 1.5e-3, f: float = 10.0, nbl: int = 40, ap_min: int = 200, ap_max: int = 600,
                 t_min: float = 1.5, t_max: float = 3.0, rec_stride: int = 4, seed: int = 0,
                 vmin: float = 1500.0, vmax: float = 6000.0, smooth_cells: float = 6.0) -> Survey:
    """Batched-shot survey over the layered model: per shot, aperture sides
    (x, y) uniform in [ap_min, ap_max] cells (full depth), centred on a source
    drawn uniformly over the surface at depth nbl+2 and shifted to stay in the
    grid, record length uniform in [t_min, t_max] s, receivers on every
    rec_stride-th (x, y) node of the aperture at the source depth."""
    rng = np.random.default_rng(seed)
    v_true = layered_velocity(nx, ny, nz, seed=seed, water=min(nbl + 10, nz // 3), vmin=vmin, vmax=vmax)
    v0 = smooth(v_true, smooth_cells)
    zs = min(nbl + 2, nz - 1)
    shots = []
    for _ in range(nshots):
        ax = min(int(rng.integers(ap_min, ap_max + 1)), nx)
        ay = min(int(rng.integers(ap_min, ap_max + 1)), ny)
        sx, sy = int(rng.integers(0, nx)), int(rng.integers(0, ny))
        x0 = int(np.clip(sx - ax // 2, 0, nx - ax))
        y0 = int(np.clip(sy - ay // 2, 0, ny - ay))
        sx = int(np.clip(sx, x0, x0 + ax - 1))
        sy = int(np.clip(sy, y0, y0 + ay - 1))
        nt = max(1, int(round(rng.uniform(t_min, t_max) / dt)))
        X, Y = np.meshgrid(np.arange(x0, x0 + ax, rec_stride), np.arange(y0, y0 + ay, rec_stride), indexing="xy")
        rec = np.stack([X.ravel(), Y.ravel(), np.full(X.size, zs)], axis=1).astype(np.int32)
        shots.append(ShotSpec(x0, y0, 0, ax, ay, nz, nt, (sx, sy, zs), rec))
    geom = Geometry(nx=nx, ny=ny, nz=nz, h=h, dt=dt, nt=max(s.nt for s in shots), nbl=nbl,
                    vmax=float(v_true.max()))
    return Survey(geom, f, v_true, v0, shots)
