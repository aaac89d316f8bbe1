"""Multi-shot FWI with lossy checkpoint compression (the inversion of Sec. 4.6).

The objective is the sum over shots of 1/2 ||d_sim - d_obs||^2 (Eq. (3));
its gradient is the stack (sum) of per-shot gradients (Sec. 2, stacking),
each computed through the checkpointed, compressed adjoint sweep.  The first
gradient's norm scales all later ones (Sec. 3: "the gradient was scaled by
dividing by the norm of the original gradient in the first iteration").

    python -m paper_2009_12623_gb300.invert --help
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import api, autograd, synth


def misfit_and_gradient(c: torch.Tensor, shots, d_obs, stores, mode, k, atol):
    """Sum over shots of the misfit and its gradient w.r.t. velocity c."""
    c = c.detach().requires_grad_(True)
    total = torch.zeros((), dtype=torch.float64, device=c.device)
    for (geom, w, src, rec), dobs, st in zip(shots, d_obs, stores):
        d = autograd.model_velocity(c, geom, w, src, rec, st, mode=mode, k=k, atol=atol)
        r = d - dobs
        loss = 0.5 * (r.double() * r.double()).sum()
        loss.backward()
        total = total + loss.detach()
    return float(total), c.grad.detach()


def misfit_and_gradient_batched(c: torch.Tensor, plan: api.Batch, wavelets, d_obs_flat: torch.Tensor):
    """The same through one batch plan: all shots in one batched forward and
    one batched reverse sweep (autograd.SurveyModeling)."""
    c = c.detach().requires_grad_(True)
    d = autograd.survey_velocity(c, plan, wavelets)
    r = d - d_obs_flat
    loss = 0.5 * (r.double() * r.double()).sum()
    loss.backward()
    return float(loss.detach()), c.grad.detach()


def descend(c0: torch.Tensor, grad_fn, iters: int, step: float, vmin: float, vmax: float,
            mask: torch.Tensor | None, resume: dict | None = None, on_iter=None):
    """Steepest descent on velocity.  Every gradient is divided by the size of
    the first iteration's gradient (its largest magnitude), so the first
    update changes the model by at most step x mean velocity and later
    updates shrink with the gradient; returns (c, misfit history, first gradient).

    `resume` (a dict from load_state) continues an earlier run where it
    stopped: its model, misfit history, gradient scale and the starting
    model's mean velocity, so that the continued iterations are the ones an
    uninterrupted run would take.  `on_iter(state)` is called after every
    iteration with that dict (save_state writes it to a file)."""
    c = c0.clone()
    hist = []
    g0 = None
    cmean = float(c0.mean())
    if resume is not None:
        c = resume["c"].to(device=c0.device, dtype=c0.dtype).clone()
        hist = list(resume["hist"])
        g0 = resume["g0"]
        cmean = resume["c0_mean"]
    first = None
    for _ in range(len(hist), iters):
        phi, g = grad_fn(c)
        if mask is not None:
            g = g * mask
        if g0 is None:
            g0 = float(g.abs().max())
            first = g.clone()
        hist.append(phi)
        c = (c - step * cmean * g / g0).clamp(vmin, vmax)
        if on_iter is not None:
            on_iter({"c": c, "hist": hist, "g0": g0, "c0_mean": cmean})
    return c, hist, first


def save_state(path: str, state: dict) -> None:
    """Write a descent state (model, misfit history, gradient scale, starting
    mean velocity) to an .npz file, atomically."""
    tmp = path + ".tmp.npz"
    np.savez(tmp, c=state["c"].detach().cpu().numpy(), hist=np.asarray(state["hist"], np.float64),
             g0=np.float64(state["g0"]), c0_mean=np.float64(state["c0_mean"]))
    os.replace(tmp, path)


def load_state(path: str) -> dict:
    """Read a descent state written by save_state."""
    with np.load(path) as z:
        return {"c": torch.from_numpy(z["c"]), "hist": [float(x) for x in z["hist"]],
                "g0": float(z["g0"]), "c0_mean": float(z["c0_mean"])}


def invert(c0: torch.Tensor, shots, d_obs, iters: int = 10, mode=api.FWI_CKPT_FULL, k: int = 1,
           atol: float = 1e-4, step: float = 0.02, store_bytes: int = 16 << 30,
           vmin: float = 1400.0, vmax: float = 6500.0, mask: torch.Tensor | None = None,
           resume: dict | None = None, on_iter=None):
    """Steepest descent with one checkpointed gradient call per shot; each
    shot's backward runs right after its forward, so one store serves them
    all.  Returns (c, misfit history)."""
    store = api.CheckpointStore(store_bytes)
    stores = [store] * len(shots)
    try:
        c, hist, _ = descend(c0, lambda cc: misfit_and_gradient(cc, shots, d_obs, stores, mode, k, atol),
                             iters, step, vmin, vmax, mask, resume, on_iter)
    finally:
        store.close()
    return c, hist


def invert_batched(c0: torch.Tensor, plan: api.Batch, wavelets, d_obs_flat: torch.Tensor, iters: int = 10,
                   step: float = 0.02, vmin: float = 1400.0, vmax: float = 6500.0,
                   mask: torch.Tensor | None = None, resume: dict | None = None, on_iter=None):
    """Steepest descent through a batch plan (all shots per launch)."""
    c, hist, _ = descend(c0, lambda cc: misfit_and_gradient_batched(cc, plan, wavelets, d_obs_flat),
                         iters, step, vmin, vmax, mask, resume, on_iter)
    return c, hist


def _main():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--grid", default="300,300,150")
    p.add_argument("--h", type=float, default=20.0)
    p.add_argument("--shots", type=int, default=16)
    p.add_argument("--t", type=float, default=2.0, help="record length, s")
    p.add_argument("--f", type=float, default=10.0)
    p.add_argument("--iters", type=int, default=10)
    p.add_argument("--atol", type=float, default=1e-4)
    p.add_argument("--per-shot", action="store_true", help="one gradient call per shot instead of a batch plan")
    p.add_argument("--save", default=None, help="write the descent state (.npz) after every iteration")
    p.add_argument("--resume", default=None, help="continue from a state written by --save")
    a = p.parse_args()
    resume = load_state(a.resume) if a.resume else None
    on_iter = (lambda st: save_state(a.save, st)) if a.save else None
    nx, ny, nz = (int(v) for v in a.grid.split(","))
    dev = torch.device("cuda")
    nbl = min(20, nz // 6)
    v = synth.layered_velocity(nx, ny, nz, seed=1, water=nbl + 5)
    v_true = synth.add_anomalies(v, seed=2, amplitude=0.08)
    v0 = synth.smooth(v_true, 4.0)
    vmax = float(v_true.max())
    dt = 0.4 * a.h / vmax
    nt = int(round(a.t / dt))
    geom = api.Geometry(nx=nx, ny=ny, nz=nz, h=a.h, dt=dt, nt=nt, nbl=nbl, vmax=vmax)
    w = synth.wavelet(nt, dt, a.f)
    zr = nbl + 2
    xs = np.arange(nbl, nx - nbl, 2)
    X, Y = np.meshgrid(xs, np.arange(nbl, ny - nbl, 2))
    rec = torch.from_numpy(np.stack([X.ravel(), Y.ravel(), np.full(X.size, zr)], 1).astype(np.int32)).to(dev)
    side = int(math.ceil(math.sqrt(a.shots)))
    sxs = np.linspace(nbl + 10, nx - nbl - 10, side).astype(int)
    srcs = [(int(sxs[i % side]), int(sxs[i // side]), zr) for i in range(a.shots)]
    shots = [(geom, w, s, rec) for s in srcs]
    mt = torch.from_numpy(synth.slowness2(v_true)).to(dev)
    d_obs = [api.forward(geom, mt, w, s, rec) for s in srcs]
    c0 = torch.from_numpy(v0).to(dev)
    interior = torch.zeros_like(c0)
    interior[nbl:nz - nbl, nbl:ny - nbl, nbl:nx - nbl] = 1.0
    t0 = time.time()
    if a.per_shot:
        c, hist = invert(c0, shots, d_obs, iters=a.iters, atol=a.atol, mask=interior, resume=resume,
                         on_iter=on_iter)
    else:
        specs = [api.ShotSpec(0, 0, 0, nx, ny, nz, nt, s, rec.cpu().numpy()) for s in srcs]
        with api.Batch(geom, specs, mode=api.FWI_CKPT_FULL, atol=a.atol, arena_bytes=64 << 30,
                       graph=True, tune=True) as plan:
            c, hist = invert_batched(c0, plan, [w] * len(srcs), plan.concat(d_obs), iters=a.iters,
                                     mask=interior, resume=resume, on_iter=on_iter)
    torch.cuda.synchronize()
    err0 = float(torch.linalg.vector_norm(c0 - torch.from_numpy(v_true).to(dev)))
    err = float(torch.linalg.vector_norm(c - torch.from_numpy(v_true).to(dev)))
    print(json.dumps({"misfit": hist, "model_error_start": err0, "model_error_end": err,
                      "seconds": time.time() - t0, "nt": nt, "shots": a.shots,
                      "path": "per-shot" if a.per_shot else "batch plan"}))


if __name__ == "__main__":
    _main()
