"""Differentiable forward modelling: torch.autograd.Function over the C ABI.

The forward pass runs the checkpointed forward sweep (fwi_forward_store), which
returns the shot record d = P_r A(m)^-1 P_s^T q (Sec. 2, Eq. (2)) and keeps the
forward wavefield as (optionally compressed) checkpoints in a store.  The
backward pass receives dL/dd for whatever loss the caller built and runs the
reverse sweep from those checkpoints (fwi_adjoint_store), returning
dL/dm = J^T dL/dd -- the imaging condition of Eq. (4) with dL/dd as adjoint
source.  Lossy checkpoint compression (Sec. 1.4) thus replaces full-history
storage in an ordinary PyTorch training loop.
"""
from __future__ import annotations

import torch

from . import api


class ShotModeling(torch.autograd.Function):
    """m (squared slowness, [nz, ny, nx]) -> records [nt, nrec] for one shot."""

    @staticmethod
    def forward(ctx, m, geom, wavelet, src, rec, store, mode, k, atol):
        m = m.detach().contiguous()
        d = api.forward_store(geom, m, wavelet, src, rec, store, mode=mode, k=k, atol=atol)
        ctx.save_for_backward(m)
        ctx.args = (geom, wavelet, src, rec, store, mode, k, atol)
        return d

    @staticmethod
    def backward(ctx, grad_d):
        (m,) = ctx.saved_tensors
        geom, wavelet, src, rec, store, mode, k, atol = ctx.args
        g = api.adjoint_store(geom, m, wavelet, src, rec, grad_d.contiguous(), store, mode=mode, k=k,
                              atol=atol)
        return g, None, None, None, None, None, None, None, None


def model(m: torch.Tensor, geom: api.Geometry, wavelet, src, rec: torch.Tensor,
          store: api.CheckpointStore, mode: int = api.FWI_CKPT_FULL, k: int = 1,
          atol: float = 0.0) -> torch.Tensor:
    """Differentiable shot record of squared slowness m."""
    return ShotModeling.apply(m, geom, wavelet, src, rec, store, mode, k, atol)


def model_velocity(c: torch.Tensor, geom: api.Geometry, wavelet, src, rec: torch.Tensor,
                   store: api.CheckpointStore, mode: int = api.FWI_CKPT_FULL, k: int = 1,
                   atol: float = 0.0) -> torch.Tensor:
    """Differentiable shot record of velocity c (m = 1/c^2, Eq. (1))."""
    return model(1.0 / (c * c), geom, wavelet, src, rec, store, mode, k, atol)


class SurveyModeling(torch.autograd.Function):
    """m (model grid) -> the flat records of every shot of a batch plan
    (api.Batch): one batched forward sweep keeps all shots' checkpoints in
    the plan; the backward is one batched reverse sweep, returning
    sum_s J_s^T dL/dd_s stacked on the model grid.  Each backward must follow
    its own forward (the plan holds one set of checkpoints)."""

    @staticmethod
    def forward(ctx, m, plan, wavelets):
        m = m.detach().contiguous()
        d = plan.forward(m, wavelets)
        ctx.save_for_backward(m)
        ctx.plan, ctx.wavelets = plan, wavelets
        return d

    @staticmethod
    def backward(ctx, grad_d):
        (m,) = ctx.saved_tensors
        g = ctx.plan.adjoint(m, ctx.wavelets, grad_d.contiguous())
        return g, None, None


def survey(m: torch.Tensor, plan: api.Batch, wavelets) -> torch.Tensor:
    """Differentiable flat records of all shots of `plan` (split with plan.split)."""
    return SurveyModeling.apply(m, plan, wavelets)


def survey_velocity(c: torch.Tensor, plan: api.Batch, wavelets) -> torch.Tensor:
    """Differentiable flat records of all shots as a function of velocity c."""
    return survey(1.0 / (c * c), plan, wavelets)
