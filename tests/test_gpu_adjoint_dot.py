"""Dot-product tests of the GPU operators through the library's own entry
points (Sec. 2: the wave operator is self-adjoint, and the gradient of
Eq. (4) is the adjoint of the linearised modelling), with every inner
product reduced in FP64 on the GPU (fwi_dot_f64).

* Forward modelling d = F q = P_r A^-1 P_s^T q (Eq. (2)) is linear in the
  source samples.  Its transpose is correlation with the same Green's
  function, and source-receiver reciprocity of the discrete scheme makes
  that a time-reversed forward run from the receiver to the source:
  <F_{s->r} q, w> = <q, R F_{r->s} R w>, R reversing time.
* The linearised modelling J dm (the Born record) of a single-cell
  perturbation dm = e_c is a forward run with a point source at c whose
  samples are -(u^{n+1} - 2u^n + u^{n-1})/dt^2 at c (the m-term of the
  discrete equation, differentiated), u at c being recorded by a first
  forward run.  The adjoint sweep of the library (fwi_forward_store +
  fwi_adjoint_store, the path the gradient takes) must give
  <J e_c, dd> = (J^T dd)[c] for any residual dd.

Cells are taken outside the absorbing layer, whose damping the gradient
holds fixed.  Both sides are FP32 sweeps of a few hundred steps, so they
agree to FP32 rounding; the bound is the benchmark spec's tolerance 1e-4."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _case(nt=160):
    from paper_2009_12623_gb300 import synth
    from paper_2009_12623_gb300.api import Geometry
    nx, ny, nz, nbl = 44, 40, 36, 8
    v = synth.layered_velocity(nx, ny, nz, seed=3, water=nbl + 3, vmax=3000.0, nlayers=5, fault_shift=4)
    v = synth.smooth(v, 1.5)
    g = Geometry(nx=nx, ny=ny, nz=nz, h=10.0, dt=1e-3, nt=nt, nbl=nbl, vmax=float(v.max()))
    return g, synth.slowness2(v), synth.wavelet(nt, g.dt, 20.0)


def _t(cuda, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(cuda)


def _fwd(cuda, g, m, w, src, rec):
    from paper_2009_12623_gb300 import api
    return api.forward(g, m, np.asarray(w, np.float32), src, _t(cuda, np.asarray(rec, np.int32).reshape(-1, 3)))


def test_forward_dot_product_by_reciprocity(cuda):
    from paper_2009_12623_gb300 import api
    g, m_h, w = _case()
    m = _t(cuda, m_h)
    src = (22, 20, 11)
    recs = [(14, 12, 11), (30, 27, 20), (25, 18, 26)]
    rng = np.random.default_rng(5)
    q = rng.normal(size=g.nt).astype(np.float32)
    lhs = rhs = 0.0
    for r in recs:
        wr = rng.normal(size=g.nt).astype(np.float32)
        d = _fwd(cuda, g, m, q, src, [r])[:, 0].contiguous()                # F_{s->r} q
        back = _fwd(cuda, g, m, wr[::-1].copy(), r, [src])[:, 0].flip(0).contiguous()  # R F_{r->s} R w
        lhs += api.dot_f64(d, _t(cuda, wr))
        rhs += api.dot_f64(_t(cuda, q), back)
    assert abs(lhs - rhs) <= TOL * max(abs(lhs), abs(rhs)), (lhs, rhs)


@pytest.mark.parametrize("mode,k", [(1, 1), (2, 9), (3, 6)])
def test_born_dot_product_through_the_adjoint_sweep(cuda, mode, k):
    from paper_2009_12623_gb300 import api
    g, m_h, w = _case()
    m = _t(cuda, m_h)
    src = (22, 20, 11)
    rec = np.array([(i, j, 11) for i in range(8, 36, 3) for j in (12, 28)], np.int32)
    rng = np.random.default_rng(7)
    dd = _t(cuda, rng.normal(size=(g.nt, len(rec))).astype(np.float32))
    with api.CheckpointStore(1 << 28) as st:
        api.forward_store(g, m, w, src, _t(cuda, rec), st, mode=mode, k=k)
        grad = api.adjoint_store(g, m, w, src, _t(cuda, rec), dd, st, mode=mode, k=k)   # J^T dd
    gh = grad.cpu().numpy()
    for c in [(22, 20, 16), (15, 26, 22), (29, 13, 27)]:
        uc = _fwd(cuda, g, m, w, src, [c])[:, 0].double().cpu().numpy()   # u^{n+1} at c, n = 0..nt-1
        u = np.concatenate([[0.0, 0.0], uc])                                # u^{-1}, u^0, u^1, ...
        qb = -(u[2:] - 2.0 * u[1:-1] + u[:-2]) / g.dt ** 2                  # Born source at c
        jdm = _fwd(cuda, g, m, qb.astype(np.float32), c, rec)               # J e_c
        lhs = api.dot_f64(jdm.contiguous(), dd)
        rhs = float(gh[c[2], c[1], c[0]])
        assert abs(lhs - rhs) <= TOL * abs(rhs), (c, lhs, rhs)
