"""Differentiable modelling (autograd over the checkpointed sweeps): the
backward pass is the adjoint sweep with dL/dd as adjoint source (Sec. 2,
Eq. (4)), checked against the one-call gradient, the FP64 oracle, the Taylor
expansion of the misfit (Sec. 4.4) and a short inversion (Sec. 4.6)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _shot(nx=40, ny=36, nz=30, nt=90, nbl=6):
    from paper_2009_12623_gb300 import synth
    from paper_2009_12623_gb300.api import Geometry
    rng = np.random.default_rng(4)
    z = np.arange(nz)[:, None, None]
    v0 = (np.where(z < nz // 2, 1500.0, 2200.0) * np.ones((nz, ny, nx))).astype(np.float32)
    vt = (v0 * (1 + 0.04 * rng.uniform(-1, 1, v0.shape))).astype(np.float32)
    rec = np.array([(i, j, 3) for i in range(nbl, nx - nbl, 3) for j in (ny // 3, 2 * ny // 3)], np.int32)
    g = Geometry(nx=nx, ny=ny, nz=nz, h=10.0, dt=1e-3, nt=nt, nbl=nbl, vmax=2400.0)
    return synth.Shot("ad", g, 25.0, (nx // 2, ny // 2, 4), rec, vt, v0)


def _t(cuda, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(cuda)


@pytest.mark.parametrize("mode,k,atol", [(1, 1, 0.0), (2, 7, 0.0), (1, 1, 1e-5), (2, 10, 1e-5),
                                         (3, 3, 0.0), (3, 4, 1e-5)])
def test_autograd_equals_one_call_gradient(cuda, mode, k, atol):
    from paper_2009_12623_gb300 import api, autograd, synth
    shot = _shot()
    m = _t(cuda, synth.slowness2(shot.v0))
    rec = _t(cuda, shot.rec)
    d_obs = api.forward(shot.geom, _t(cuda, synth.slowness2(shot.v_true)), shot.wavelet, shot.src, rec)
    with api.CheckpointStore(1 << 28) as st:
        g_ref, phi_ref = api.gradient(shot.geom, m, shot.wavelet, shot.src, rec, d_obs, st, mode=mode, k=k,
                                      atol=atol)
    with api.CheckpointStore(1 << 28) as st:
        mm = m.clone().requires_grad_(True)
        d = autograd.model(mm, shot.geom, shot.wavelet, shot.src, rec, st, mode=mode, k=k, atol=atol)
        loss = 0.5 * ((d - d_obs).double() ** 2).sum()
        loss.backward()
    assert float(loss) == pytest.approx(phi_ref, rel=1e-12)
    assert torch.equal(mm.grad, g_ref)


def test_adjoint_requires_matching_forward(cuda):
    from paper_2009_12623_gb300 import api, synth
    shot = _shot(nt=20)
    m = _t(cuda, synth.slowness2(shot.v0))
    rec = _t(cuda, shot.rec)
    resid = torch.zeros((20, len(shot.rec)), device=cuda)
    with api.CheckpointStore(1 << 26) as st:
        with pytest.raises(api.FwiError):   # empty store
            api.adjoint_store(shot.geom, m, shot.wavelet, shot.src, rec, resid, st)
        api.forward_store(shot.geom, m, shot.wavelet, shot.src, rec, st, mode=2, k=5, atol=1e-4)
        with pytest.raises(api.FwiError):   # different policy
            api.adjoint_store(shot.geom, m, shot.wavelet, shot.src, rec, resid, st, mode=2, k=4, atol=1e-4)
        g = api.adjoint_store(shot.geom, m, shot.wavelet, shot.src, rec, resid, st, mode=2, k=5, atol=1e-4)
        assert float(g.abs().max()) == 0.0


def test_autograd_matches_fp64_oracle(cuda, oracle):
    from paper_2009_12623_gb300 import api, autograd, synth
    shot = _shot()
    g = shot.geom
    og = oracle.geometry(g.nx, g.ny, g.nz, g.h, g.dt, g.nt, g.nbl, g.sponge_R, g.vmax)
    w = shot.wavelet.astype(np.float64)
    d_obs = oracle.forward(og, synth.slowness2(shot.v_true).astype(np.float64), w, shot.src, shot.rec)
    g_ref, *_ = oracle.gradient(og, synth.slowness2(shot.v0).astype(np.float64), w, shot.src, shot.rec, d_obs)
    mm = _t(cuda, synth.slowness2(shot.v0)).requires_grad_(True)
    with api.CheckpointStore(1 << 28) as st:
        d = autograd.model(mm, g, shot.wavelet, shot.src, _t(cuda, shot.rec), st)
        (0.5 * ((d - _t(cuda, d_obs.astype(np.float32))).double() ** 2).sum()).backward()
    gg = mm.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - g_ref) / np.linalg.norm(g_ref) < 1e-4


def test_taylor_second_order_on_gpu(cuda):
    """|Phi(m + h dm) - Phi(m) - h <g, dm>| shrinks ~4x per halving of h; the
    perturbation vanishes inside the absorbing layer (where the layer's
    damping is tied to the model)."""
    from paper_2009_12623_gb300 import api, autograd, synth
    shot = _shot(nt=120)
    m = _t(cuda, synth.slowness2(shot.v0))
    rec = _t(cuda, shot.rec)
    d_obs = api.forward(shot.geom, _t(cuda, synth.slowness2(shot.v_true)), shot.wavelet, shot.src, rec)

    def phi(mm):
        d = api.forward(shot.geom, mm, shot.wavelet, shot.src, rec)
        return float(0.5 * ((d - d_obs).double() ** 2).sum())

    with api.CheckpointStore(1 << 28) as st:
        mm = m.clone().requires_grad_(True)
        d = autograd.model(mm, shot.geom, shot.wavelet, shot.src, rec, st)
        loss = 0.5 * ((d - d_obs).double() ** 2).sum()
        loss.backward()
    g = mm.grad
    rng = np.random.default_rng(0)
    dm = np.zeros(shot.geom.shape, np.float32)
    nb = shot.geom.nbl
    inner = rng.normal(size=dm[nb:-nb, nb:-nb, nb:-nb].shape)
    dm[nb:-nb, nb:-nb, nb:-nb] = inner * 0.02 * float(m.mean())
    dmt = _t(cuda, dm)
    lin = api.dot_f64(g, dmt)
    p0 = float(loss)
    hs = [1.0, 0.5, 0.25, 0.125]
    rem = [abs(phi(m + h * dmt) - p0 - h * lin) for h in hs]
    slopes = np.diff(np.log(rem)) / np.diff(np.log(hs))
    assert np.all(np.abs(slopes - 2.0) < 0.25), (rem, slopes)


def test_short_inversion_reduces_misfit(cuda):
    from paper_2009_12623_gb300 import api, invert, synth
    shots = []
    base = _shot(nt=100)
    rec = _t(cuda, base.rec)
    mt = _t(cuda, synth.slowness2(base.v_true))
    d_obs = []
    for sx in (12, 20, 28):
        src = (sx, base.geom.ny // 2, 4)
        shots.append((base.geom, base.wavelet, src, rec))
        d_obs.append(api.forward(base.geom, mt, base.wavelet, src, rec))
    c0 = _t(cuda, base.v0)
    c, hist = invert.invert(c0, shots, d_obs, iters=4, atol=1e-5, step=0.01, store_bytes=1 << 28)
    assert hist[-1] < hist[0], hist


def test_gradient_angle_vs_fp64_oracle_across_atol(cuda, oracle):
    """The angle between the autograd gradient with compressed checkpoints
    and the uncompressed FP64 oracle gradient (Sec. 4.4's gradient-angle
    experiment) on a reduced version of the differentiable-FWI case (layered
    model with +-8% anomalies, smoothed start): it shrinks as atol tightens
    and stays small at every tolerance."""
    from paper_2009_12623_gb300 import api, autograd, synth
    nx, ny, nz, nbl, nt = 48, 44, 36, 8, 220
    v = synth.layered_velocity(nx, ny, nz, seed=1, water=nbl + 3, vmax=3000.0, nlayers=6, fault_shift=4)
    vt = synth.add_anomalies(v, seed=2, amplitude=0.08)
    v0 = synth.smooth(vt, 2.0)
    g = api.Geometry(nx=nx, ny=ny, nz=nz, h=10.0, dt=1e-3, nt=nt, nbl=nbl, vmax=float(vt.max()))
    w = synth.wavelet(nt, g.dt, 20.0)
    src = (nx // 2, ny // 2, nbl + 2)
    rec = np.array([(i, j, nbl + 2) for i in range(nbl, nx - nbl, 2) for j in range(nbl, ny - nbl, 4)], np.int32)
    og = oracle.geometry(nx, ny, nz, g.h, g.dt, nt, nbl, g.sponge_R, g.vmax)
    d_obs = oracle.forward(og, synth.slowness2(vt).astype(np.float64), w.astype(np.float64), src, rec)
    g_ref, *_ = oracle.gradient(og, synth.slowness2(v0).astype(np.float64), w.astype(np.float64), src, rec, d_obs)
    obs = _t(cuda, d_obs.astype(np.float32))
    angles = {}
    for atol in (1e-2, 1e-4, 1e-6):
        mm = _t(cuda, synth.slowness2(v0)).requires_grad_(True)
        with api.CheckpointStore(1 << 30) as st:
            d = autograd.model(mm, g, w, src, _t(cuda, rec), st, mode=api.FWI_CKPT_FULL, atol=atol)
            (0.5 * ((d - obs).double() ** 2).sum()).backward()
        gg = mm.grad.cpu().numpy().astype(np.float64)
        cos = float(np.dot(gg.ravel(), g_ref.ravel()) / (np.linalg.norm(gg) * np.linalg.norm(g_ref)))
        angles[atol] = float(np.arccos(min(1.0, cos)))
    print("gradient angle vs FP64 oracle:", angles)
    assert angles[1e-2] >= angles[1e-4] >= angles[1e-6] * 0.9
    assert angles[1e-6] < 1e-3 and angles[1e-4] < 1e-3 and angles[1e-2] < 5e-2
