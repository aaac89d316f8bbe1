"""Batched shots on the GPU (fwi_batch_*): the stacked gradient of a survey
with uneven apertures and record lengths, all shots advanced together in
persistent multi-shot launches.  Checked bit for bit against one
fwi_gradient call per shot (the plain path), and against the FP64 oracle's
stacked gradient; graph replay, the autotuner and the forward/adjoint split
must not change a bit."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _survey(nshots=5, seed=1, **kw):
    from paper_2009_12623_gb300 import synth
    args = dict(nx=56, ny=48, nz=28, nshots=nshots, h=10.0, dt=1e-3, f=25.0, nbl=6, ap_min=20, ap_max=40,
                t_min=0.03, t_max=0.06, rec_stride=3, seed=seed, vmax=3000.0)
    args.update(kw)
    return synth.batch_survey(**args)


def _setup(cuda, sv):
    from paper_2009_12623_gb300 import api, synth
    m = torch.from_numpy(synth.slowness2(sv.v0)).to(cuda)
    mt = torch.from_numpy(synth.slowness2(sv.v_true)).to(cuda)
    w = sv.wavelets()
    d_obs = []
    for s, wi in zip(sv.shots, w):
        origin = torch.tensor([s.x0, s.y0, s.z0], dtype=torch.int32, device=cuda)
        rec = (torch.from_numpy(np.asarray(s.rec, np.int32)).to(cuda) - origin).contiguous()
        src = (s.src[0] - s.x0, s.src[1] - s.y0, s.src[2] - s.z0)
        d_obs.append(api.forward(s.local_geometry(sv.geom), mt[s.window].contiguous(), wi, src, rec))
    return m, w, d_obs


@pytest.mark.parametrize("mode,k,atol", [(1, 1, 0.0), (2, 4, 0.0), (2, 5, 1e-4), (1, 1, 1e-4)])
def test_batch_equals_per_shot_calls_bitwise(cuda, mode, k, atol):
    from paper_2009_12623_gb300 import api
    sv = _survey()
    m, w, d_obs = _setup(cuda, sv)
    with api.CheckpointStore(1 << 28) as st:
        g_ref, phi_ref = api.gradient_per_shot(sv.geom, m, sv.shots, w, d_obs, st, mode=mode, k=k, atol=atol)
    with api.Batch(sv.geom, sv.shots, mode=mode, k=k, atol=atol, arena_bytes=1 << 29) as b:
        g, phi = b.gradient(m, w, b.concat(d_obs))
        stats = b.stats()
    assert torch.equal(g, g_ref)
    assert np.array_equal(phi, phi_ref)
    assert stats["launches_per_call"] > 0 and stats["used_bytes"] > 0


@pytest.mark.parametrize("size", ["small", "mid"])
def test_batch_matches_fp64_oracle(cuda, oracle, size):
    """The stacked gradient of a survey against the FP64 oracle's, within 1e-4.
    The mid-size survey (apertures of 100-180 cells over a 200 x 176 x 96
    model) gives every shot several 64 x 16 tiles and z-chunks, so the
    persistent multi-shot kernels walk many tiles per CTA and carry their
    barrier phases across tiles and shots."""
    from paper_2009_12623_gb300 import api, synth
    if size == "small":
        sv = _survey(seed=3)
    else:
        sv = _survey(nshots=4, seed=4, nx=200, ny=176, nz=96, nbl=10, ap_min=100, ap_max=180, t_min=0.05,
                     t_max=0.08, rec_stride=5, h=12.0)
    g = sv.geom
    og = oracle.geometry(g.nx, g.ny, g.nz, g.h, g.dt, g.nt, g.nbl, g.sponge_R, g.vmax)
    m64 = synth.slowness2(sv.v0).astype(np.float64)
    mt64 = synth.slowness2(sv.v_true).astype(np.float64)
    w = sv.wavelets()
    d_obs = []
    for s, wi in zip(sv.shots, w):
        lg = oracle.geometry(s.nx, s.ny, s.nz, g.h, g.dt, s.nt, g.nbl, g.sponge_R, g.vmax)
        rec = np.asarray(s.rec) - np.array([s.x0, s.y0, s.z0])
        d_obs.append(oracle.forward(lg, mt64[s.window], wi.astype(np.float64),
                                    (s.src[0] - s.x0, s.src[1] - s.y0, s.src[2] - s.z0), rec))
    shots = [(s.x0, s.y0, s.z0, s.nx, s.ny, s.nz, s.nt, s.src) for s in sv.shots]
    g_ref, phi_ref = oracle.gradient_batch(og, m64, shots, [x.astype(np.float64) for x in w],
                                           [s.rec for s in sv.shots], d_obs)
    m = torch.from_numpy(synth.slowness2(sv.v0)).to(cuda)
    with api.Batch(g, sv.shots, mode=2, k=6, atol=0.0, arena_bytes=1 << (29 if size == "small" else 32)) as b:
        gg, phi = b.gradient(m, w, b.concat([d.astype(np.float32) for d in d_obs]))
    gg = gg.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - g_ref) / np.linalg.norm(g_ref) < 1e-4
    assert np.allclose(phi, phi_ref, rtol=1e-4)
    outside = np.ones(g_ref.shape, bool)
    for s in sv.shots:
        outside[s.window] = False
    assert not gg[outside].any()


def test_graph_replay_and_tuning_change_no_bit(cuda):
    from paper_2009_12623_gb300 import api
    sv = _survey(seed=2)
    m, w, d_obs = _setup(cuda, sv)
    with api.Batch(sv.geom, sv.shots, mode=2, k=5, atol=1e-4, arena_bytes=1 << 29) as b:
        obs = b.concat(d_obs)
        g0, p0 = b.gradient(m, w, obs)
    with api.Batch(sv.geom, sv.shots, mode=2, k=5, atol=1e-4, arena_bytes=1 << 29, graph=True, tune=True) as b:
        obs = b.concat(d_obs)
        grads = []
        for _ in range(3):  # capture, then two replays
            grads.append(b.gradient(m, w, obs))
        stats = b.stats()
    for g, p in grads:
        assert torch.equal(g, g0)
        assert np.array_equal(p, p0)
    assert stats["tuned"] == 1 and stats["graph_nodes"] > 0
    assert stats["zc"] >= 0 and stats["ctas"] > 0


def test_forward_adjoint_split_equals_fused(cuda):
    from paper_2009_12623_gb300 import api
    sv = _survey(seed=5)
    m, w, d_obs = _setup(cuda, sv)
    with api.Batch(sv.geom, sv.shots, mode=1, atol=1e-4, arena_bytes=1 << 29) as b:
        obs = b.concat(d_obs)
        g_fused, phi = b.gradient(m, w, obs)
        d = b.forward(m, w)
        g_split = b.adjoint(m, w, (d - obs).contiguous())
        for di, s in zip(b.split(d), sv.shots):
            assert di.shape == (s.nt, len(s.rec))
    assert torch.equal(g_split, g_fused)
    resid = (d - obs).double()
    assert float(0.5 * (resid ** 2).sum()) == pytest.approx(phi.sum(), rel=1e-12)


def test_more_shots_than_one_launch_holds(cuda):
    """35 shots: the multi-shot launches split into groups of at most 32."""
    from paper_2009_12623_gb300 import api
    sv = _survey(nshots=35, seed=7, nx=40, ny=40, nz=20, ap_min=16, ap_max=24, t_min=0.012, t_max=0.02,
                 nbl=4, rec_stride=4)
    m, w, d_obs = _setup(cuda, sv)
    with api.CheckpointStore(1 << 26) as st:
        g_ref, phi_ref = api.gradient_per_shot(sv.geom, m, sv.shots, w, d_obs, st, mode=2, k=3, atol=0.0)
    with api.Batch(sv.geom, sv.shots, mode=2, k=3, atol=0.0, arena_bytes=1 << 28) as b:
        g, phi = b.gradient(m, w, b.concat(d_obs))
    assert torch.equal(g, g_ref)
    assert np.array_equal(phi, phi_ref)


def test_batch_errors(cuda):
    from paper_2009_12623_gb300 import api
    from paper_2009_12623_gb300.api import ShotSpec
    sv = _survey(seed=6)
    m, w, d_obs = _setup(cuda, sv)
    # compressed checkpoints overflowing the arena
    with api.Batch(sv.geom, sv.shots, mode=1, atol=1e-4, arena_bytes=1 << 14) as b:
        with pytest.raises(api.FwiError) as e:
            b.gradient(m, w, b.concat(d_obs))
        assert e.value.status == -2
    # raw checkpoints that cannot fit are refused at creation
    with pytest.raises(api.FwiError) as e:
        api.Batch(sv.geom, sv.shots, mode=1, atol=0.0, arena_bytes=1 << 14)
    assert e.value.status == -2
    # a receiver outside its shot's aperture
    s = sv.shots[0]
    bad = ShotSpec(s.x0, s.y0, s.z0, s.nx, s.ny, s.nz, s.nt, s.src,
                   np.array([[s.x0 + s.nx, s.y0, 3]], np.int32))
    with pytest.raises(api.FwiError) as e:
        api.Batch(sv.geom, [bad], mode=1, atol=0.0, arena_bytes=1 << 26)
    assert e.value.status == -1
    # the adjoint half needs a forward call first
    with api.Batch(sv.geom, sv.shots, mode=2, k=4, atol=0.0, arena_bytes=1 << 28) as b:
        with pytest.raises(api.FwiError):
            b.adjoint(m, w, b.concat(d_obs))


@pytest.mark.parametrize("graph", [False, True])
def test_survey_autograd_equals_batch_gradient(cuda, graph):
    """Autograd over the batch plan (one batched forward, one batched reverse
    sweep) gives the fused stacked gradient bit for bit."""
    from paper_2009_12623_gb300 import api, autograd
    sv = _survey(seed=8)
    m, w, d_obs = _setup(cuda, sv)
    with api.Batch(sv.geom, sv.shots, mode=2, k=4, atol=1e-4, arena_bytes=1 << 29, graph=graph) as b:
        obs = b.concat(d_obs)
        g_ref, phi = b.gradient(m, w, obs)
        for _ in range(2):  # the second pass replays the captured graphs
            mm = m.clone().requires_grad_(True)
            d = autograd.survey(mm, b, w)
            loss = 0.5 * ((d - obs).double() ** 2).sum()
            loss.backward()
            assert torch.equal(mm.grad, g_ref)
            assert float(loss) == pytest.approx(phi.sum(), rel=1e-12)


def test_batched_inversion_tracks_per_shot_inversion(cuda):
    """Steepest descent through the batch plan and through one call per shot
    (full-grid apertures): same first gradient up to FP32 summation order,
    same misfit history."""
    from paper_2009_12623_gb300 import api, invert, synth
    from paper_2009_12623_gb300.api import ShotSpec
    base = _survey(seed=9, nshots=1)
    g = base.geom
    rec = np.array([(i, j, 8) for i in range(6, g.nx - 6, 4) for j in range(6, g.ny - 6, 6)], np.int32)
    nt = 40
    geom = api.Geometry(nx=g.nx, ny=g.ny, nz=g.nz, h=g.h, dt=g.dt, nt=nt, nbl=g.nbl, vmax=g.vmax)
    srcs = [(14, 12, 8), (40, 30, 8), (28, 20, 8)]
    w = synth.wavelet(nt, g.dt, 25.0)
    mt = torch.from_numpy(synth.slowness2(base.v_true)).to(cuda)
    rt = torch.from_numpy(rec).to(cuda)
    d_obs = [api.forward(geom, mt, w, s, rt) for s in srcs]
    c0 = torch.from_numpy(base.v0).to(cuda)
    shots = [(geom, w, s, rt) for s in srcs]
    c1, h1 = invert.invert(c0, shots, d_obs, iters=3, atol=1e-4, step=0.01, store_bytes=1 << 27)
    specs = [ShotSpec(0, 0, 0, g.nx, g.ny, g.nz, nt, s, rec) for s in srcs]
    with api.Batch(geom, specs, mode=1, atol=1e-4, arena_bytes=1 << 28) as plan:
        c2, h2 = invert.invert_batched(c0, plan, [w] * 3, plan.concat(d_obs), iters=3, step=0.01)
    assert np.allclose(h1, h2, rtol=1e-5), (h1, h2)
    assert float(torch.linalg.vector_norm(c1 - c2)) <= 1e-4 * float(torch.linalg.vector_norm(c1 - c0))


def test_stacking_does_not_accumulate_compression_errors(cuda):
    """Sec. 4's stacking observation on the GPU path: the stacked gradient's
    relative error from compressed checkpoints (atol 1e-2) is at most the
    worst single shot's, and the batch plan's stacked gradient has that same
    error (it is bitwise the sum of the per-shot calls)."""
    from paper_2009_12623_gb300 import api
    sv = _survey(seed=11)
    m, w, d_obs = _setup(cuda, sv)

    def per_shot(atol):
        with api.CheckpointStore(1 << 28) as st:
            return [api.gradient_per_shot(sv.geom, m, [s], [wi], [d], st, mode=1, atol=atol)[0]
                    for s, wi, d in zip(sv.shots, w, d_obs)]

    def rel(a, b):
        return float(torch.linalg.vector_norm((a - b).double()) / torch.linalg.vector_norm(b.double()))

    raw, lossy = per_shot(0.0), per_shot(1e-2)
    per = [rel(a, b) for a, b in zip(lossy, raw)]
    stacked = rel(sum(lossy), sum(raw))
    assert 0 < stacked <= max(per), (stacked, per)
    with api.Batch(sv.geom, sv.shots, mode=1, atol=1e-2, arena_bytes=1 << 29) as b:
        g, _ = b.gradient(m, w, b.concat(d_obs))
    assert rel(g, sum(raw)) == pytest.approx(stacked, rel=1e-3)
