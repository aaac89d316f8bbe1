"""GPU forward sweep, checkpointed gradient and reductions vs the FP64 oracle
(Sec. 2 Eq. (2)-(4); Sec. 1.3-1.4).  Tolerance: FP32 fields within 1e-4
relative L2 of the FP64 oracle."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
TOL = 1e-4


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _og(oracle, g):
    return oracle.geometry(g.nx, g.ny, g.nz, g.h, g.dt, g.nt, g.nbl, g.sponge_R, g.vmax)


def _small_shot(nx=37, ny=29, nz=23, nt=80, nbl=5):
    from paper_2009_12623_gb300 import synth
    from paper_2009_12623_gb300.api import Geometry
    rng = np.random.default_rng(11)
    z = np.arange(nz)[:, None, None]
    v0 = (np.where(z < nz // 2, 1500.0, 2300.0) * np.ones((nz, ny, nx))).astype(np.float32)
    vt = (v0 * (1 + 0.05 * rng.uniform(-1, 1, v0.shape))).astype(np.float32)
    rec = np.array([(i, ny // 2, 3) for i in range(0, nx, 3)] + [(nx - 1, ny - 1, nz - 1)], np.int32)
    g = Geometry(nx=nx, ny=ny, nz=nz, h=10.0, dt=1e-3, nt=nt, nbl=nbl, vmax=2500.0)
    return synth.Shot("small", g, 25.0, (nx // 3, ny // 2, 4), rec, vt, v0)


@pytest.fixture(scope="module")
def two_layer(oracle):
    """The plain-gradient case (64^3, 200 steps of 1 ms).  Within 0.2 s no
    wave scattered by the centre blob reaches the z=4 receivers, so data of the
    specified true model differ from the two-layer data only below FP32
    resolution; gradient parity therefore uses d_obs = 0 (Phi = 1/2 |d_sim|^2),
    which drives the same sweeps with a residual of full size."""
    from paper_2009_12623_gb300 import synth
    shot = synth.two_layer_shot()
    return shot, np.zeros((shot.geom.nt, len(shot.rec)))


def phi_tol(d_sim, resid):
    # Phi changes by <r, dd> for a data change dd; |dd| <= TOL |d_sim| in FP32
    return 2 * TOL * np.linalg.norm(d_sim) * np.linalg.norm(resid) + 1e-30


def _dev(cuda, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(cuda)


@pytest.mark.parametrize("which", ["two_layer", "ragged"])
def test_forward_records_match_oracle(cuda, oracle, two_layer, which):
    from paper_2009_12623_gb300 import api, synth
    shot = two_layer[0] if which == "two_layer" else _small_shot()
    m = synth.slowness2(shot.v0)
    ref, ub, ul = oracle.forward(_og(oracle, shot.geom), m.astype(np.float64), shot.wavelet.astype(np.float64),
                                 shot.src, shot.rec, return_state=True)
    d, up, ulast = api.forward(shot.geom, _dev(cuda, m), shot.wavelet, shot.src, _dev(cuda, shot.rec),
                               return_state=True)
    assert rel(d.cpu().numpy(), ref) < TOL
    assert rel(ulast.cpu().numpy(), ul) < TOL
    assert rel(up.cpu().numpy(), ub) < TOL


def test_forward_from_state(cuda, oracle):
    from paper_2009_12623_gb300 import api, synth
    shot = _small_shot(nt=15)
    rng = np.random.default_rng(3)
    u0 = rng.normal(size=shot.geom.shape).astype(np.float32)
    u1 = rng.normal(size=shot.geom.shape).astype(np.float32)
    m = synth.slowness2(shot.v0)
    ref, _, ul = oracle.forward(_og(oracle, shot.geom), m.astype(np.float64), shot.wavelet.astype(np.float64),
                                shot.src, shot.rec, u_prev_init=u0.astype(np.float64),
                                u_cur_init=u1.astype(np.float64), return_state=True)
    d, _, ulast = api.forward(shot.geom, _dev(cuda, m), shot.wavelet, shot.src, _dev(cuda, shot.rec),
                              u_prev_init=_dev(cuda, u0), u_cur_init=_dev(cuda, u1), return_state=True)
    assert rel(ulast.cpu().numpy(), ul) < TOL
    assert rel(d.cpu().numpy(), ref) < TOL


def _grad(cuda, shot, d_obs, mode, k=1, atol=0.0, cap=1 << 30):
    from paper_2009_12623_gb300 import api, synth
    m = synth.slowness2(shot.v0)
    with api.CheckpointStore(cap) as st:
        g, phi = api.gradient(shot.geom, _dev(cuda, m), shot.wavelet, shot.src, _dev(cuda, shot.rec),
                              _dev(cuda, np.asarray(d_obs, np.float32)), st, mode=mode, k=k, atol=atol)
        stats = st.stats()
    return g.cpu().numpy(), phi, stats


def test_gradient_raw_matches_oracle(cuda, oracle, two_layer):
    from paper_2009_12623_gb300 import synth
    shot, d_obs = two_layer
    og = _og(oracle, shot.geom)
    gref, phiref, dsim, _ = oracle.gradient(og, synth.slowness2(shot.v0).astype(np.float64),
                                            shot.wavelet.astype(np.float64), shot.src, shot.rec, d_obs)
    g, phi, _ = _grad(cuda, shot, d_obs, 1)
    assert rel(g, gref) < TOL
    assert abs(phi - phiref) <= phi_tol(dsim, dsim - d_obs)


def test_specified_true_model_residual_is_below_fp32_resolution(cuda, oracle):
    """The true-model data of the plain-gradient case match the two-layer data
    to within the FP32 tolerance, on both sides."""
    from paper_2009_12623_gb300 import api, synth
    shot = synth.two_layer_shot()
    og = _og(oracle, shot.geom)
    w = shot.wavelet.astype(np.float64)
    d_true = oracle.forward(og, synth.slowness2(shot.v_true).astype(np.float64), w, shot.src, shot.rec)
    d0 = oracle.forward(og, synth.slowness2(shot.v0).astype(np.float64), w, shot.src, shot.rec)
    assert rel(d0, d_true) < 1e-5
    d_gpu = api.forward(shot.geom, _dev(cuda, synth.slowness2(shot.v0)), shot.wavelet, shot.src,
                        _dev(cuda, shot.rec)).cpu().numpy()
    assert rel(d_gpu, d_true) < TOL


def test_gradient_ragged_every_k(cuda, oracle):
    from paper_2009_12623_gb300 import synth
    shot = _small_shot()
    og = _og(oracle, shot.geom)
    d_obs = oracle.forward(og, synth.slowness2(shot.v_true).astype(np.float64), shot.wavelet.astype(np.float64),
                           shot.src, shot.rec)
    gref, phiref, dsim, _ = oracle.gradient(og, synth.slowness2(shot.v0).astype(np.float64),
                                            shot.wavelet.astype(np.float64), shot.src, shot.rec, d_obs)
    g, phi, _ = _grad(cuda, shot, d_obs, 2, k=7)
    assert rel(g, gref) < TOL
    assert abs(phi - phiref) <= phi_tol(dsim, dsim - d_obs)


@pytest.mark.parametrize("snaps", [1, 3, 8])
def test_binomial_raw_bitwise_equals_full_history(cuda, two_layer, snaps):
    """Binomial (Revolve-family) checkpointing with raw pairs is bitwise exact."""
    shot, d_obs = two_layer
    g_full, phi_full, _ = _grad(cuda, shot, d_obs, 1)
    g_b, phi_b, stats = _grad(cuda, shot, d_obs, 3, k=snaps)
    assert np.array_equal(g_full, g_b) and phi_full == phi_b
    assert stats["n_checkpoints"] == 2 * snaps


def test_binomial_compressed_tracks_oracle(cuda, oracle):
    from paper_2009_12623_gb300 import synth
    shot = _small_shot()
    og = _og(oracle, shot.geom)
    m = synth.slowness2(shot.v0).astype(np.float64)
    w = shot.wavelet.astype(np.float64)
    d_obs = oracle.forward(og, synth.slowness2(shot.v_true).astype(np.float64), w, shot.src, shot.rec)
    g_raw, phi_raw, *_ = oracle.gradient(og, m, w, shot.src, shot.rec, d_obs)
    g_oz, *_ = oracle.gradient(og, m, w, shot.src, shot.rec, d_obs, mode=3, k=4, atol=1e-4)
    g_graw, *_ = _grad(cuda, shot, d_obs, 3, k=4)
    g_gz, phi_gz, stats = _grad(cuda, shot, d_obs, 3, k=4, atol=1e-4)
    _same_compression_error(g_gz, g_graw, g_oz, g_raw)
    assert stats["used_bytes"] < stats["raw_bytes"] / 2


def test_subsampling_matches_oracle(cuda, oracle):
    """Subsampled imaging (Sec. 4.7) on the GPU: f = 1 is bitwise full history,
    f = 4 follows the FP64 oracle's subsampled gradient."""
    from paper_2009_12623_gb300 import synth
    shot = _small_shot()
    og = _og(oracle, shot.geom)
    m = synth.slowness2(shot.v0).astype(np.float64)
    w = shot.wavelet.astype(np.float64)
    d_obs = oracle.forward(og, synth.slowness2(shot.v_true).astype(np.float64), w, shot.src, shot.rec)
    g_full, *_ = _grad(cuda, shot, d_obs, 1)
    g_s1, *_ = _grad(cuda, shot, d_obs, 4, k=1)
    assert np.array_equal(g_full, g_s1)
    g_o4, *_ = oracle.gradient(og, m, w, shot.src, shot.rec, d_obs, mode=4, k=4)
    g_g4, _, stats = _grad(cuda, shot, d_obs, 4, k=4)
    assert rel(g_g4, g_o4) < TOL
    assert stats["n_checkpoints"] == shot.geom.nt // 4


@pytest.mark.parametrize("k", [1, 4, 10, 33, 500])
def test_every_k_raw_bitwise_equals_full_history(cuda, two_layer, k):
    """Checkpointing alone is bitwise exact (Sec. 1.3) on the GPU too."""
    shot, d_obs = two_layer
    g_full, phi_full, _ = _grad(cuda, shot, d_obs, 1)
    g_k, phi_k, _ = _grad(cuda, shot, d_obs, 2, k=k)
    assert np.array_equal(g_full, g_k) and phi_full == phi_k


def _same_compression_error(g_gz, g_graw, g_oz, g_oraw):
    """Both sides compress their own (FP32 vs FP64-rounded) checkpoints, so
    their lossy gradients are two draws of the compression error, not the
    same numbers.  Each side's error is measured against its own raw-
    checkpoint gradient, which removes the FP32-vs-FP64 floor (about 1e-6
    here, above the errors being compared), and the two must agree within a
    factor of two either way."""
    e_o, e_g = rel(g_oz, g_oraw), rel(g_gz, g_graw)
    print(f"compression error: GPU {e_g:.3e}, oracle {e_o:.3e}, ratio {e_g / e_o:.3f}")
    assert 0.5 <= e_g / e_o <= 2.0, (e_g, e_o)
    assert rel(g_graw, g_oraw) < TOL


def test_compressed_gradient_tracks_oracle(cuda, oracle, two_layer):
    """Plain checkpointed gradient: every 10 steps, atol = 1e-4; the GPU's
    compression error matches the oracle's (two-sided, no additive slack)."""
    from paper_2009_12623_gb300 import synth
    shot, d_obs = two_layer
    og = _og(oracle, shot.geom)
    m = synth.slowness2(shot.v0).astype(np.float64)
    w = shot.wavelet.astype(np.float64)
    g_raw, *_ = oracle.gradient(og, m, w, shot.src, shot.rec, d_obs)
    g_oz, *_ = oracle.gradient(og, m, w, shot.src, shot.rec, d_obs, mode=2, k=10, atol=1e-4)
    g_graw, *_ = _grad(cuda, shot, d_obs, 2, k=10)
    g_gz, _, stats = _grad(cuda, shot, d_obs, 2, k=10, atol=1e-4)
    _same_compression_error(g_gz, g_graw, g_oz, g_raw)
    assert stats["used_bytes"] < stats["raw_bytes"]


@pytest.mark.parametrize("atol", [1e-6, 1e-9])
def test_compressed_full_history_converges(cuda, oracle, two_layer, atol):
    from paper_2009_12623_gb300 import synth
    shot, d_obs = two_layer
    og = _og(oracle, shot.geom)
    g_raw, *_ = oracle.gradient(og, synth.slowness2(shot.v0).astype(np.float64),
                                shot.wavelet.astype(np.float64), shot.src, shot.rec, d_obs)
    g, _, stats = _grad(cuda, shot, d_obs, 1, atol=atol)
    assert rel(g, g_raw) < (1e-3 if atol > 1e-8 else TOL)
    assert not stats["overflowed"]


def test_capacity_overflow_reported(cuda, two_layer):
    from paper_2009_12623_gb300 import api, synth, _lib
    shot, d_obs = two_layer
    m = synth.slowness2(shot.v0)
    grad = torch.zeros(shot.geom.shape, device=cuda)
    for atol in (0.0, 1e-4):
        with api.CheckpointStore(1 << 20) as st:
            with pytest.raises(api.FwiError) as e:
                api.gradient(shot.geom, _dev(cuda, m), shot.wavelet, shot.src, _dev(cuda, shot.rec),
                             _dev(cuda, d_obs.astype(np.float32)), st, mode=1, atol=atol, grad=grad)
            assert e.value.status == _lib.FWI_ERR_CAPACITY
            s = st.stats()
            assert s["overflowed"] and s["used_bytes"] > (1 << 20)
    assert float(grad.abs().max()) == 0.0


@pytest.mark.parametrize("mode,k", [(1, 1), (2, 10), (3, 4)])
def test_gradient_host_equals_device(cuda, two_layer, mode, k):
    """The host-memory entry point (uploads overlapped with the forward sweep,
    then misfit and reverse sweep) gives the device call's bits."""
    from paper_2009_12623_gb300 import api, synth
    shot, d_obs = two_layer
    g_dev, phi_dev, _ = _grad(cuda, shot, d_obs, mode, k=k, atol=1e-4)
    with api.CheckpointStore(1 << 30) as st:
        g_host, phi_host = api.gradient_host(shot.geom, synth.slowness2(shot.v0), shot.wavelet, shot.src,
                                             shot.rec, d_obs.astype(np.float32), st, mode=mode, k=k,
                                             atol=1e-4)
    assert np.array_equal(g_host, g_dev) and phi_host == phi_dev


def test_misfit_and_dot_f64(cuda):
    from paper_2009_12623_gb300 import api
    rng = np.random.default_rng(0)
    a = rng.normal(size=100003).astype(np.float32)
    b = rng.normal(size=100003).astype(np.float32)
    r, phi = api.misfit(_dev(cuda, a), _dev(cuda, b))
    d = a.astype(np.float64) - b
    assert np.array_equal(r.cpu().numpy(), a - b)
    assert phi == pytest.approx(0.5 * np.sum((a - b).astype(np.float64) ** 2), rel=1e-12)
    assert api.dot_f64(_dev(cuda, a), _dev(cuda, b)) == pytest.approx(np.dot(a.astype(np.float64), b), rel=1e-12)
    del d


def test_bad_receiver_rejected(cuda):
    from paper_2009_12623_gb300 import api, synth
    shot = _small_shot(nt=3)
    rec = shot.rec.copy()
    rec[0, 0] = shot.geom.nx + 5
    with pytest.raises(api.FwiError):
        api.forward(shot.geom, _dev(cuda, synth.slowness2(shot.v0)), shot.wavelet, shot.src, _dev(cuda, rec))


def test_bounded_wait_times_out_and_context_survives(cuda, two_layer):
    """A device wait that nothing completes gives up, reports FWI_ERR_TIMEOUT,
    and the next call on the same context works."""
    import time
    from paper_2009_12623_gb300 import _lib, api
    t0 = time.time()
    assert api.selftest_bounded_wait(2000) == _lib.FWI_ERR_TIMEOUT
    assert time.time() - t0 < 30.0
    shot, d_obs = two_layer
    g, phi, _ = _grad(cuda, shot, d_obs, 2, k=10)
    assert np.isfinite(g).all() and phi > 0


def test_damped_quotient_within_one_ulp_of_ieee_division(cuda):
    """The stencil kernels divide by the damping factor 1 + eta with a
    reciprocal estimate, one Newton-Raphson step and a remainder correction
    instead of IEEE division.  Against CUDA's correctly rounded division, on
    divisors over [1, 2) (the layer's range and beyond) and up to 1e30, with
    numerators spanning zero, subnormal and huge magnitudes: never more than
    1 ulp apart, and equal in all but a tiny fraction of cases."""
    from paper_2009_12623_gb300 import api
    g = torch.Generator().manual_seed(11)
    n = 1 << 22
    num = torch.randn(n, generator=g) * torch.exp(6 * torch.randn(n, generator=g))
    num[:1024] = 0.0
    num[1024:2048] = torch.randn(1024, generator=g) * 1e-40   # subnormal
    num[2048:3072] = torch.randn(1024, generator=g) * 1e37
    den = 1.0 + torch.rand(n, generator=g)
    den[:4096] = 1.0
    den[4096:8192] = torch.exp(torch.rand(4096, generator=g) * 69.0)  # up to ~1e30
    num, den = num.float().to(cuda), den.float().to(cuda)
    got = api.selftest_damped_quotient(num, den)
    ref = num / den
    assert torch.isfinite(got).all()
    gi, ri = got.view(torch.int32).long(), ref.view(torch.int32).long()
    same_sign = (got >= 0) == (ref >= 0)
    ulps = torch.where(same_sign, (gi - ri).abs(), gi.abs() + ri.abs())
    assert int(ulps.max()) <= 1
    assert float((ulps == 0).double().mean()) > 0.999


def test_lossy_restart_propagation_matches_oracle(cuda, oracle):
    """The restart experiment of Sec. 4 on the GPU path (FP32 steps through
    fwi_forward, the GPU codec): the difference between the runs continued
    from the exact and from the lossy state pair follows the oracle's curve
    step by step and has its shape (sharp rise, then decay, bounded)."""
    from paper_2009_12623_gb300 import api, synth
    from test_oracle_restart import STEPS, T1, restart_curve
    atol = 1e-4  # well above the FP32 rounding of two runs that differ only in their start
    shot = synth.two_layer_shot(n=48, nt=T1 + STEPS, h=10.0, dt=1e-3, nbl=8, f=25.0)
    g = shot.geom
    m = torch.from_numpy(synth.slowness2(shot.v0)).to(cuda)
    rec = torch.from_numpy(shot.rec).to(cuda)
    g1 = api.Geometry(**{**g.__dict__, "nt": T1})
    _, up, uc = api.forward(g1, m, shot.wavelet[:T1], shot.src, rec, return_state=True)
    exact = [up, uc]
    lossy = [api.zfp_decompress(api.zfp_compress(f, atol), f.shape) for f in exact]
    e0 = float((lossy[1] - exact[1]).abs().max())
    one = api.Geometry(**{**g.__dict__, "nt": 1})
    linf, l2 = [], []
    for i in range(STEPS):
        wi = shot.wavelet[T1 + i:T1 + i + 1]
        _, a0, a1 = api.forward(one, m, wi, shot.src, rec, u_prev_init=exact[0], u_cur_init=exact[1],
                                return_state=True)
        _, b0, b1 = api.forward(one, m, wi, shot.src, rec, u_prev_init=lossy[0], u_cur_init=lossy[1],
                                return_state=True)
        exact, lossy = [a0, a1], [b0, b1]
        d = (a1 - b1).double()
        linf.append(float(d.abs().max()))
        l2.append(float(torch.linalg.vector_norm(d)))
    linf, l2 = np.array(linf), np.array(l2)
    o_linf, o_l2, o_e0 = restart_curve(oracle, atol)
    assert 0 < e0 <= atol and 0 < o_e0 <= atol  # the codec's bound at the restart
    # step by step within 10%: the curves start within 0.3% and drift apart as the FP32 rounding
    # of the two GPU runs (which differ only in their start) adds to their difference
    assert np.all(np.abs(l2 - o_l2) <= 0.10 * o_l2), np.max(np.abs(l2 - o_l2) / o_l2)
    assert abs(l2[0] - o_l2[0]) <= 0.01 * o_l2[0]
    k = int(np.argmax(l2))
    assert 1 <= k <= 30 and l2[k] > 1.5 * l2[0]
    assert l2[-1] < 0.8 * l2[k]
    assert linf.max() <= 2 * atol


def test_slot_bytes_report_each_checkpoint(cuda, two_layer):
    """fwi_ckpt_store_slot_bytes: one entry per stored state, consistent with
    the store's totals; compressed states grow as the wave spreads through
    the grid (the compressibility trend of Sec. 4.1); raw and every-K stores
    report field sizes and pair slots."""
    from paper_2009_12623_gb300 import api, synth
    shot, d_obs = two_layer
    g = shot.geom
    m = _dev(cuda, synth.slowness2(shot.v0))
    rec = _dev(cuda, shot.rec)
    obs = _dev(cuda, np.asarray(d_obs, np.float32))
    field = g.nx * g.ny * g.nz * 4
    with api.CheckpointStore(1 << 30) as st:
        assert st.slot_bytes().size == 0
        api.gradient(g, m, shot.wavelet, shot.src, rec, obs, st, mode=api.FWI_CKPT_FULL, atol=1e-4)
        b = st.slot_bytes().astype(np.int64)
        s = st.stats()
        assert b.size == g.nt == s["n_checkpoints"]
        assert np.all(b > 0) and np.all(b <= field + 4096)
        assert b.sum() <= s["used_bytes"] <= b.sum() + 256 * b.size
        q = g.nt // 5
        assert b[:q].mean() < b[-q:].mean()
        api.gradient(g, m, shot.wavelet, shot.src, rec, obs, st, mode=api.FWI_CKPT_FULL, atol=0.0)
        assert np.all(st.slot_bytes() == field)
        api.gradient(g, m, shot.wavelet, shot.src, rec, obs, st, mode=api.FWI_CKPT_EVERY_K, k=10, atol=1e-4)
        b10 = st.slot_bytes()
        assert b10.size == st.stats()["n_checkpoints"] and b10.size % 2 == 0 and b10.size <= 2 * (g.nt // 10 + 1)


@pytest.mark.parametrize("which,atol", [("two_layer", 1e-4), ("two_layer", 1e-2), ("ragged", 1e-5),
                                        ("mid", 1e-4)])
def test_zero_block_skipping_is_exact(cuda, two_layer, which, atol):
    """Blocks a state codes as zero are skipped on both sides of the full-history
    sweep: the forward step marks the blocks that reach the tolerance's last
    coded plane and the encoder codes the others as zero unread; the reverse
    sweep leaves them undecoded and skips u^k and g there (the imaging term is
    exactly 0).  Every-1 checkpoint pairs read and decode every block, so the
    two gradients must agree bit for bit.  The early states of these shots are
    mostly zero blocks; the mid-size grid (ragged in every direction) runs the
    forward step in several z-chunks per tile column."""
    from paper_2009_12623_gb300 import synth
    if which == "two_layer":
        shot, d_obs = two_layer
    else:
        shot = _small_shot() if which == "ragged" else _small_shot(nx=161, ny=122, nz=150, nt=70, nbl=8)
        d_obs = np.zeros((shot.geom.nt, len(shot.rec)))
    g_full, phi_full, _ = _grad(cuda, shot, d_obs, 1, atol=atol)
    g_k1, phi_k1, _ = _grad(cuda, shot, d_obs, 2, k=1, atol=atol)
    assert np.array_equal(g_full.view(np.uint32), g_k1.view(np.uint32)) and phi_full == phi_k1


def test_slot_zero_blocks_match_the_oracle_streams(cuda, oracle, two_layer):
    """fwi_ckpt_store_slot_zero_blocks: per stored state, the blocks coded as
    the single bit 0, equal to the count in the oracle's stream of the same
    FP32 state (read from its u16 length table); raw stores report 0."""
    import struct
    from paper_2009_12623_gb300 import api, synth
    shot, d_obs = two_layer
    g = shot.geom
    m = _dev(cuda, synth.slowness2(shot.v0))
    rec = _dev(cuda, shot.rec)
    obs = _dev(cuda, np.asarray(d_obs, np.float32))
    atol = 1e-4
    with api.CheckpointStore(1 << 30) as st:
        api.gradient(g, m, shot.wavelet, shot.src, rec, obs, st, mode=api.FWI_CKPT_FULL, atol=atol)
        z = st.slot_zero_blocks().astype(np.int64)
        assert z.size == g.nt
        for k in (1, 20, 90, g.nt):
            gk = api.Geometry(**{**g.__dict__, "nt": k})
            _, _, uk = api.forward(gk, m, shot.wavelet[:k], shot.src, rec, return_state=True)
            s = oracle.zfp_compress(uk.cpu().numpy(), atol)
            nblocks, = struct.unpack_from("<Q", s, 24)
            nchunks, = struct.unpack_from("<I", s, 36)
            lens = np.frombuffer(s, np.uint16, nblocks, 64 + 8 * nchunks)
            assert z[k - 1] == int((lens == 1).sum()), k
        assert z[0] > z[-1] > 0
        api.gradient(g, m, shot.wavelet, shot.src, rec, obs, st, mode=api.FWI_CKPT_FULL, atol=0.0)
        assert np.all(st.slot_zero_blocks() == 0)


@pytest.mark.parametrize("atol", [1e-4, 1e-2])
def test_nonfinite_wavefield_is_reported_not_skipped(cuda, atol):
    """The forward step's block-liveness map counts NaN and Inf as live, so a
    non-finite state still reaches the encoder and the full-history
    compressed gradient fails with FWI_ERR_NONFINITE instead of coding the
    block as zero; the caller's gradient is left untouched.  The model is
    finite and positive (setup accepts it) but one cell's tiny squared
    slowness makes the leapfrog step there unstable: the wavefield
    overflows to Inf and NaN within a few steps of the wave's arrival."""
    from paper_2009_12623_gb300 import _lib, api, synth
    shot = _small_shot(nt=30)
    m = synth.slowness2(shot.v0).copy()
    m[12, 14, 10] = 1e-30
    d_obs = torch.zeros((shot.geom.nt, len(shot.rec)), device=cuda)
    grad = torch.full(shot.geom.shape, 7.0, device=cuda)
    with api.CheckpointStore(1 << 28) as st:
        with pytest.raises(api.FwiError) as e:
            api.gradient(shot.geom, _dev(cuda, m), shot.wavelet, shot.src, _dev(cuda, shot.rec), d_obs, st,
                         mode=api.FWI_CKPT_FULL, atol=atol, grad=grad)
    assert e.value.status == _lib.FWI_ERR_NONFINITE
    assert bool((grad == 7.0).all())


def test_subsampling_compressed_tracks_oracle(cuda, oracle):
    """Subsampled imaging (Sec. 4.7) with compressed states: every f-th state
    stored at atol, the reverse sweep alternating plain adjoint steps with
    imaging ones (decoded and imaged by the decoder).  The GPU's compression
    error against its own raw subsampled gradient matches the oracle's."""
    from paper_2009_12623_gb300 import synth
    shot = _small_shot()
    og = _og(oracle, shot.geom)
    m = synth.slowness2(shot.v0).astype(np.float64)
    w = shot.wavelet.astype(np.float64)
    d_obs = oracle.forward(og, synth.slowness2(shot.v_true).astype(np.float64), w, shot.src, shot.rec)
    g_oraw, *_ = oracle.gradient(og, m, w, shot.src, shot.rec, d_obs, mode=4, k=3)
    g_oz, *_ = oracle.gradient(og, m, w, shot.src, shot.rec, d_obs, mode=4, k=3, atol=1e-4)
    g_graw, *_ = _grad(cuda, shot, d_obs, 4, k=3)
    g_gz, _, stats = _grad(cuda, shot, d_obs, 4, k=3, atol=1e-4)
    _same_compression_error(g_gz, g_graw, g_oz, g_oraw)
    assert stats["n_checkpoints"] == shot.geom.nt // 3
