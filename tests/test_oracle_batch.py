"""Pins of the oracle's stacked survey gradient (Sec. 2: the misfit of a
survey is the sum of the shots' misfits, Eq. (3), so its gradient is the sum
of the shots' Eq. (4); every shot lives on its own aperture of the model).
The pins do not restate the windowing: a full-grid shot must equal the
single-shot gradient, a translated shot in a homogeneous model must give the
translated gradient, a finite-difference derivative of the total misfit
(with windows cut here by numpy) must match, and shot order must not matter."""
import numpy as np
import pytest

from paper_2009_12623_gb300 import synth
from paper_2009_12623_gb300.api import ShotSpec


def _survey(seed=1, nshots=5):
    return synth.batch_survey(nx=44, ny=40, nz=22, nshots=nshots, h=10.0, dt=1e-3, f=25.0, nbl=5,
                              ap_min=18, ap_max=30, t_min=0.025, t_max=0.045, rec_stride=3, seed=seed,
                              vmax=3000.0)


def _obs(oracle, sv, m, m0=None):
    """Records of every shot, each modelled on the numpy-cut window of m (the
    layer's damping weighted by m0, default m)."""
    g = sv.geom
    out = []
    for s, w in zip(sv.shots, sv.wavelets()):
        lg = oracle.geometry(s.nx, s.ny, s.nz, g.h, g.dt, s.nt, g.nbl, g.sponge_R, g.vmax)
        rec = np.asarray(s.rec) - np.array([s.x0, s.y0, s.z0])
        src = (s.src[0] - s.x0, s.src[1] - s.y0, s.src[2] - s.z0)
        out.append(oracle.forward(lg, m[s.window], w, src, rec, m0=None if m0 is None else m0[s.window]))
    return out


def _tuples(shots):
    return [(s.x0, s.y0, s.z0, s.nx, s.ny, s.nz, s.nt, s.src) for s in shots]


def test_full_grid_shot_equals_single_shot_gradient(oracle):
    g = synth.two_layer_shot(n=24, nt=40, nbl=5, f=25.0)
    og = oracle.geometry(24, 24, 24, g.geom.h, g.geom.dt, 40, 5, g.geom.sponge_R, g.geom.vmax)
    m = synth.slowness2(g.v0).astype(np.float64)
    mt = synth.slowness2(g.v_true).astype(np.float64)
    w = g.wavelet.astype(np.float64)
    d_obs = oracle.forward(og, mt, w, g.src, g.rec)
    g_ref, phi_ref, *_ = oracle.gradient(og, m, w, g.src, g.rec, d_obs)
    shot = (0, 0, 0, 24, 24, 24, 40, g.src)
    gb, phib = oracle.gradient_batch(og, m, [shot], [w], [g.rec], [d_obs])
    assert np.array_equal(gb, g_ref)
    assert phib[0] == phi_ref


def test_translated_shot_gives_translated_gradient(oracle):
    """In a homogeneous model a shot whose aperture, source and receivers move
    by (dx, dy) has a gradient moved by (dx, dy), and nothing outside its
    aperture; a transposed or misplaced window breaks this."""
    nx, ny, nz, nt = 40, 34, 20, 30
    og = oracle.geometry(nx, ny, nz, 10.0, 1e-3, nt, 5, 1e-3, 2000.0)
    m = np.full((nz, ny, nx), 1.0 / 2000.0 ** 2)
    w = synth.wavelet(nt, 1e-3, 25.0).astype(np.float64)
    rng = np.random.default_rng(3)
    rec0 = np.array([(i, j, 4) for i in range(2, 20, 3) for j in (3, 11)], np.int32)
    d = rng.normal(size=(nt, len(rec0))) * 1e-3
    a = (0, 0, 0, 22, 16, nz, nt, (9, 7, 5))
    dx, dy = 13, 11
    b = (dx, dy, 0, 22, 16, nz, nt, (9 + dx, 7 + dy, 5))
    ga, pa = oracle.gradient_batch(og, m, [a], [w], [rec0], [d])
    gb, pb = oracle.gradient_batch(og, m, [b], [w], [rec0 + np.array([dx, dy, 0], np.int32)], [d])
    assert pa[0] == pb[0]
    assert np.abs(ga).max() > 0
    assert np.array_equal(gb[:, dy:dy + 16, dx:dx + 22], ga[:, :16, :22])
    mask = np.ones_like(gb, bool)
    mask[:, dy:dy + 16, dx:dx + 22] = False
    assert not gb[mask].any()


def test_stacked_gradient_matches_finite_difference(oracle):
    sv = _survey()
    g = sv.geom
    og = oracle.geometry(g.nx, g.ny, g.nz, g.h, g.dt, g.nt, g.nbl, g.sponge_R, g.vmax)
    m = synth.slowness2(sv.v0).astype(np.float64)
    d_obs = _obs(oracle, sv, synth.slowness2(sv.v_true).astype(np.float64))
    grad, phis = oracle.gradient_batch(og, m, _tuples(sv.shots), sv.wavelets(), [s.rec for s in sv.shots], d_obs)

    def total(mm):  # the gradient holds the layer's damping at m fixed
        return sum(0.5 * np.sum((d - o) ** 2) for d, o in zip(_obs(oracle, sv, mm, m0=m), d_obs))

    assert total(m) == pytest.approx(phis.sum(), rel=1e-12)
    rng = np.random.default_rng(5)
    dm = rng.normal(size=m.shape) * 0.01 * m.mean()
    eps = 1e-5
    fd = (total(m + eps * dm) - total(m - eps * dm)) / (2 * eps)
    assert fd == pytest.approx(float(np.sum(grad * dm)), rel=2e-6)


def test_shot_order_does_not_matter(oracle):
    sv = _survey(seed=2, nshots=4)
    g = sv.geom
    og = oracle.geometry(g.nx, g.ny, g.nz, g.h, g.dt, g.nt, g.nbl, g.sponge_R, g.vmax)
    m = synth.slowness2(sv.v0).astype(np.float64)
    d_obs = _obs(oracle, sv, synth.slowness2(sv.v_true).astype(np.float64))
    w = sv.wavelets()
    recs = [s.rec for s in sv.shots]
    g1, p1 = oracle.gradient_batch(og, m, _tuples(sv.shots), w, recs, d_obs)
    r = list(reversed(range(len(sv.shots))))
    g2, p2 = oracle.gradient_batch(og, m, _tuples([sv.shots[i] for i in r]), [w[i] for i in r],
                                   [recs[i] for i in r], [d_obs[i] for i in r])
    assert np.array_equal(p2, p1[r])
    assert np.linalg.norm(g2 - g1) <= 1e-13 * np.linalg.norm(g1)


def test_every_k_raw_stack_equals_full_history(oracle):
    sv = _survey(seed=4, nshots=3)
    g = sv.geom
    og = oracle.geometry(g.nx, g.ny, g.nz, g.h, g.dt, g.nt, g.nbl, g.sponge_R, g.vmax)
    m = synth.slowness2(sv.v0).astype(np.float64)
    d_obs = _obs(oracle, sv, synth.slowness2(sv.v_true).astype(np.float64))
    args = (og, m, _tuples(sv.shots), sv.wavelets(), [s.rec for s in sv.shots], d_obs)
    g1, p1 = oracle.gradient_batch(*args)
    g2, p2 = oracle.gradient_batch(*args, mode=oracle.CKPT_EVERY_K, k=7)
    assert np.array_equal(g1, g2) and np.array_equal(p1, p2)


def test_batch_rejects_window_outside_grid(oracle):
    og = oracle.geometry(20, 20, 20, 10.0, 1e-3, 5, 2, 1e-3, 2000.0)
    m = np.full((20, 20, 20), 1.0 / 2000.0 ** 2)
    w = np.zeros(5)
    with pytest.raises(RuntimeError):
        oracle.gradient_batch(og, m, [(10, 0, 0, 12, 10, 20, 5, (12, 2, 2))], [w], [np.zeros((0, 3), np.int32)],
                              [np.zeros((5, 0))])


def test_survey_generator_shapes():
    sv = _survey(nshots=8)
    for s in sv.shots:
        assert 0 <= s.x0 and s.x0 + s.nx <= sv.geom.nx and 0 <= s.y0 and s.y0 + s.ny <= sv.geom.ny
        assert s.x0 <= s.src[0] < s.x0 + s.nx and s.y0 <= s.src[1] < s.y0 + s.ny
        r = np.asarray(s.rec)
        assert (r[:, 0] >= s.x0).all() and (r[:, 0] < s.x0 + s.nx).all()
        assert (r[:, 1] >= s.y0).all() and (r[:, 1] < s.y0 + s.ny).all()
    assert isinstance(sv.shots[0], ShotSpec)
