"""Pins of the oracle's adjoint sweep, gradient and checkpoint schedules
(Sec. 2 Eq. (2)-(4); Sec. 1.3 -- checkpointing alone is bitwise exact)."""
import numpy as np
import pytest

N = 22
NT = 70
H = 10.0
DT = 1e-3


def _case(oracle, nbl=5, nt=NT, seed=0):
    from paper_2009_12623_gb300 import synth
    rng = np.random.default_rng(seed)
    g = oracle.geometry(N, N - 2, N + 1, H, DT, nt, nbl, 1e-3, 3000.0)
    z = np.arange(N + 1)[:, None, None]
    v = np.where(z < 10, 1500.0, 2400.0) * np.ones((N + 1, N - 2, N))
    v *= 1.0 + 0.05 * rng.uniform(-1, 1, size=v.shape)
    m = 1.0 / v ** 2
    q = synth.wavelet(nt, DT, 25.0).astype(np.float64)
    src = (11, 9, 6)
    rec = np.array([(i, 10, 4) for i in range(3, 19, 2)] + [(7, 4, 15)], dtype=np.int32)
    return g, m, q, src, rec


def test_dot_product_adjoint(oracle):
    """<F q, d> = <q, F^T d> with F: q -> P_r A^-1 P_s^T q (random q, d)."""
    rng = np.random.default_rng(1)
    g, m, _, src, rec = _case(oracle)
    q = rng.normal(size=NT)
    d = rng.normal(size=(NT, len(rec)))
    Fq = oracle.forward(g, m, q, src, rec)
    Ftd = oracle.adjoint_trace(g, m, d, rec, src)
    lhs, rhs = np.vdot(Fq, d), np.vdot(q, Ftd)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def test_dot_product_adjoint_no_sponge(oracle):
    rng = np.random.default_rng(2)
    g, m, _, src, rec = _case(oracle, nbl=0)
    q = rng.normal(size=NT)
    d = rng.normal(size=(NT, len(rec)))
    lhs = np.vdot(oracle.forward(g, m, q, src, rec), d)
    rhs = np.vdot(q, oracle.adjoint_trace(g, m, d, rec, src))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _phi(oracle, g, m, m0, q, src, rec, dobs):
    d = oracle.forward(g, m, q, src, rec, m0=m0)
    return 0.5 * np.sum((d - dobs) ** 2)


def _obs(oracle, g, m, q, src, rec):
    m_true = m * (1 + 0.08 * np.exp(-((np.indices(m.shape) - np.array(m.shape)[:, None, None, None] / 2) ** 2).sum(0) / 8.0))
    return oracle.forward(g, m_true, q, src, rec)


def test_gradient_matches_central_differences(oracle):
    g, m, q, src, rec = _case(oracle)
    dobs = _obs(oracle, g, m, q, src, rec)
    grad, phi, _, _ = oracle.gradient(g, m, q, src, rec, dobs)
    assert phi == pytest.approx(_phi(oracle, g, m, m, q, src, rec, dobs), rel=1e-13)
    rng = np.random.default_rng(5)
    dm = rng.normal(size=m.shape) * m.mean()
    an = np.vdot(grad, dm)
    rel = []
    for eps in (1e-4, 1e-5):
        fd = (_phi(oracle, g, m + eps * dm, m, q, src, rec, dobs)
              - _phi(oracle, g, m - eps * dm, m, q, src, rec, dobs)) / (2 * eps)
        rel.append(abs(fd - an) / abs(an))
    # the central difference converges to <g, dm> at second order in eps
    assert rel[1] <= 1e-6, rel
    assert 50 < rel[0] / rel[1] < 200, rel


def test_taylor_second_order(oracle):
    """|Phi(m + h dm) - Phi(m) - h <g, dm>| = O(h^2) (the linearisation test of
    Sec. 4.4, whose remainder roughly quadruples per doubling of h)."""
    g, m, q, src, rec = _case(oracle)
    dobs = _obs(oracle, g, m, q, src, rec)
    grad, phi, _, _ = oracle.gradient(g, m, q, src, rec, dobs)
    rng = np.random.default_rng(7)
    dm = rng.normal(size=m.shape) * m.mean() * 0.02
    hs = [1.0, 0.5, 0.25, 0.125]
    rem = [abs(_phi(oracle, g, m + h * dm, m, q, src, rec, dobs) - phi - h * np.vdot(grad, dm)) for h in hs]
    slopes = np.diff(np.log(rem)) / np.diff(np.log(hs))
    assert np.all(np.abs(slopes - 2.0) < 0.15), slopes


def test_gradient_zero_at_true_model(oracle):
    g, m, q, src, rec = _case(oracle)
    dobs = oracle.forward(g, m, q, src, rec)
    grad, phi, _, _ = oracle.gradient(g, m, q, src, rec, dobs)
    assert phi == 0.0 and np.all(grad == 0.0)


@pytest.mark.parametrize("k", [1, 3, 7, 10, NT, NT + 5])
def test_every_k_raw_bitwise_equals_full_history(oracle, k):
    """Checkpointing alone keeps the result bitwise identical (Sec. 1.3)."""
    g, m, q, src, rec = _case(oracle)
    dobs = _obs(oracle, g, m, q, src, rec)
    g_full, phi_full, d_full, _ = oracle.gradient(g, m, q, src, rec, dobs, mode=oracle.CKPT_FULL)
    g_k, phi_k, d_k, _ = oracle.gradient(g, m, q, src, rec, dobs, mode=oracle.CKPT_EVERY_K, k=k)
    assert np.array_equal(g_full, g_k) and phi_full == phi_k and np.array_equal(d_full, d_k)


def test_compressed_gradient_converges_as_atol_shrinks(oracle):
    """Lossy checkpoints: the gradient error falls as atol falls and tends to
    the uncompressed gradient (Sec. 4.4, the PSNR plateau)."""
    g, m, q, src, rec = _case(oracle)
    dobs = _obs(oracle, g, m, q, src, rec)
    g_ref, *_ = oracle.gradient(g, m, q, src, rec, dobs)
    errs, cfs = [], []
    for atol in (1e-1, 1e-3, 1e-5, 1e-7):
        gz, _, _, nbytes = oracle.gradient(g, m, q, src, rec, dobs, atol=atol)
        errs.append(np.linalg.norm(gz - g_ref) / np.linalg.norm(g_ref))
        cfs.append(NT * m.size * 4 / nbytes)
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-4, errs
    assert all(a >= b for a, b in zip(cfs, cfs[1:])), cfs


def test_every_k_compressed_close_to_full(oracle):
    g, m, q, src, rec = _case(oracle)
    dobs = _obs(oracle, g, m, q, src, rec)
    g_ref, *_ = oracle.gradient(g, m, q, src, rec, dobs)
    gz, *_ = oracle.gradient(g, m, q, src, rec, dobs, mode=oracle.CKPT_EVERY_K, k=10, atol=1e-6)
    assert np.linalg.norm(gz - g_ref) / np.linalg.norm(g_ref) < 1e-3


@pytest.mark.parametrize("nt,k", [(0, 1), (1, 1), (10, 3), (9, 3), (20, 20), (5, 8)])
def test_schedule_every_k_structure(oracle, nt, k):
    acts = oracle.ckpt_schedule(nt, oracle.CKPT_EVERY_K, k)
    adj = [s for kind, s, _ in acts if kind == oracle.ACT_ADJOINT]
    assert adj == sorted(set(adj), reverse=True) and adj == list(range(nt, 0, -1))
    stores = [s for kind, s, _ in acts if kind == oracle.ACT_STORE]
    assert stores == [0] + [c for c in range(k, nt + 1, k)]
    adv = [s for kind, s, _ in acts if kind == oracle.ACT_ADVANCE]
    assert adv == list(range(nt))
    # recomputation = forward steps not kept: N - (number of stored states) at most
    rec = sum(1 for kind, *_ in acts if kind == oracle.ACT_RECOMPUTE)
    assert rec <= nt


def test_schedule_full_structure(oracle):
    acts = oracle.ckpt_schedule(5, oracle.CKPT_FULL)
    kinds = [a[0] for a in acts]
    assert kinds == [1, 2] * 5 + [3, 5] * 5


def _griewank_min_steps(n, snaps):
    """Griewank's minimal number of extra forward steps to reverse n steps with
    `snaps` snapshots: r n - C(snaps + r, snaps + 1), r the repetition number
    with C(snaps + r - 1, snaps) < n <= C(snaps + r, snaps)."""
    from math import comb
    r = 0
    while comb(snaps + r, snaps) < n:
        r += 1
    return r * n - comb(snaps + r, snaps + 1)


@pytest.mark.parametrize("n,s", [(1, 1), (5, 1), (10, 2), (37, 3), (100, 4), (257, 6), (300, 2)])
def test_binomial_cost_is_griewank_minimum(oracle, n, s):
    # s spare slots besides the stored start state: Griewank's count with s + 1
    # snapshots, plus the n steps of the first pass
    assert oracle.binomial_cost(n, s) == n + _griewank_min_steps(n, s + 1)


@pytest.mark.parametrize("nt,s", [(1, 1), (10, 2), (25, 3), (70, 4), (40, 0)])
def test_binomial_schedule_structure(oracle, nt, s):
    acts = oracle.ckpt_schedule(nt, oracle.CKPT_BINOMIAL, s)
    assert [st for kind, st, _ in acts if kind == oracle.ACT_ADJOINT] == list(range(nt, 0, -1))
    assert [st for kind, st, _ in acts if kind == oracle.ACT_ADVANCE] == list(range(nt))
    live, peak = 0, 0
    steps = 0
    for kind, st, _ in acts:
        if kind == oracle.ACT_STORE and st > 0:
            live += 1
            peak = max(peak, live)
        elif kind == oracle.ACT_FREE:
            live -= 1
        elif kind in (oracle.ACT_ADVANCE, oracle.ACT_RECOMPUTE):
            steps += 1
    assert peak <= s and live == 0
    assert steps == oracle.binomial_cost(nt, s)


@pytest.mark.parametrize("s", [1, 3, 8])
def test_binomial_raw_bitwise_equals_full_history(oracle, s):
    g, m, q, src, rec = _case(oracle)
    dobs = _obs(oracle, g, m, q, src, rec)
    g_full, phi_full, d_full, _ = oracle.gradient(g, m, q, src, rec, dobs)
    g_b, phi_b, d_b, _ = oracle.gradient(g, m, q, src, rec, dobs, mode=oracle.CKPT_BINOMIAL, k=s)
    assert np.array_equal(g_full, g_b) and phi_full == phi_b and np.array_equal(d_full, d_b)


def test_binomial_compressed_close_to_full(oracle):
    g, m, q, src, rec = _case(oracle)
    dobs = _obs(oracle, g, m, q, src, rec)
    g_ref, phi_ref, *_ = oracle.gradient(g, m, q, src, rec, dobs)
    gz, phi_z, *_ = oracle.gradient(g, m, q, src, rec, dobs, mode=oracle.CKPT_BINOMIAL, k=3, atol=1e-6)
    assert phi_z == phi_ref   # data come from the exact first forward pass
    assert np.linalg.norm(gz - g_ref) / np.linalg.norm(g_ref) < 1e-3


def test_subsampling_f1_is_full_history(oracle):
    g, m, q, src, rec = _case(oracle)
    dobs = _obs(oracle, g, m, q, src, rec)
    g_full, phi, *_ = oracle.gradient(g, m, q, src, rec, dobs)
    g_s, phi_s, *_ = oracle.gradient(g, m, q, src, rec, dobs, mode=oracle.CKPT_SUBSAMPLE, k=1)
    assert np.array_equal(g_full, g_s) and phi == phi_s


def test_subsampling_weighted_sum_estimates_full_sum(oracle):
    """Imaging every f-th step with weight f is a rectangle-rule estimate of
    the full sum over steps (Sec. 4.7): for small f the subsampled gradient's
    component along the full gradient is the full gradient's size (within
    10%), where an unweighted subsample would give about 1/f of it."""
    g, m, q, src, rec = _case(oracle)
    dobs = _obs(oracle, g, m, q, src, rec)
    g_full, *_ = oracle.gradient(g, m, q, src, rec, dobs)
    for f in (2, 3, 4):
        gs, *_ = oracle.gradient(g, m, q, src, rec, dobs, mode=oracle.CKPT_SUBSAMPLE, k=f)
        proj = np.vdot(gs, g_full) / np.vdot(g_full, g_full)
        assert abs(proj - 1.0) < 0.1, (f, proj)


def test_subsampling_error_grows_with_factor(oracle):
    """Subsampled imaging (Sec. 4.7): the gradient's angle to the full one
    grows with the subsampling factor while the stored states shrink as 1/f."""
    g, m, q, src, rec = _case(oracle)
    dobs = _obs(oracle, g, m, q, src, rec)
    g_full, *_ = oracle.gradient(g, m, q, src, rec, dobs)
    angles = []
    for f in (2, 4, 8, 16):
        gs, _, _, nbytes = oracle.gradient(g, m, q, src, rec, dobs, mode=oracle.CKPT_SUBSAMPLE, k=f)
        cos = np.vdot(gs, g_full) / (np.linalg.norm(gs) * np.linalg.norm(g_full))
        angles.append(np.arccos(min(1.0, cos)))
        assert nbytes == (NT // f) * m.size * 4
    # grows, then saturates near the paper's largest angles (~0.8 rad at f=20)
    assert angles[0] < angles[1] < angles[2], angles
    assert min(angles[2:]) > 0.5, angles
    acts = oracle.ckpt_schedule(NT, oracle.CKPT_SUBSAMPLE, 4)
    assert sum(1 for k, *_ in acts if k == oracle.ACT_STORE) == NT // 4
