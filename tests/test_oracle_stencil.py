"""Pins of the oracle's spatial operator and forward sweep against mathematics
that does not come from the oracle itself (Sec. 2, Eq. (1))."""
import numpy as np
import pytest


def _geom(o, n, h=1.0, nt=1, nbl=0, dt=1e-3, vmax=1500.0):
    return o.geometry(n, n, n, h, dt, nt, nbl, 1e-3, vmax)


def test_laplacian_exact_on_degree9_polynomials(oracle):
    # the 9-point 8th-order second difference is exact on polynomials of degree <= 9
    n, h = 24, 0.5
    g = _geom(oracle, n, h=h)
    c = np.arange(n) * h - (n - 1) * h / 2
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    u = 0.01 * x ** 9 + 0.3 * y ** 7 * x ** 2 - 0.2 * z ** 8 + x * y * z + 1.0
    lap_exact = (0.01 * 72 * x ** 7 + 0.3 * (42 * y ** 5 * x ** 2 + 2 * y ** 7) - 0.2 * 56 * z ** 6)
    Lu = oracle.laplacian(g, u)
    s = slice(4, n - 4)
    err = np.abs(Lu[s, s, s] - lap_exact[s, s, s]).max()
    assert err <= 1e-9 * np.abs(lap_exact[s, s, s]).max()


def test_laplacian_degree10_is_not_exact(oracle):
    # sanity of the previous pin: one degree higher leaves an h^8 error term
    n, h = 24, 0.5
    g = _geom(oracle, n, h=h)
    c = np.arange(n) * h - (n - 1) * h / 2
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    Lu = oracle.laplacian(g, x ** 10)
    s = slice(4, n - 4)
    err = np.abs(Lu[s, s, s] - 90 * x[s, s, s] ** 8).max()
    # leading error term: 2 * (-1/630) * h^8 * u^(10) / 2 ... is nonzero
    assert err > 1e-3


def test_laplacian_eighth_order_convergence(oracle):
    errs = []
    L = 1.0
    for n in (16, 32):
        h = L / n
        g = _geom(oracle, n + 8, h=h)
        c = (np.arange(n + 8) - 4) * h
        z, y, x = np.meshgrid(c, c, c, indexing="ij")
        k = 2 * np.pi * np.array([1.0, 1.5, 0.75])
        u = np.sin(k[0] * x) * np.sin(k[1] * y + 0.3) * np.sin(k[2] * z + 0.1)
        Lu = oracle.laplacian(g, u)
        s = slice(4, n + 4)
        errs.append(np.abs(Lu[s, s, s] + (k ** 2).sum() * u[s, s, s]).max())
    slope = np.log2(errs[0] / errs[1])
    assert abs(slope - 8.0) < 0.3, slope


def test_laplacian_symmetric(oracle):
    rng = np.random.default_rng(3)
    n = 13
    g = _geom(oracle, n, h=0.7)
    u, v = rng.normal(size=(2, n, n, n))
    a = np.vdot(oracle.laplacian(g, u), v)
    b = np.vdot(u, oracle.laplacian(g, v))
    assert abs(a - b) <= 1e-12 * abs(a)


def test_sponge_profile_closed_form(oracle):
    n, nbl, h, vmax, R = 30, 6, 10.0, 3000.0, 1e-3
    s = oracle.sponge_profile(n, nbl, h, vmax, R)
    W = nbl * h
    peak = 3 * vmax / (2 * W) * np.log(1 / R)
    assert s[0] == pytest.approx(peak, rel=1e-14)
    assert s[n - 1] == pytest.approx(peak, rel=1e-14)
    assert s[nbl - 1] == pytest.approx(peak / nbl ** 2, rel=1e-14)
    assert np.all(s[nbl:n - nbl] == 0.0)
    assert np.allclose(s, s[::-1])


def test_homogeneous_greens_function(oracle):
    """Far field of a point source in a homogeneous medium:
    u(r,t) = h^3 q(t - r/c) / (4 pi r)  (unit injection at one cell = h^3 delta)."""
    from paper_2009_12623_gb300 import synth
    n, h, c, f = 72, 10.0, 1500.0, 15.0
    dt = 5e-4
    nt = 640                                   # 0.32 s: before any boundary reflection
    g = oracle.geometry(n, n, n, h, dt, nt, 0, 1e-3, c)
    m = np.full((n, n, n), 1.0 / c ** 2)
    q = synth.wavelet(nt, dt, f).astype(np.float64)
    s = (36, 36, 36)
    rs = [10, 12, 14]
    rec = [(s[0] + r, s[1], s[2]) for r in rs] + [(s[0], s[1] - r, s[2]) for r in rs]
    rec += [(s[0] + 8, s[1] + 8, s[2]), (s[0], s[1] + 7, s[2] - 7)]
    d = oracle.forward(g, m, q, s, np.array(rec))
    t = (np.arange(nt) + 1) * dt               # d^n = u^{n+1}
    for j, (i, jj, k) in enumerate(rec):
        r = h * np.sqrt((i - s[0]) ** 2 + (jj - s[1]) ** 2 + (k - s[2]) ** 2)
        ana = h ** 3 * synth.ricker(t - r / c, f, 1.5 / f) / (4 * np.pi * r)
        rel = np.abs(d[:, j] - ana).max() / np.abs(ana).max()
        assert rel < 0.02, (rec[j], rel)


def test_greens_function_error_shrinks_with_dt(oracle):
    from paper_2009_12623_gb300 import synth
    n, h, c, f = 64, 10.0, 1500.0, 15.0
    errs = []
    for dt in (2e-3, 1e-3):
        T = 0.3
        nt = int(round(T / dt))
        g = oracle.geometry(n, n, n, h, dt, nt, 0, 1e-3, c)
        m = np.full((n, n, n), 1.0 / c ** 2)
        q = synth.wavelet(nt, dt, f).astype(np.float64)
        s = (32, 32, 32)
        rec = np.array([(44, 32, 32)])
        d = oracle.forward(g, m, q, s, rec)[:, 0]
        t = (np.arange(nt) + 1) * dt
        ana = h ** 3 * synth.ricker(t - 120.0 / c, f, 1.5 / f) / (4 * np.pi * 120.0)
        errs.append(np.abs(d - ana).max())
    # second order in time: halving dt cuts the (time-dominated) error ~4x
    assert errs[0] / errs[1] > 2.5, errs


def test_sponge_absorbs(oracle):
    """With the absorbing layer the energy left in the grid after the wave has
    reached the boundary is far below the undamped case."""
    from paper_2009_12623_gb300 import synth
    n, h, c, f = 40, 10.0, 1500.0, 15.0
    dt = 1e-3
    nt = 500
    m = np.full((n, n, n), 1.0 / c ** 2)
    q = synth.wavelet(nt, dt, f).astype(np.float64)
    e = []
    for nbl in (0, 10):
        g = oracle.geometry(n, n, n, h, dt, nt, nbl, 1e-3, c)
        _, _, ul = oracle.forward(g, m, q, (20, 20, 20), np.zeros((0, 3)), return_state=True)
        e.append(np.sum(ul ** 2))
    assert e[1] < 0.01 * e[0], e
