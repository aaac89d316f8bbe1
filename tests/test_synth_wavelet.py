"""The source wavelet (Sec. 3: an 8 Hz Ricker source) pinned by closed-form
properties of the Ricker function r(t) = (1 - 2 a) exp(-a),
a = (pi f (t - t0))^2, rather than by retyping it:

* r(t0) = 1 is the global maximum (the wavelet is not inverted or scaled);
* its zeros lie at t0 +- 1/(pi f sqrt 2) and its two minima at
  t0 +- sqrt(3/2)/(pi f) with value -2 exp(-3/2);
* it integrates to zero (the second derivative of a Gaussian);
* its amplitude spectrum peaks at the dominant frequency f;
* the sampled source q^n = r(n dt) is delayed by t0 = 1.5/f (the reading of
  the unstated delay) so that it starts from ~1e-8 of its peak.

A wrong delay, sign, frequency scaling or exponent fails one of these."""
import numpy as np
import pytest

from paper_2009_12623_gb300 import synth


@pytest.mark.parametrize("f", [8.0, 10.0, 15.0, 25.0])
def test_ricker_extrema_and_zeros(f):
    t0 = 0.3
    assert synth.ricker(t0, f, t0) == pytest.approx(1.0, abs=1e-15)
    tz = 1.0 / (np.pi * f * np.sqrt(2.0))
    for s in (-1, 1):
        assert abs(synth.ricker(t0 + s * tz, f, t0)) < 1e-14
    tm = np.sqrt(1.5) / (np.pi * f)
    for s in (-1, 1):
        assert synth.ricker(t0 + s * tm, f, t0) == pytest.approx(-2.0 * np.exp(-1.5), rel=1e-13)
        eps = 1e-4 / f
        assert synth.ricker(t0 + s * tm + eps, f, t0) > synth.ricker(t0 + s * tm, f, t0)
        assert synth.ricker(t0 + s * tm - eps, f, t0) > synth.ricker(t0 + s * tm, f, t0)
    t = np.linspace(t0 - 2.0 / f, t0 + 2.0 / f, 20001)
    r = synth.ricker(t, f, t0)
    assert r.max() == pytest.approx(1.0, abs=1e-6) and abs(t[np.argmax(r)] - t0) < 1e-3 / f
    assert r.min() == pytest.approx(-2.0 * np.exp(-1.5), rel=1e-6)


@pytest.mark.parametrize("f", [8.0, 10.0, 20.0])
def test_ricker_zero_mean_and_peak_frequency(f):
    dt = 1e-4
    t = np.arange(0, 4.0, dt)
    r = synth.ricker(t, f, 2.0)
    assert abs(r.sum() * dt) < 1e-9
    spec = np.abs(np.fft.rfft(r))
    nu = np.fft.rfftfreq(len(r), dt)
    assert abs(nu[np.argmax(spec)] - f) <= 0.25 + 1e-9


def test_wavelet_delay_and_onset():
    # 8 Hz at dt = 1.75 ms (the reference problem): t0 = 187.5 ms
    w = synth.wavelet(2286, 1.75e-3, 8.0)
    assert w.dtype == np.float32 and w.shape == (2286,)
    n_peak = int(np.argmax(w))
    assert abs(n_peak * 1.75e-3 - 1.5 / 8.0) <= 1.75e-3 / 2
    assert abs(w[0]) < 1e-7 and abs(w[-1]) < 1e-30 + 1e-7
    # 10 Hz at dt = 1 ms: t0 = 150 ms falls on sample 150 exactly
    w = synth.wavelet(400, 1e-3, 10.0)
    assert int(np.argmax(w)) == 150 and w[150] == np.float32(1.0)
    assert w[150 - 23] < 0 < w[150 - 22] and w[150 + 22] > 0 > w[150 + 23]   # zeros at +-22.5 ms
