"""Shot stacking (Sec. 2: the survey gradient is the sum of the shots'
gradients; Sec. 4's stacking experiment): the compression errors of the
individual shot gradients do not accumulate through the sum -- for useful
tolerances the stacked gradient's relative error stays at or below the worst
single shot's -- and the stacked error shrinks with atol.  On the oracle, a
small layered model with four shots sharing a receiver plane."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def survey(oracle):
    from paper_2009_12623_gb300 import synth
    n, nz, nt, h, dt = 40, 28, 110, 10.0, 1e-3
    vt = synth.layered_velocity(n, n, nz, seed=3, nlayers=4, vmin=1500.0, vmax=3000.0, water=6, fault_shift=3)
    m0 = synth.slowness2(synth.smooth(vt, 2.0)).astype(np.float64)
    mt = synth.slowness2(vt).astype(np.float64)
    w = synth.wavelet(nt, dt, 25.0).astype(np.float64)
    g = oracle.geometry(n, n, nz, h, dt, nt, 6, 1e-3, 3000.0)
    rec = np.array([(i, j, 8) for i in range(7, n - 7, 3) for j in range(7, n - 7, 3)], np.int32)
    srcs = [(12, 12, 8), (27, 12, 8), (12, 27, 8), (20, 20, 8)]
    d_obs = [oracle.forward(g, mt, w, s, rec) for s in srcs]
    raw = [oracle.gradient(g, m0, w, s, rec, d)[0] for s, d in zip(srcs, d_obs)]
    return g, m0, w, rec, srcs, d_obs, raw


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_stacking_does_not_accumulate_compression_errors(oracle, survey):
    g, m0, w, rec, srcs, d_obs, raw = survey
    stacked = {}
    for atol in (1e-2, 1e-4):
        lossy = [oracle.gradient(g, m0, w, s, rec, d, mode=oracle.CKPT_FULL, atol=atol)[0]
                 for s, d in zip(srcs, d_obs)]
        per_shot = [_rel(a, b) for a, b in zip(lossy, raw)]
        stacked[atol] = _rel(sum(lossy), sum(raw))
        assert 0 < stacked[atol] <= max(per_shot)
    assert stacked[1e-2] > 10 * stacked[1e-4]
