"""The forward-propagation experiment of Sec. 4 (restart from a lossy
checkpoint): stop the simulation, compress its state pair (u^{T-1}, u^T) at a
fixed absolute tolerance, continue from the lossy and from the exact state,
and follow the difference of the two runs.  The paper reports that the L_inf
and L2 norms of that difference rise sharply over the first few steps and
then settle into a decreasing trend.  The oracle (FP64 steps from FP32
states, the oracle codec) must show the same shape, with the difference
bounded by a small multiple of the tolerance."""
import numpy as np

T1, STEPS = 100, 150


def restart_curve(oracle, atol, t1=T1, steps=STEPS):
    """(L_inf per step, L2 per step, L_inf of the codec error at the restart)."""
    from paper_2009_12623_gb300 import synth
    shot = synth.two_layer_shot(n=48, nt=t1 + steps, h=10.0, dt=1e-3, nbl=8, f=25.0)
    g = shot.geom
    m = synth.slowness2(shot.v0).astype(np.float64)
    w = shot.wavelet.astype(np.float64)
    og = oracle.geometry(g.nx, g.ny, g.nz, g.h, g.dt, t1, g.nbl, g.sponge_R, g.vmax)
    _, up, uc = oracle.forward(og, m, w[:t1], shot.src, shot.rec, return_state=True)
    exact = [f.astype(np.float32).astype(np.float64) for f in (up, uc)]
    lossy = [oracle.zfp_decompress(oracle.zfp_compress(f.astype(np.float32), atol), f.shape).astype(np.float64)
             for f in (up, uc)]
    e0 = float(np.abs(lossy[1] - exact[1]).max())
    one = oracle.geometry(g.nx, g.ny, g.nz, g.h, g.dt, 1, g.nbl, g.sponge_R, g.vmax)
    linf, l2 = [], []
    for i in range(steps):
        wi = w[t1 + i:t1 + i + 1]
        _, a0, a1 = oracle.forward(one, m, wi, shot.src, shot.rec, u_prev_init=exact[0], u_cur_init=exact[1],
                                   return_state=True)
        _, b0, b1 = oracle.forward(one, m, wi, shot.src, shot.rec, u_prev_init=lossy[0], u_cur_init=lossy[1],
                                   return_state=True)
        exact, lossy = [a0, a1], [b0, b1]
        d = a1 - b1
        linf.append(float(np.abs(d).max()))
        l2.append(float(np.sqrt((d * d).sum())))
    return np.array(linf), np.array(l2), e0


def test_lossy_restart_error_rises_then_decays(oracle):
    atol = 1e-6  # the paper's setting for this experiment
    linf, l2, e0 = restart_curve(oracle, atol)
    assert 0 < e0 <= atol                      # the codec's bound at the restart
    k = int(np.argmax(l2))
    assert 1 <= k <= 30 and l2[k] > 1.5 * l2[0]  # sharp rise over the first steps
    assert l2[-1] < 0.8 * l2[k]                # then a decreasing trend
    assert linf[-1] < 0.8 * linf.max()
    assert linf.max() <= 2 * atol              # bounded: no growth of the perturbation
