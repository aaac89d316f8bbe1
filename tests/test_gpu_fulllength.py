"""The Overthrust-shaped shot at its full record length against the FP64
oracle (Sec. 3, "Reference Problem": 4000 ms at dt = 1.75 ms = 2286 steps,
8 Hz Ricker source just under the surface, h = 25 m, 40-cell absorbing
layer, layered 1500-6000 m/s model with thrust faults, gradient at a
smoothed copy).

The lateral and vertical extent is reduced to 161 x 161 x 127 cells so the
FP64 oracle finishes in minutes on the host cores; every other parameter is
the full workload's.  What this checks is the accumulated FP32 error of the
GPU path over 2286 leapfrog steps forward and 2286 adjoint steps (Eq. (4)
summed over the whole record): the GPU gradient with full-history raw
checkpoints and with checkpoints compressed at atol = 1e-6 must each stay
within 1e-4 relative L2 of the uncompressed FP64 oracle gradient, element
by element over the whole grid, and the records and misfit within their
FP32 tolerances.  The oracle takes its every-48 raw mode, which equals its
full-history gradient bit for bit (pinned in the oracle tests)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
TOL = 1e-4
NX, NY, NZ, NT = 161, 161, 127, 2286


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def full_length(oracle):
    from paper_2009_12623_gb300 import synth
    shot = synth.overthrust_like_shot(nx=NX, ny=NY, nz=NZ, nt=NT)
    g = shot.geom
    assert (g.h, g.dt, g.nt, g.nbl, shot.f) == (25.0, 1.75e-3, 2286, 40, 8.0)
    og = oracle.geometry(g.nx, g.ny, g.nz, g.h, g.dt, g.nt, g.nbl, g.sponge_R, g.vmax)
    w = shot.wavelet.astype(np.float64)
    d_obs = oracle.forward(og, synth.slowness2(shot.v_true).astype(np.float64), w, shot.src, shot.rec)
    g_ref, phi_ref, d_sim, _ = oracle.gradient(og, synth.slowness2(shot.v0).astype(np.float64), w, shot.src,
                                               shot.rec, d_obs, mode=oracle.CKPT_EVERY_K, k=48)
    return shot, d_obs, g_ref, phi_ref, d_sim


@pytest.mark.parametrize("atol", [0.0, 1e-6])
def test_full_length_gradient_matches_fp64_oracle(cuda, full_length, atol):
    from paper_2009_12623_gb300 import api, synth
    shot, d_obs, g_ref, phi_ref, d_sim = full_length
    g = shot.geom
    m = torch.from_numpy(synth.slowness2(shot.v0)).to(cuda)
    rec = torch.from_numpy(shot.rec).to(cuda)
    obs = torch.from_numpy(d_obs.astype(np.float32)).to(cuda)
    raw_bytes = NX * NY * NZ * 4 * NT
    with api.CheckpointStore(raw_bytes + (4 << 30)) as st:
        grad, phi = api.gradient(g, m, shot.wavelet, shot.src, rec, obs, st, mode=api.FWI_CKPT_FULL, atol=atol)
        stats = st.stats()
    assert not stats["overflowed"] and stats["n_checkpoints"] == NT
    e = rel(grad.cpu().numpy(), g_ref)
    print(f"atol={atol}: gradient rel L2 vs FP64 oracle over {NT} steps {e:.3e}, "
          f"CF {stats['raw_bytes'] / max(stats['used_bytes'], 1):.1f}")
    assert e < TOL
    resid = d_sim - d_obs
    assert abs(phi - phi_ref) <= 2 * TOL * np.linalg.norm(d_sim) * np.linalg.norm(resid)


def test_full_length_records_match_fp64_oracle(cuda, full_length):
    from paper_2009_12623_gb300 import api, synth
    shot, _, _, _, d_sim = full_length
    d = api.forward(shot.geom, torch.from_numpy(synth.slowness2(shot.v0)).to(cuda), shot.wavelet, shot.src,
                    torch.from_numpy(shot.rec).to(cuda))
    e = rel(d.cpu().numpy(), d_sim)
    print(f"records rel L2 vs FP64 oracle over {NT} steps {e:.3e}")
    assert e < TOL
