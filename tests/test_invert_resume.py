"""Host logic of the inversion driver: a steepest-descent run interrupted,
saved to a file and resumed takes exactly the iterations of an uninterrupted
run (same models, same misfit history).  A quadratic misfit stands in for the
GPU gradient, so this runs on the CPU."""
import numpy as np
import torch


def _quadratic(target):
    def grad_fn(c):
        r = (c - target).double()
        return float(0.5 * (r * r).sum()), (c - target)
    return grad_fn


def test_resume_continues_exactly(tmp_path):
    from paper_2009_12623_gb300 import invert
    g = torch.Generator().manual_seed(0)
    target = 2000.0 + 300.0 * torch.rand((6, 7, 8), generator=g)
    c0 = 2000.0 + 300.0 * torch.rand((6, 7, 8), generator=g)
    mask = torch.ones_like(c0)
    mask[0] = 0.0
    fn = _quadratic(target)
    kw = dict(step=0.05, vmin=1500.0, vmax=4000.0, mask=mask)
    c_ref, h_ref, _ = invert.descend(c0, fn, 6, **kw)

    path = str(tmp_path / "state.npz")
    c_half, h_half, _ = invert.descend(c0, fn, 3, on_iter=lambda st: invert.save_state(path, st), **kw)
    st = invert.load_state(path)
    assert len(st["hist"]) == 3 and torch.equal(st["c"], c_half)
    c_res, h_res, first = invert.descend(c0, fn, 6, resume=st, **kw)
    assert first is None  # the gradient scale came from the saved state
    assert torch.equal(c_res, c_ref)
    assert h_res == h_ref
    # the misfit falls and the masked plane never moves
    assert h_ref[-1] < h_ref[0]
    assert torch.equal(c_ref[0], c0[0])


def test_resume_of_a_finished_run_is_a_no_op(tmp_path):
    from paper_2009_12623_gb300 import invert
    c0 = torch.full((4, 4, 4), 2500.0)
    target = torch.full((4, 4, 4), 2600.0)
    path = str(tmp_path / "s.npz")
    c, h, _ = invert.descend(c0, _quadratic(target), 2, 0.01, 1500.0, 4000.0, None,
                             on_iter=lambda st: invert.save_state(path, st))
    calls = []

    def never(c):
        calls.append(1)
        raise AssertionError("no gradient expected")
    c2, h2, _ = invert.descend(c0, never, 2, 0.01, 1500.0, 4000.0, None, resume=invert.load_state(path))
    assert not calls and torch.equal(c2, c) and h2 == h
    assert np.isclose(h[0], 0.5 * 64 * 100.0 ** 2)
