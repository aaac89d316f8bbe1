"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, exports
every symbol include/fwi.h declares, and its host-only logic (checkpoint
schedules, argument validation, status strings) behaves -- no kernel runs."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "fwi.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M)))


def test_header_declarations_parsed():
    names = _declared()
    assert "fwi_gradient" in names and "zfp_compress_fixed_accuracy" in names
    assert len(names) >= 14


def test_library_exports_every_declared_symbol(fwi_lib):
    from paper_2009_12623_gb300 import _lib
    for name in _declared():
        assert hasattr(fwi_lib, name), name
    assert sorted(_lib.EXPORTS) == _declared()


def test_oracle_library_exports(oracle):
    L = oracle.lib()
    text = open(os.path.join(ROOT, "oracle", "oracle.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    for name in re.findall(r"\b(oracle_\w+)\s*\(", text):
        assert hasattr(L, name), name


def test_status_strings(fwi_lib):
    from paper_2009_12623_gb300 import _lib
    assert _lib.status_string(0) == "ok"
    assert "capacity" in _lib.status_string(-2)
    assert "corrupt" in _lib.status_string(-3)


@pytest.mark.parametrize("nt,mode,k", [(0, 1, 1), (7, 1, 1), (12, 2, 1), (12, 2, 5), (13, 2, 4),
                                       (40, 2, 10), (5, 2, 9), (2286, 2, 10), (2286, 1, 1),
                                       (0, 3, 2), (1, 3, 1), (10, 3, 2), (70, 3, 4), (40, 3, 0),
                                       (333, 3, 7), (2286, 3, 12), (6, 4, 2), (200, 4, 3),
                                       (17, 4, 5), (2286, 4, 8)])
def test_schedule_matches_oracle(fwi_lib, oracle, nt, mode, k):
    from paper_2009_12623_gb300 import api
    assert api.ckpt_schedule(nt, mode, k) == oracle.ckpt_schedule(nt, mode, k)


def test_schedule_rejects_bad_policy(fwi_lib):
    from paper_2009_12623_gb300 import _lib
    pol = _lib.Policy(2, 0, 0.0)
    n = C.c_size_t(0)
    assert fwi_lib.fwi_ckpt_schedule(10, C.byref(pol), None, 0, C.byref(n)) == _lib.FWI_ERR_ARG
    pol = _lib.Policy(9, 1, 0.0)
    assert fwi_lib.fwi_ckpt_schedule(10, C.byref(pol), None, 0, C.byref(n)) == _lib.FWI_ERR_ARG


def test_max_bytes_matches_oracle(fwi_lib, oracle):
    from paper_2009_12623_gb300 import api
    for shape in [(1, 1, 1), (64, 64, 64), (881, 881, 287), (5, 9, 13), (512, 512, 512)]:
        assert api.zfp_max_compressed_bytes(*shape) == oracle.zfp_max_bytes(*shape)
    assert api.zfp_max_compressed_bytes(0, 4, 4) == 0


def test_argument_validation_without_gpu(fwi_lib):
    from paper_2009_12623_gb300 import _lib
    g = _lib.Geometry(0, 4, 4, 1.0, 1e-3, 5, 0, 1e-3, 1500.0)
    pol = _lib.Policy(1, 1, 0.0)
    phi = C.c_double()
    # invalid geometry is rejected before any device work
    assert fwi_lib.fwi_gradient(C.byref(g), None, None, 0, 0, 0, None, 0, None, None, C.byref(phi),
                                None, C.byref(pol), None) == _lib.FWI_ERR_ARG
    n = C.c_size_t()
    assert fwi_lib.zfp_compress_fixed_accuracy(None, 4, 4, 4, 1e-3, None, 0, C.byref(n), None) == _lib.FWI_ERR_ARG
    assert fwi_lib.zfp_decompress(None, 0, None, 4, 4, 4, None) == _lib.FWI_ERR_ARG


def test_batch_argument_validation_without_gpu(fwi_lib):
    from paper_2009_12623_gb300 import _lib
    g = _lib.Geometry(40, 40, 20, 10.0, 1e-3, 0, 4, 1e-3, 2000.0)
    ok = _lib.Shot(0, 0, 0, 20, 20, 20, 10, 5, 5, 3, 0, 0, 0, 0)
    out = C.c_void_p()
    pol = _lib.Policy(2, 4, 1e-4)
    create = fwi_lib.fwi_batch_create
    shots = (_lib.Shot * 1)(ok)
    assert create(C.byref(g), 0, shots, None, C.byref(pol), 1 << 20, 0, C.byref(out)) == _lib.FWI_ERR_ARG
    for bad in [_lib.Shot(30, 0, 0, 20, 20, 20, 10, 35, 5, 3, 0, 0, 0, 0),   # window past the grid
                _lib.Shot(0, 0, 0, 20, 20, 20, 0, 5, 5, 3, 0, 0, 0, 0),     # no time steps
                _lib.Shot(0, 0, 0, 20, 20, 20, 10, 25, 5, 3, 0, 0, 0, 0),   # source outside the window
                _lib.Shot(0, 0, 0, 20, 20, 20, 10, 5, 5, 3, 0, 4, 0, 0)]:   # receivers but no array
        arr = (_lib.Shot * 1)(bad)
        assert create(C.byref(g), 1, arr, None, C.byref(pol), 1 << 20, 0, C.byref(out)) == _lib.FWI_ERR_ARG
    for p in [_lib.Policy(3, 2, 0.0), _lib.Policy(4, 2, 0.0), _lib.Policy(2, 0, 0.0)]:
        assert create(C.byref(g), 1, shots, None, C.byref(p), 1 << 20, 0, C.byref(out)) == _lib.FWI_ERR_ARG
    assert create(C.byref(g), 1, shots, None, C.byref(pol), 1 << 20, 8, C.byref(out)) == _lib.FWI_ERR_ARG
    assert fwi_lib.fwi_batch_destroy(None) == _lib.FWI_ERR_ARG
    assert fwi_lib.fwi_batch_get_stats(None, None) == _lib.FWI_ERR_ARG


def test_selftest_argument_validation_without_gpu(fwi_lib):
    from paper_2009_12623_gb300 import _lib
    assert fwi_lib.fwi_selftest_bounded_wait(0, None) == _lib.FWI_ERR_ARG
    assert fwi_lib.fwi_selftest_bounded_wait((1 << 20) + 1, None) == _lib.FWI_ERR_ARG
    assert fwi_lib.fwi_selftest_damped_quotient(None, None, None, -1, None) == _lib.FWI_ERR_ARG
    assert fwi_lib.fwi_selftest_damped_quotient(None, None, None, 4, None) == _lib.FWI_ERR_ARG
    n = C.c_int(-1)
    assert fwi_lib.fwi_ckpt_store_slot_bytes(None, None, 0, C.byref(n)) == _lib.FWI_ERR_ARG


def test_python_binding_rejects_bad_tensors_without_gpu():
    """The binding checks devices, dtypes and shapes before any library call."""
    import torch
    from paper_2009_12623_gb300 import api
    with pytest.raises(ValueError):
        api.selftest_damped_quotient(torch.ones(3), torch.ones(4))
    with pytest.raises(TypeError):
        api.selftest_damped_quotient(torch.ones(3), torch.ones(3))  # host tensors
    with pytest.raises(TypeError):
        api.dot_f64(torch.ones(3, dtype=torch.float64), torch.ones(3, dtype=torch.float64))
