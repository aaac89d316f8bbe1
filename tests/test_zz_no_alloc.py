"""The allocation-free compress entry point
(zfp_compress_fixed_accuracy_noalloc), for callers that cannot allocate
device memory mid-run: it must produce exactly the stream of the regular
entry point, on consecutive calls that share its fixed scratch block.
Collected last on purpose (file name), so a failure here does not hide the
results of the other tests."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _call(lib, name, field, atol, cap):
    nz, ny, nx = field.shape
    out = torch.zeros(cap, dtype=torch.uint8, device=field.device)
    n = C.c_size_t(0)
    st = getattr(lib, name)(field.data_ptr(), nx, ny, nz, float(atol), out.data_ptr(), cap, C.byref(n),
                            torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st, n.value, out


@pytest.mark.parametrize("shape", [(1, 1, 1), (9, 10, 11), (37, 29, 23), (64, 96, 130)])
def test_noalloc_matches_regular_entry_point(cuda, fwi_lib, shape):
    from paper_2009_12623_gb300 import api
    rng = np.random.default_rng(sum(shape))
    cap = api.zfp_max_compressed_bytes(shape[2], shape[1], shape[0])
    for call in range(2):  # two calls in a row share the fixed scratch
        f = torch.from_numpy((rng.normal(size=shape) * np.exp(rng.normal(size=shape))).astype(np.float32)).to(cuda)
        for atol in (1e-2, 1e-5):
            st0, n0, ref = _call(fwi_lib, "zfp_compress_fixed_accuracy", f, atol, cap)
            st1, n1, got = _call(fwi_lib, "zfp_compress_fixed_accuracy_noalloc", f, atol, cap)
            assert st0 == 0 and st1 == 0
            assert n1 == n0
            assert torch.equal(got[:n1], ref[:n0])
            dec = api.zfp_decompress(got[:n1].clone(), shape)
            assert (dec - f).abs().max().item() <= atol


def test_noalloc_reports_capacity_and_rejects_oversize(cuda, fwi_lib):
    from paper_2009_12623_gb300 import _lib
    f = torch.randn((20, 21, 22), device=cuda)
    st0, n0, _ = _call(fwi_lib, "zfp_compress_fixed_accuracy", f, 1e-4, 1 << 20)
    st, n, _ = _call(fwi_lib, "zfp_compress_fixed_accuracy_noalloc", f, 1e-4, n0 // 2)
    assert st0 == 0 and st == _lib.FWI_ERR_CAPACITY and n == n0
    # a field larger than the fixed scratch is refused before any device work
    n = C.c_size_t(0)
    out = torch.zeros(64, dtype=torch.uint8, device=cuda)
    st = fwi_lib.zfp_compress_fixed_accuracy_noalloc(f.data_ptr(), 4096, 4096, 4096, 1e-3, out.data_ptr(),
                                                     64, C.byref(n), torch.cuda.current_stream().cuda_stream)
    assert st == _lib.FWI_ERR_ARG


def test_noalloc_bitwise_at_the_largest_accepted_field(cuda, fwi_lib):
    """At exactly the fixed scratch's limit (131,072 chunks: 1024 x 512 x 512
    values) the single-pass encoder's look-back runs across many waves of
    CTAs; its stream must still equal the regular entry point's bit for bit,
    on two calls in a row.  One chunk row more is refused."""
    from paper_2009_12623_gb300 import _lib, api
    nz, ny, nx = 512, 512, 1024
    gen = torch.Generator(device=cuda)
    gen.manual_seed(12)
    z = torch.arange(nz, device=cuda, dtype=torch.float32)[:, None, None]
    y = torch.arange(ny, device=cuda, dtype=torch.float32)[None, :, None]
    x = torch.arange(nx, device=cuda, dtype=torch.float32)[None, None, :]
    # a wave packet over a quiet background: chunk sizes from one bit per block to dense
    f = torch.sin(0.11 * x + 0.05 * y) * torch.cos(0.07 * z) * torch.exp(-((x - 500) ** 2 + (y - 260) ** 2) / 4e4)
    f = (f + 1e-3 * torch.randn((nz, ny, nx), device=cuda, generator=gen)).contiguous()
    cap = api.zfp_max_compressed_bytes(nx, ny, nz)
    for atol in (1e-4, 1e-2):
        st0, n0, ref = _call(fwi_lib, "zfp_compress_fixed_accuracy", f, atol, cap)
        st1, n1, got = _call(fwi_lib, "zfp_compress_fixed_accuracy_noalloc", f, atol, cap)
        assert st0 == 0 and st1 == 0 and n1 == n0
        assert torch.equal(got[:n1], ref[:n0])
        del ref, got
    n = C.c_size_t(0)
    out = torch.zeros(64, dtype=torch.uint8, device=cuda)
    st = fwi_lib.zfp_compress_fixed_accuracy_noalloc(f.data_ptr(), nx + 4, ny, nz, 1e-3, out.data_ptr(), 64,
                                                     C.byref(n), torch.cuda.current_stream().cuda_stream)
    assert st == _lib.FWI_ERR_ARG
