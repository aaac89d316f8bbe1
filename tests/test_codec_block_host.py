"""The GPU codec's per-block code (csrc/codec_block.cuh, host-compilable) run
on the CPU against the oracle codec, block by block: the same bit count, the
same bits and the same decoded values (Sec. 1.4's fixed-accuracy
compression).  This checks, without a GPU, the arithmetic that the encode and
decode kernels execute for every block -- block-floating-point conversion,
lifting transform, sequency order, negabinary, the two plane transposes, the
exact bit count, the embedded coder and its inverse -- with the plane-mask
accessors the kernels use; the kernels add only the placement of blocks in
the stream, which the GPU tests check bit for bit."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("codec_block") / "codec_block_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-x", "c++", os.path.join(HERE, "host", "codec_block_check.cpp"),
                    "-o", exe], check=True)
    return exe


def _blocks(rng, n):
    """Blocks of several kinds: wide-range, smooth, sparse, tiny, subnormal, huge, constant."""
    out = []
    for i in range(n):
        kind = i % 7
        if kind == 0:
            b = rng.normal(size=64) * np.exp(3 * rng.normal(size=64))
        elif kind == 1:
            z, y, x = np.meshgrid(np.arange(4), np.arange(4), np.arange(4), indexing="ij")
            b = (np.sin(rng.uniform(0, 1) * x + rng.uniform(0, 1) * y - 0.3 * z) * rng.uniform(0.1, 10)).ravel()
        elif kind == 2:
            b = rng.normal(size=64) * (rng.uniform(size=64) < 0.1)
        elif kind == 3:
            b = rng.normal(size=64) * 1e-6
        elif kind == 4:
            b = rng.normal(size=64) * 1e-41
        elif kind == 5:
            b = rng.normal(size=64) * 1e35
        else:
            b = np.full(64, rng.normal())
        out.append(b)
    return np.asarray(out, dtype=np.float32).reshape(n, 4, 4, 4)


def _harness(exe, minexp, blocks):
    data = struct.pack("<ii", minexp, len(blocks)) + np.ascontiguousarray(blocks, np.float32).tobytes()
    raw = subprocess.run([exe], input=data, capture_output=True, check=True).stdout
    res, off = [], 0
    for _ in range(len(blocks)):
        nbits, nwords = struct.unpack_from("<ii", raw, off)
        off += 8
        words = np.frombuffer(raw, np.uint64, nwords, off)
        off += 8 * nwords
        vals = np.frombuffer(raw, np.uint32, 64, off)
        off += 256
        ok, cut_ok, long_ok = struct.unpack_from("<iii", raw, off)
        off += 12
        res.append((nbits, words, vals, (ok, cut_ok, long_ok)))
    assert off == len(raw)
    return res


def _oracle_block(oracle, block, atol):
    """(minexp, bit count, payload words, decoded values) of a one-block field."""
    s = oracle.zfp_compress(block, atol)
    minexp = struct.unpack_from("<i", s, 20)[0]
    nblocks, = struct.unpack_from("<Q", s, 24)
    nchunks, = struct.unpack_from("<I", s, 36)
    words, = struct.unpack_from("<Q", s, 40)
    assert nblocks == 1 and nchunks == 1
    length_table = 64 + 8 * nchunks
    payload = length_table + (2 * nblocks + 7) // 8 * 8
    nbits, = struct.unpack_from("<H", s, length_table)
    pw = np.frombuffer(s, np.uint64, words, payload)
    dec = oracle.zfp_decompress(s, block.shape)
    return minexp, nbits, pw, dec


@pytest.mark.parametrize("atol", [1e-1, 1e-3, 1e-6, 1e-30, 1e30])
def test_block_code_matches_oracle(oracle, harness, atol):
    rng = np.random.default_rng(int(-np.log10(atol)) + 40)
    blocks = _blocks(rng, 350)
    ref = [_oracle_block(oracle, b, atol) for b in blocks]
    minexp = ref[0][0]
    assert all(r[0] == minexp for r in ref)
    got = _harness(harness, minexp, blocks)
    for (nbits, words, vals, ok), (_, o_nbits, o_words, o_dec), b in zip(got, ref, blocks):
        # accepted at its coded length, rejected when declared one bit shorter or longer (the
        # decoder checks the block's bounds once, against the bits it consumed)
        assert ok == (1, 0, 0)
        assert nbits == o_nbits
        assert np.array_equal(words, o_words)
        assert np.array_equal(vals, o_dec.reshape(-1).view(np.uint32))
        # the codec's bound: atol, or 2^(emax-24) where atol is finer than FP32 resolves at the
        # block's scale (emax = frexp exponent of the block's largest magnitude)
        emax = np.frexp(np.float64(np.abs(b).max()))[1]
        bound = max(atol, 2.0 ** (emax - 24))
        assert np.all(np.abs(vals.view(np.float32).astype(np.float64) - b.reshape(-1)) <= bound)


def test_embedded_coder_edges(tmp_path):
    """The coder's group-coded assembly at its edges: all 64 coefficients
    significant in the top plane (128 bits), coefficient 63 alone, runs that
    end at 63, plus 2000 random plane sets -- bit for bit against a direct
    restatement of the group coding, the exact bit count, and the decoder."""
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "emit_edge_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-x", "c++", os.path.join(HERE, "host", "emit_edge_check.cpp"),
                    "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.startswith("ok "), out.stdout
