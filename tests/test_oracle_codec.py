"""Pins of the oracle's fixed-accuracy codec (Sec. 1.4; the appendix figure on
direct compression: L_inf of the error stays below atol)."""
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "codec_blocks.json")


def test_minexp_is_floor_log2(oracle):
    for atol in (1.0, 0.5, 0.75, 1e-2, 1e-4, 1e-6, 3e-7, 2.0 ** -21, 1e-30, 123.0):
        assert oracle.zfp_minexp(atol) == int(np.floor(np.log2(atol)))


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"], ids=lambda c: c["name"])
def test_golden_blocks(oracle, case):
    v = np.full(64, case["value"], dtype=np.float32)
    minexp = oracle.zfp_minexp(case["atol"])
    words, n = oracle.zfp_encode_block(v, minexp)
    assert n == case["nbits"]
    if "word0" in case:
        mask = (1 << min(n, 64)) - 1
        assert int(words[0]) & mask == case["word0"]
    out, used = oracle.zfp_decode_block(words, n, minexp)
    assert used == n
    assert np.all(np.abs(out.astype(np.float64) - case["value"]) <= case["atol"])
    if case["name"] in ("lossless_three", "const_plus_one", "const_minus_one", "all_zero"):
        assert np.all(out == np.float32(case["value"]))


def _nega_digits(q):
    """Textbook base -2 digits by repeated division (brute force)."""
    digits = 0
    i = 0
    while q != 0:
        r = q % 2
        q = -(q - r) // 2
        digits |= r << i
        i += 1
    return digits


def test_negabinary_formula_matches_base_minus_two():
    rng = np.random.default_rng(0)
    for q in list(rng.integers(-2 ** 30, 2 ** 30, 2000)) + [0, 1, -1, 2 ** 24, -2 ** 24, 3 * 2 ** 23]:
        q = int(q)
        u = ((q + 0xAAAAAAAA) & 0xFFFFFFFF) ^ 0xAAAAAAAA
        assert u == _nega_digits(q)


def test_lift4_exhaustive_invertible(oracle):
    r = np.arange(-8, 8)
    grid = np.stack(np.meshgrid(r, r, r, r, indexing="ij"), -1).reshape(-1, 4)
    for x in grid:
        assert np.array_equal(oracle.zfp_lift4(oracle.zfp_lift4(x), inverse=True), x)


def test_lift4_means_are_floor_means(oracle):
    """The forward lifting's averages are floor means (rounding toward minus
    infinity, an arithmetic shift), as the format states: S is the floor mean
    of the two pairs' floor means and D their difference, on every input in
    [-8, 7]^4 (truncation toward zero differs on negative odd sums)."""
    r = np.arange(-8, 8)
    grid = np.stack(np.meshgrid(r, r, r, r, indexing="ij"), -1).reshape(-1, 4)
    for x in grid:
        a = (int(x[0]) + int(x[1])) // 2
        b = (int(x[2]) + int(x[3])) // 2
        out = oracle.zfp_lift4(x)
        assert out[0] == (a + b) // 2 and out[1] == b - a, (x, out)


def test_lift4_random_large_invertible(oracle):
    rng = np.random.default_rng(1)
    for x in rng.integers(-2 ** 28, 2 ** 28, size=(3000, 4)):
        assert np.array_equal(oracle.zfp_lift4(oracle.zfp_lift4(x), inverse=True), x)


def test_lift4_is_the_stated_linear_map_on_exact_inputs(oracle):
    """Where no rounding happens (inputs divisible by 8) the forward lifting
    equals S = mean, D = (x2+x3-x0-x1)/2, d0 = x1-x0-D/2, d1 = x3-x2-D/2."""
    rng = np.random.default_rng(2)
    for x in 8 * rng.integers(-1000, 1000, size=(500, 4)):
        S = x.sum() / 4
        D = (x[2] + x[3] - x[0] - x[1]) / 2
        expect = [S, D, x[1] - x[0] - D / 2, x[3] - x[2] - D / 2]
        assert np.array_equal(oracle.zfp_lift4(x), np.array(expect))


def test_xform3d_invertible_and_in_range(oracle):
    rng = np.random.default_rng(3)
    lim = 2 ** 25
    for _ in range(300):
        q = rng.integers(-lim + 1, lim, 64).astype(np.int32)
        c = oracle.zfp_fwd_xform(q)
        assert np.abs(c.astype(np.int64)).max() < 2 ** 30
        assert np.array_equal(oracle.zfp_inv_xform(c), q)
    # extreme sign patterns: per-axis worst case is the pattern maximising |d0 - D/2|
    pats = [np.array([(s >> b) & 1 for b in range(4)]) * 2 - 1 for s in range(16)]
    worst = 0
    for px in pats:
        for py in pats:
            for pz in pats:
                q = ((lim - 1) * pz[:, None, None] * py[None, :, None] * px[None, None, :]).reshape(64).astype(np.int32)
                c = oracle.zfp_fwd_xform(q)
                worst = max(worst, int(np.abs(c.astype(np.int64)).max()))
                assert np.array_equal(oracle.zfp_inv_xform(c), q)
    assert worst < 2 ** 30


def test_perm_is_sequency_order(oracle):
    p = oracle.zfp_perm()
    assert sorted(p) == list(range(64))
    keys = [(i & 3) + ((i >> 2) & 3) + (i >> 4) for i in p]
    assert keys == sorted(keys) and p[0] == 0


def _inverse_linear_bound(k):
    """Worst |q - q'| when every transform coefficient loses its lowest k
    negabinary digits, for the inverse lifting (derived independently here:
    linear part exactly over the digit box, plus 1/2 per floor step)."""
    hi = sum(2 ** b for b in range(0, k, 2))
    lo = -sum(2 ** b for b in range(1, k, 2))
    forms = {i: (np.eye(64)[i], 0.0) for i in range(64)}

    def half(a):
        return a[0] / 2, a[1] / 2 + 0.5

    def add(a, b, s=1):
        return a[0] + s * b[0], a[1] + b[1]

    def inv1(S, D, d0, d1):
        d1 = add(d1, half(D))
        d0 = add(d0, half(D))
        s0 = add(S, half(D), -1)
        s1 = add(D, s0)
        x2 = add(s1, half(d1), -1)
        x3 = add(d1, x2)
        x0 = add(s0, half(d0), -1)
        x1 = add(d0, x0)
        return x0, x1, x2, x3

    for stride in (16, 4, 1):
        new = dict(forms)
        for base in range(64):
            if (base // stride) % 4:
                continue
            ids = [base + t * stride for t in range(4)]
            for i, o in zip(ids, inv1(*[forms[i] for i in ids])):
                new[i] = o
        forms = new
    worst = 0.0
    for a, R in forms.values():
        mx = np.sum(np.where(a > 0, a * hi, a * lo))
        mn = np.sum(np.where(a > 0, a * lo, a * hi))
        worst = max(worst, max(mx, -mn) + R)
    return worst


@pytest.mark.parametrize("k", range(3, 16))
def test_guard_planes_prove_the_tolerance(k):
    """With 25 fraction bits and 11 guard planes a block that keeps planes
    31..k has emax - 25 = minexp - 4 - k, so
      |x - x'| <= 2^(emax-25) (1 + B(k))  [truncation + dropped digits]
                + 2^(emax-24)             [one FP32 rounding of the result]
    stays <= 2^minexp iff 3 + B(k) <= 2^(4+k).  Planes 30/31 are coded
    losslessly, so every lossy block has k >= 3."""
    assert 3 + _inverse_linear_bound(k) <= 2.0 ** (4 + k)


def test_guard_planes_are_needed_for_small_k():
    # the raise of planes 30/31 to 32 is required: k = 1, 2 would break the bound
    assert 1 + _inverse_linear_bound(1) > 2.0 ** 5
    assert 1 + _inverse_linear_bound(2) > 2.0 ** 6


def _blocks(rng, n):
    out = []
    for t in range(n):
        kind = t % 6
        x = rng.normal(size=64)
        if kind == 1:
            x = 1e-6 * x
            x[rng.integers(64)] = 1e3
        elif kind == 2:
            x = np.where(np.arange(64) % 2, -1.0, 1.0) * rng.uniform(0.5, 2)
        elif kind == 3:
            x = np.ldexp(1.0, rng.integers(-20, 20, 64)) * rng.choice([-1, 1], 64)
        elif kind == 4:
            i = np.arange(64)
            x = np.sin(0.4 * (i & 3) + 0.3 * ((i >> 2) & 3) + 0.2 * (i >> 4)) * rng.uniform(0.01, 10)
        elif kind == 5:
            x = np.ldexp(x, rng.integers(-30, 30))
        out.append(x.astype(np.float32))
    return out


@pytest.mark.parametrize("atol", [1e-1, 1e-2, 1e-4, 1e-6])
def test_error_bound_brute_force(oracle, atol):
    rng = np.random.default_rng(int(-np.log10(atol)))
    minexp = oracle.zfp_minexp(atol)
    for v in _blocks(rng, 600):
        words, n = oracle.zfp_encode_block(v, minexp)
        out, used = oracle.zfp_decode_block(words, n, minexp)
        assert used == n
        _, emax, planes = oracle.zfp_block_quantise(v, minexp)
        err = np.abs(out.astype(np.float64) - v.astype(np.float64)).max()
        if planes == 0 or emax - minexp <= 24:
            assert err <= 2.0 ** minexp <= atol, (err, emax, minexp)
        else:  # tolerance finer than FP32 resolves at this block's scale
            assert err < 2.0 ** (emax - 24)


def test_lossless_planes_reproduce_truncated_integers(oracle):
    rng = np.random.default_rng(9)
    for v in _blocks(rng, 200):
        minexp = oracle.zfp_minexp(2.0 ** -40)
        q, emax, planes = oracle.zfp_block_quantise(v, minexp)
        if planes != 32:
            continue
        words, n = oracle.zfp_encode_block(v, minexp)
        out, _ = oracle.zfp_decode_block(words, n, minexp)
        expect = np.ldexp(q.astype(np.float64), emax - 25).astype(np.float32)
        assert np.array_equal(out, expect)


def test_thirty_and_thirty_one_planes_are_coded_losslessly(oracle):
    """A block whose plane count comes out as 30 or 31 (emax - minexp = 19 or
    20) must be coded with all 32 planes -- dropping one or two planes would
    break the error bound (test_guard_planes_are_needed_for_small_k) -- so it
    decodes to its truncated block-floating-point integers exactly."""
    rng = np.random.default_rng(13)
    for v in _blocks(rng, 120):
        emax = int(np.frexp(np.float64(np.abs(v).max()))[1])
        for d in (19, 20):
            q, e2, planes = oracle.zfp_block_quantise(v, emax - d)
            assert e2 == emax and planes == 32, (d, planes)
            words, n = oracle.zfp_encode_block(v, emax - d)
            out, _ = oracle.zfp_decode_block(words, n, emax - d)
            assert np.array_equal(out, np.ldexp(q.astype(np.float64), emax - 25).astype(np.float32))


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 5, 7), (9, 10, 11), (8, 8, 8), (13, 4, 17)])
def test_stream_roundtrip_ragged(oracle, shape):
    rng = np.random.default_rng(sum(shape))
    f = (rng.normal(size=shape) * np.exp(rng.normal(size=shape))).astype(np.float32)
    for atol in (1e-1, 1e-3):
        s = oracle.zfp_compress(f, atol)
        g = oracle.zfp_decompress(s, shape)
        assert np.abs(g.astype(np.float64) - f).max() <= atol
        hdr = np.frombuffer(s[:64], dtype=np.uint32)
        assert hdr[0] == 0x315A4346 and tuple(hdr[2:5]) == shape[::-1]
        nblocks = int(np.prod([(d + 3) // 4 for d in shape]))
        assert int(np.frombuffer(s[24:32], np.uint64)[0]) == nblocks
        assert int(np.frombuffer(s[48:56], np.uint64)[0]) == len(s)


def test_stream_rejects_corruption(oracle):
    rng = np.random.default_rng(4)
    f = rng.normal(size=(12, 9, 10)).astype(np.float32)
    s = oracle.zfp_compress(f, 1e-3)
    for cut in (10, 63, 100, len(s) - 8):
        st, _ = oracle.zfp_decompress_status(s[:cut], f.shape)
        assert st == oracle.ERR_CORRUPT
    bad = bytearray(s)
    bad[0] ^= 1
    assert oracle.zfp_decompress_status(bytes(bad), f.shape)[0] == oracle.ERR_CORRUPT
    # a length-table entry that does not match its block
    bad = bytearray(s)
    lt = 64 + 8 * int(np.frombuffer(s[36:40], np.uint32)[0])
    bad[lt] ^= 0x3
    assert oracle.zfp_decompress_status(bytes(bad), f.shape)[0] == oracle.ERR_CORRUPT


def test_nonfinite_rejected(oracle):
    f = np.zeros((4, 4, 4), np.float32)
    f[1, 2, 3] = np.nan
    with pytest.raises(ValueError):
        oracle.zfp_compress(f, 1e-3)
    f[1, 2, 3] = np.inf
    with pytest.raises(ValueError):
        oracle.zfp_compress(f, 1e-3)


def test_linf_below_atol_and_psnr_rises(oracle):
    """Direct compression (Sec. 4.2): L_inf < atol at every tolerance and the
    PSNR grows as atol shrinks."""
    from paper_2009_12623_gb300 import synth
    f = synth.shells_field(48, seed=1, rmin=5, rmax=20)
    R = f.max() - f.min()
    psnr = []
    for atol in (1e-1, 1e-2, 1e-4, 1e-6):
        g = oracle.zfp_decompress(oracle.zfp_compress(f, atol), f.shape)
        e = g.astype(np.float64) - f
        assert np.abs(e).max() < atol
        psnr.append(10 * np.log10(R ** 2 / np.mean(e ** 2)))
    assert all(a < b for a, b in zip(psnr, psnr[1:])), psnr


def test_compressibility_falls_as_the_wave_spreads(oracle):
    """Evolution of compressibility (Sec. 4.1): early states (mostly zeros)
    compress far better than late ones."""
    from paper_2009_12623_gb300 import synth
    n, h, c, f = 40, 10.0, 1500.0, 15.0
    dt = 1e-3
    m = np.full((n, n, n), 1.0 / c ** 2)
    cfs = []
    for nt in (60, 200):
        g = oracle.geometry(n, n, n, h, dt, nt, 8, 1e-3, c)
        _, _, u = oracle.forward(g, m, synth.wavelet(nt, dt, f).astype(np.float64), (20, 20, 20),
                                 np.zeros((0, 3)), return_state=True)
        s = oracle.zfp_compress(u.astype(np.float32), 1e-4)
        cfs.append(u.size * 4 / len(s))
    assert cfs[0] > 2 * cfs[1], cfs
