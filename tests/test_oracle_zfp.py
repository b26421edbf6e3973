"""Pins of the fixed-rate ZFP oracle (Alg. 3; the reading is in oracle/zfp.c),
CPU only: the transform against hand values and its exact inverse, negabinary
against the base -2 digits, the sequency order, the embedded coding against a
stream worked by hand and its prefix property, and the whole codec: the
fixed-point error bound at a budget that codes every plane, fixed sizes,
error falling with the rate, zero and constant fields, partial blocks."""
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "zfp_planes_small.txt")


def _golden():
    g = {}
    for ln in open(GOLD):
        if ln.startswith("#") or not ln.strip():
            continue
        k, *v = ln.split()
        g[k] = [int(x) for x in v]
    return g


def test_transform_hand_values_and_inverse():
    # s0 = floor(7/2) = 3, d0 = 3; s1 = floor(4/2) = 2, d1 = -10; S = floor(5/2) = 2, D = 1
    assert list(oracle.zfp_fwd_line([5, 2, -3, 7])) == [2, 1, 3, -10]
    # a ramp: s0 = 0, d0 = -1, s1 = 2, d1 = -1, S = 1, D = -2
    assert list(oracle.zfp_fwd_line([0, 1, 2, 3])) == [1, -2, -1, -1]
    # negative odd sums round down: s0 = floor(-7/2) = -4
    assert list(oracle.zfp_fwd_line([-5, -2, 0, 0])) == [-2, -4, -3, 0]
    for c in (0, 7, -9, 2 ** 26):
        assert list(oracle.zfp_fwd_line([c] * 4)) == [c, 0, 0, 0]
    rng = np.random.default_rng(1)
    for _ in range(2000):
        a = rng.integers(-2 ** 27, 2 ** 27, size=4)
        assert np.array_equal(oracle.zfp_inv_line(oracle.zfp_fwd_line(a)), a)


def test_negabinary_digits():
    def digits_value(u, P):
        return sum(((u >> k) & 1) * (-2) ** k for k in range(P))
    assert [oracle.negabinary(q, 32) for q in (0, 1, -1, 2, -2, 3)] == [0, 1, 3, 6, 2, 7]
    rng = np.random.default_rng(2)
    for P, lim in ((32, 2 ** 30), (64, 2 ** 62)):
        for q in list(rng.integers(-lim, lim, size=300)) + [lim - 1, -lim, 0]:
            u = oracle.negabinary(int(q), P)
            assert u < 2 ** P and digits_value(u, P) == int(q)
            assert oracle.from_negabinary(u, P) == int(q)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_sequency_order(d):
    cls = [0, 1, 2, 2]
    perm = oracle.zfp_order(d)
    assert sorted(perm) == list(range(4 ** d)) and perm[0] == 0

    def key(i):
        s = 0
        for _ in range(d):
            s += cls[i % 4]
            i //= 4
        return s
    keys = [key(i) for i in perm]
    assert keys == sorted(keys)
    for a, b in zip(perm, perm[1:]):
        assert key(a) < key(b) or a < b


def test_planes_worked_by_hand():
    g = _golden()
    u, P = g["u"], g["P"][0]
    w = oracle.zfp_encode_planes(u, P, 32)
    assert int(w[0]) == g["word_full"][0]
    assert np.array_equal(oracle.zfp_decode_planes(w, 4, P, 32), u)
    w6 = oracle.zfp_encode_planes(u, P, 6)
    assert int(w6[0]) == g["word_6"][0]
    assert list(oracle.zfp_decode_planes(w6, 4, P, 6)) == g["decoded_6"]


@pytest.mark.parametrize("B,P", [(4, 32), (16, 32), (64, 32), (64, 64)])
def test_planes_exact_and_prefix(B, P):
    rng = np.random.default_rng(B + P)
    for trial in range(20):
        # magnitudes fall along the order, as transform coefficients do
        top = np.maximum(1, (P - 3) - np.arange(B) // max(1, B // 8) * 3)
        u = np.array([int(rng.integers(0, 2 ** int(t))) for t in top], dtype=np.uint64)
        full = 2 * B * P + 64
        assert np.array_equal(oracle.zfp_decode_planes(oracle.zfp_encode_planes(u, P, full), B, P, full), u)
        for budget in (1, 7, 40, B * 3, B * 8):
            dec = oracle.zfp_decode_planes(oracle.zfp_encode_planes(u, P, budget), B, P, budget)
            # every decoded value keeps a top run of the true bits and zeros below
            for x, y in zip(u.astype(object), dec.astype(object)):
                assert y & ~x == 0
                low = x ^ y
                assert low == 0 or (y >> low.bit_length()) == (x >> low.bit_length())


def _blocks_emax(u):
    """exponent e (x = f 2^e, 1/2 <= |f| < 1) of the largest value of each 4^d block, per value"""
    d = u.ndim
    e = np.full(u.shape, -10 ** 6, dtype=np.int64)
    pad = [(0, (-s) % 4) for s in u.shape]
    up = np.pad(np.abs(u), pad, mode="edge")
    shp = []
    for s in up.shape:
        shp += [s // 4, 4]
    blk = up.reshape(shp)
    ax = tuple(range(1, 2 * d, 2))
    mx = blk.max(axis=ax)
    _, ex = np.frexp(mx)
    full = ex
    for k in range(d):
        full = np.repeat(full, 4, axis=k)
    return full[tuple(slice(0, s) for s in u.shape)]


@pytest.mark.parametrize("shape", [(1000,), (65, 33), (33, 17, 9), (8, 8, 8), (5, 6, 7)], ids=str)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_codec_error_bound_at_full_budget(shape, dtype):
    from paper_2503_06322_gb300 import fields
    u = (fields.powerlaw_field(shape, seed=4, dtype=dtype) if len(shape) > 1
         else np.random.default_rng(4).standard_normal(shape).astype(dtype))
    P = 32 if dtype == np.float32 else 64
    B = 4 ** len(shape)
    # a plane costs at most 2B + 1 bits (B verbatim or scanned, B + 1 tests):
    # the smallest rate whose budget holds every plane and the block header
    rate = -(-(P * (2 * B + 1) + 1 + 12) // B)
    while (rate * B) % 32:
        rate += 1
    b = oracle.zfp_compress(u, rate)
    nb = int(np.prod([(s + 3) // 4 for s in shape]))
    assert b.size == 64 + nb * rate * B // 8
    r = oracle.zfp_decompress(b)
    emax = _blocks_emax(u.astype(np.float64))
    # truncation to P-5 fraction bits below the block exponent, plus the
    # final rounding to binary32
    bound = np.ldexp(1.0, (emax - (P - 5)).astype(np.int64))
    if dtype == np.float32:
        bound = bound + np.abs(u).astype(np.float64) * 2.0 ** -24
    assert np.all(np.abs(r - u.astype(np.float64)) <= bound)


def test_error_falls_with_rate_and_sizes_are_fixed():
    from paper_2503_06322_gb300 import fields
    u = fields.powerlaw_field((40, 36, 28), seed=5, dtype=np.float32)
    errs = []
    for rate in (2, 4, 8, 12, 16, 24):
        b = oracle.zfp_compress(u, rate)
        assert b.size == 64 + 10 * 9 * 7 * rate * 64 // 8
        e = oracle.zfp_decompress(b) - u
        errs.append(float(np.sqrt(np.mean(e * e))))
    assert all(a > b for a, b in zip(errs, errs[1:])), errs


def test_zero_constant_and_rates():
    z = np.zeros((9, 10), dtype=np.float32)
    assert np.array_equal(oracle.zfp_decompress(oracle.zfp_compress(z, 2)), z)
    c = np.full((6, 7, 5), 3.25, dtype=np.float32)
    assert np.array_equal(oracle.zfp_decompress(oracle.zfp_compress(c, 1)), c)
    with pytest.raises(ValueError):
        oracle.zfp_compress(np.zeros(10, np.float32), 4)     # 4 x 4 bits: not a multiple of 32
    assert oracle.zfp_bound((10,), 8) == 64 + 3 * 4
