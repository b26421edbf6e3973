"""Pins of the oracle's Huffman stage (Sec. IV-B, Alg. 2) and of its
quantization and container (Sec. IV-A) against what is fixed independently:
hand-derived golden cases, the Kraft equality, the optimal total cost of a
textbook heap Huffman, brute-force optimal lengths on small alphabets, the
round trips, the CRC-32 check value and the error-bound property."""
import heapq
import itertools
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_cases(name):
    cases, cur = [], None
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *rest = line.split()
        if key == "case":
            cur = {"name": rest[0]}
            cases.append(cur)
        else:
            (cur if cur is not None else cases.append({}) or cases[-1])[key] = rest
    return cases


def _pairs(items):
    return {int(a): b for a, b in (x.split(":") for x in items)}


@pytest.mark.parametrize("case", _read_cases("huffman_small.txt"), ids=lambda c: c["name"])
def test_golden_lengths_and_codes(oracle, case):
    D = 16
    hist = np.zeros(D, dtype=np.uint64)
    for s, f in _pairs(case["freq"]).items():
        hist[s] = int(f)
    ln = oracle.code_lengths(hist)
    code = oracle.canonical_codes(ln)
    for s, l in _pairs(case["len"]).items():
        assert ln[s] == int(l)
    for s, c in _pairs(case["code"]).items():
        assert ln[s] == len(c) and code[s] == int(c, 2)
    assert ln.sum() == sum(int(x) for x in _pairs(case["len"]).values())


def test_golden_bitstream(oracle):
    spec = {}
    for line in open(os.path.join(GOLDEN, "bitstream_small.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, *v = line.split()
            spec[k] = v
    ln = np.zeros(16, dtype=np.uint8)
    ln[[1, 2, 3, 4]] = [1, 2, 3, 3]
    sym = np.array([int(x) for x in spec["symbols"]], dtype=np.uint16)
    words, chunk, bits = oracle.encode(sym, ln, K=2)
    assert [int(w) for w in words] == [int(x, 16) for x in spec["words"]]
    assert bits == int(spec["bits"][0])
    assert [int(c) for c in chunk] == [int(x) for x in spec["chunks"]]
    assert np.array_equal(oracle.decode(words, chunk, sym.size, 2, ln), sym)


def test_golden_escape_payload(oracle):
    spec = {}
    for line in open(os.path.join(GOLDEN, "escape_small.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, *v = line.split()
            spec[k] = v
    ln = np.zeros(8, dtype=np.uint8)
    for pair in spec["lengths"]:
        s_, l_ = pair.split(":")
        ln[int(s_)] = int(l_)
    sym = np.array([int(x) for x in spec["symbols"]], dtype=np.uint16)
    esc = np.array([int(x) for x in spec["escapes"]], dtype=np.int64)
    assert oracle.escape_width(esc) == int(spec["width"][0])
    for prefix, width in (("", None), ("width5_", 5)):
        words, chunk, bits = oracle.encode(sym, ln, K=2, esc_k=esc, esc_width=width)
        assert [int(w) for w in words] == [int(x, 16) for x in spec[prefix + "words"]]
        assert bits == int(spec[prefix + "bits"][0])
        assert [int(c) for c in chunk] == [int(x) for x in spec[prefix + "chunks"]]
        w = int(spec["width"][0]) if width is None else width
        dsym, desc = oracle.decode(words, chunk, sym.size, 2, ln, esc_width=w)
        assert np.array_equal(dsym, sym) and np.array_equal(desc, esc)
    # without escapes symbol 0 is a plain symbol: 3 bits in all
    w2, c2, b2 = oracle.encode(sym, ln, K=2)
    assert b2 == 3 and [int(w) for w in w2] == [0x60000000]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_escape_payload_round_trip(oracle, seed):
    rng = np.random.default_rng(seed)
    D = 64
    N = 5000
    sym = rng.integers(0, D, N).astype(np.uint16)
    sym[rng.random(N) < 0.2] = 0
    ne = int((sym == 0).sum())
    mags = np.concatenate([[D // 2, 2 ** 40, (1 << 31) - 1],
                           rng.integers(D // 2, 2 ** 20, max(ne - 3, 0))])[:ne]
    if seed == 2:
        mags[0] = 2 ** 62 - 1
    esc = (mags * rng.choice([-1, 1], ne)).astype(np.int64)
    ln = oracle.code_lengths(oracle.histogram(sym, D))
    words, chunk, bits = oracle.encode(sym, ln, K=128, esc_k=esc)
    z = [2 * int(k) if k >= 0 else -2 * int(k) - 1 for k in esc]
    w = max(x.bit_length() for x in z)
    assert oracle.escape_width(esc) == w
    assert bits == int(ln[sym].astype(np.int64).sum()) + ne * w
    dsym, desc = oracle.decode(words, chunk, N, 128, ln, esc_width=w)
    assert np.array_equal(dsym, sym) and np.array_equal(desc, esc)


def test_escape_code_out_of_range_is_rejected(oracle):
    ln = np.zeros(4, dtype=np.uint8)
    ln[[0, 1]] = 1
    sym = np.array([0, 1], dtype=np.uint16)
    with pytest.raises(Exception):
        oracle.encode(sym, ln, K=2, esc_k=np.array([2 ** 62], dtype=np.int64), esc_width=63)
    with pytest.raises(Exception):
        oracle.encode(sym, ln, K=2, esc_k=np.array([0], dtype=np.int64), esc_width=8)
    with pytest.raises(Exception):   # a width too small for the code
        oracle.encode(sym, ln, K=2, esc_k=np.array([1000], dtype=np.int64), esc_width=5)


def _heap_cost(freqs):
    h = list(freqs)
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def _random_hist(rng, D, nsym, heavy=False):
    hist = np.zeros(D, dtype=np.uint64)
    syms = rng.choice(D, size=nsym, replace=False)
    if heavy:
        f = np.floor(np.exp(rng.uniform(0, 12, size=nsym))).astype(np.uint64) + 1
    else:
        f = rng.integers(1, 20, size=nsym).astype(np.uint64)
    hist[syms] = f
    return hist


@pytest.mark.parametrize("seed", range(12))
def test_kraft_equality_and_optimal_cost(oracle, seed):
    rng = np.random.default_rng(seed)
    D = 4096
    hist = _random_hist(rng, D, int(rng.integers(2, 3000)), heavy=bool(seed % 2))
    ln = oracle.code_lengths(hist)
    nz = hist > 0
    assert np.all(ln[nz] > 0) and np.all(ln[~nz] == 0)
    from fractions import Fraction
    assert sum(Fraction(1, 2 ** int(l)) for l in ln[nz]) == 1
    assert int((hist.astype(object) * ln.astype(object)).sum()) == _heap_cost(
        [int(x) for x in hist[nz]])


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_lengths_optimal_against_brute_force(oracle, n):
    rng = np.random.default_rng(n)
    for _ in range(5):
        f = rng.integers(1, 30, size=n)
        hist = np.zeros(8, dtype=np.uint64)
        hist[:n] = f
        ln = oracle.code_lengths(hist)[:n]
        best = None
        for lens in itertools.product(range(1, n), repeat=n):
            if sum(2.0 ** -l for l in lens) <= 1.0:
                c = int(np.dot(f, lens))
                best = c if best is None or c < best else best
        assert int(np.dot(f, ln)) == best


@pytest.mark.parametrize("seed", range(6))
def test_canonical_codes_prefix_free_and_ordered(oracle, seed):
    rng = np.random.default_rng(100 + seed)
    hist = _random_hist(rng, 512, int(rng.integers(2, 400)), heavy=True)
    ln = oracle.code_lengths(hist)
    code = oracle.canonical_codes(ln)
    present = [s for s in range(512) if ln[s]]
    strs = {s: format(int(code[s]), "0%db" % ln[s]) for s in present}
    order = sorted(present, key=lambda s: (ln[s], s))
    assert int(code[order[0]]) == 0
    for a, b in zip(order, order[1:]):          # canonical: increasing by (len, symbol)
        assert int(code[b]) > (int(code[a]) << (int(ln[b]) - int(ln[a])))
    for a in present:
        for b in present:
            if a != b:
                assert not strs[b].startswith(strs[a])


@pytest.mark.parametrize("K", [1, 7, 64, 1024])
def test_encode_decode_round_trip(oracle, K):
    rng = np.random.default_rng(K)
    sym = np.clip(np.round(rng.normal(4096, 300, size=20000)), 0, 8191).astype(np.uint16)
    hist = oracle.histogram(sym, 8192)
    ln = oracle.code_lengths(hist)
    words, chunk, bits = oracle.encode(sym, ln, K=K)
    assert bits == int(ln[sym].astype(np.int64).sum())
    offs = np.concatenate([[0], np.cumsum(ln[sym].astype(np.int64))])
    assert np.array_equal(chunk, offs[::K][:len(chunk)])
    assert np.array_equal(oracle.decode(words, chunk, sym.size, K, ln), sym)


def test_crc32_check_value(oracle):
    assert oracle.crc32(b"123456789") == 0xCBF43926


def test_quantize_definition_small(oracle):
    # one level-0 node per value: 1-D of 2 nodes, L = 0, bin q
    q = np.array([0.5])
    sym, idx, k = oracle.quantize(np.array([0.76, -0.26]), (2,), q, D=16)
    # k = sign(x) floor(|x|/q + 1/2): 0.76/0.5 = 1.52 -> 2 ; -0.26/0.5 = -0.52 -> -1
    assert list(sym) == [2 + 8, -1 + 8] and idx.size == 0
    sym, idx, k = oracle.quantize(np.array([100.0, 0.1]), (2,), q, D=16)
    assert sym[0] == 0 and list(idx) == [0] and list(k) == [200]


@pytest.mark.parametrize("shape,tol,mode,kind,D", [
    ((129, 129), 1e-3, 0, 1, 8192), ((33, 17, 9), 1e-2, 0, 1, 8192), ((100,), 1e-4, 0, 1, 256),
    ((20, 20, 20), 1e-3, 1, 1, 8192), ((9, 6, 5), 0.05, 0, 0, 64), ((65, 65), 1e-4, 0, 1, 16),
    ((2,), 1e-3, 0, 1, 8192), ((3, 2), 1e-2, 0, 1, 4)])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_container_round_trip_within_bound(oracle, shape, tol, mode, kind, D, dtype):
    u = (np.random.default_rng(sum(shape)).standard_normal(shape) * 3 + 1).astype(dtype)
    if len(shape) == 2 and shape[0] == 129:
        from paper_2503_06322_gb300.fields import sinusoid_field_2d
        u = sinusoid_field_2d().astype(dtype)
    buf = oracle.compress(u, tol, tol_kind=kind, mode=mode, D=D)
    h = oracle.parse_header(buf)
    assert h["magic"] == b"HPDR" and h["version"] == 3 and h["dims"] == shape
    assert h["crc"] == oracle.crc32(bytes(buf[:124]))
    assert h["total_bytes"] == len(buf)
    ref_norm = np.abs(u.astype(np.float64)).max() if mode == 0 else \
        np.sqrt((u.astype(np.float64) ** 2).mean())
    tau_abs = tol * ref_norm if kind == 1 else tol
    assert h["tau_abs"] == pytest.approx(tau_abs, rel=1e-13)
    r = oracle.decompress(buf)
    err = np.abs(r - u.astype(np.float64)).max()
    assert err <= tau_abs
    # the reconstruction also holds the bound after rounding to the data type
    assert np.abs(r.astype(dtype).astype(np.float64) - u.astype(np.float64)).max() <= tau_abs


def test_zero_field_is_exact(oracle):
    u = np.zeros((17, 9), dtype=np.float32)
    r = oracle.decompress(oracle.compress(u, 1e-3))
    assert np.all(r == 0)


def test_corrupt_header_rejected(oracle):
    u = np.random.default_rng(0).standard_normal((17, 9)).astype(np.float32)
    buf = bytearray(oracle.compress(u, 1e-2).tobytes())
    bad = bytearray(buf)
    bad[20] ^= 1
    with pytest.raises(RuntimeError):
        oracle.decompress(bad)
    with pytest.raises(RuntimeError):
        oracle.decompress(buf[:100])


def test_bound_floor_rejected(oracle):
    u = np.random.default_rng(0).standard_normal((513,)).astype(np.float32)
    with pytest.raises(RuntimeError):
        oracle.compress(u, 1e-7)
