"""Host-side container checks of the C ABI library, without a GPU.

hpdr_inspect and hpdr_zfp_inspect read a header in host memory with no
device work, so they run here: on containers written by the oracle (an
independent writer of the same documented format, container version 3 and
the ZFP container of Alg. 3) they must report the oracle's shape and type,
and every corruption of the header must give HPDR_ERR_FORMAT -- a flipped
bit anywhere in the CRC-covered bytes, a truncated buffer, and fields that
are out of range although their CRC was recomputed.  The decompression
entry points rely on these checks before they size any device launch."""
import ctypes as C

import numpy as np
import pytest

HPDR_OK, HPDR_ERR_ARG, HPDR_ERR_FORMAT = 0, -1, -4


@pytest.fixture(scope="module")
def lib():
    from paper_2503_06322_gb300 import build
    L = C.CDLL(build.build())
    L.hpdr_inspect.argtypes = [C.c_void_p, C.c_size_t, C.POINTER(C.c_int), C.POINTER(C.c_int),
                               C.POINTER(C.c_size_t)]
    L.hpdr_zfp_inspect.argtypes = [C.c_void_p, C.c_size_t, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                   C.POINTER(C.c_size_t), C.POINTER(C.c_uint32)]
    return L


def _inspect(lib, buf, n=None):
    b = np.ascontiguousarray(np.frombuffer(bytes(buf), dtype=np.uint8))
    dt, nd, dims = C.c_int(-7), C.c_int(-7), (C.c_size_t * 3)()
    st = lib.hpdr_inspect(b.ctypes.data, b.size if n is None else n, C.byref(dt), C.byref(nd), dims)
    return st, dt.value, nd.value, tuple(dims)[:max(nd.value, 0)]


def _zinspect(lib, buf, n=None):
    b = np.ascontiguousarray(np.frombuffer(bytes(buf), dtype=np.uint8))
    dt, nd, dims, rate = C.c_int(-7), C.c_int(-7), (C.c_size_t * 3)(), C.c_uint32(0)
    st = lib.hpdr_zfp_inspect(b.ctypes.data, b.size if n is None else n, C.byref(dt), C.byref(nd), dims,
                              C.byref(rate))
    return st, dt.value, nd.value, tuple(dims)[:max(nd.value, 0)], rate.value


def _field(shape, dtype, seed):
    return (np.random.default_rng(seed).standard_normal(shape) * 2 + 0.5).astype(dtype)


CASES = [((65, 65), np.float32, {}), ((33, 17, 9), np.float64, {}), ((100,), np.float32, {"D": 256}),
         ((20, 20, 20), np.float32, {"mode": 1}), ((9, 6, 5), np.float64, {"tol_kind": 0}),
         ((3, 2), np.float32, {"D": 4}), ((17, 9), np.float32, {"coords": "graded"})]


def _compress(oracle, shape, dtype, kw, seed=3):
    kw = dict(kw)
    if kw.get("coords") == "graded":
        kw["coords"] = [np.cumsum(np.linspace(1.0, 2.0, n)) for n in shape]
    return np.frombuffer(oracle.compress(_field(shape, dtype, seed), 1e-3, **kw).tobytes(),
                         dtype=np.uint8).copy()


@pytest.mark.parametrize("shape,dtype,kw", CASES, ids=lambda c: str(c))
def test_inspect_reports_the_oracle_header(lib, oracle, shape, dtype, kw):
    buf = _compress(oracle, shape, dtype, kw)
    h = oracle.parse_header(buf)
    st, dt, nd, dims = _inspect(lib, buf)
    assert st == HPDR_OK
    assert dt == (0 if dtype == np.float32 else 1) == h["dtype"]
    assert nd == len(shape) and dims == shape == h["dims"]


@pytest.mark.parametrize("shape,dtype,kw", CASES[:3], ids=lambda c: str(c))
def test_every_flipped_header_bit_is_rejected(lib, oracle, shape, dtype, kw):
    buf = _compress(oracle, shape, dtype, kw)
    for byte in range(128):
        for bit in range(8):
            bad = buf.copy()
            bad[byte] ^= np.uint8(1 << bit)
            assert _inspect(lib, bad)[0] == HPDR_ERR_FORMAT, (byte, bit)


def test_truncated_and_null_inputs(lib, oracle):
    buf = _compress(oracle, (33, 17, 9), np.float32, {})
    total = oracle.parse_header(buf)["total_bytes"]
    assert total == buf.size
    for n in (0, 1, 64, 127, 128, 129, total // 2, total - 4, total - 1):
        assert _inspect(lib, buf, n)[0] == HPDR_ERR_FORMAT, n
    assert _inspect(lib, buf, total)[0] == HPDR_OK
    dt, nd, dims = C.c_int(), C.c_int(), (C.c_size_t * 3)()
    assert lib.hpdr_inspect(None, total, C.byref(dt), C.byref(nd), dims) == HPDR_ERR_ARG
    assert lib.hpdr_inspect(buf.ctypes.data, total, None, C.byref(nd), dims) == HPDR_ERR_ARG


def _put(buf, off, width, value):
    buf[off:off + width] = np.frombuffer(int(value).to_bytes(width, "little"), dtype=np.uint8)


def _put_f64(buf, off, value):
    buf[off:off + 8] = np.frombuffer(np.float64(value).tobytes(), dtype=np.uint8)


def _reseal(oracle, buf):
    _put(buf, 124, 4, oracle.crc32(bytes(buf[:124])))
    return buf


# (name, byte offset, width, value): fields of the v3 header (oracle/container.c)
# set out of range; the CRC is recomputed so that only the field check can reject them
BAD_FIELDS = [
    ("version 2", 4, 4, 2), ("dtype 2", 8, 4, 2), ("ndim 0", 12, 4, 0), ("ndim 4", 12, 4, 4),
    ("dims[0] = 1", 16, 8, 1), ("dims[1] = 2^31", 24, 8, 1 << 31), ("L + 1", 40, 4, None),
    ("tol-kind reserved bit", 48, 4, 0x201), ("D odd", 52, 4, 8191), ("D = 2", 52, 4, 2),
    ("D = 2^17", 52, 4, 1 << 17), ("K not a multiple of 128", 56, 4, 1000), ("K = 2^16", 56, 4, 1 << 16),
    ("N off by one", 96, 8, None), ("escapes above N", 104, 8, None), ("bits below N", 112, 8, 5),
    ("bits above 63 N", 112, 8, None), ("s_hi >= D", 120, 2, 8192), ("reserved byte 123", 123, 1, 1),
]


@pytest.mark.parametrize("name,off,width,value", BAD_FIELDS, ids=[b[0] for b in BAD_FIELDS])
def test_out_of_range_fields_are_rejected(lib, oracle, name, off, width, value):
    buf = _compress(oracle, (33, 17, 9), np.float32, {})
    h = oracle.parse_header(buf)
    assert _inspect(lib, _reseal(oracle, buf.copy()))[0] == HPDR_OK    # resealing alone changes nothing
    if value is None:
        value = {"L + 1": h["L"] + 1, "N off by one": h["N"] + 1, "escapes above N": h["N"] + 1,
                 "bits above 63 N": 64 * h["N"] + 64}[name]
    bad = buf.copy()
    _put(bad, off, width, value)
    assert _inspect(lib, _reseal(oracle, bad))[0] == HPDR_ERR_FORMAT


def test_escape_count_and_width_must_agree(lib, oracle):
    buf = _compress(oracle, (33, 17, 9), np.float32, {})
    h = oracle.parse_header(buf)
    bad = buf.copy()
    # escapes without a payload width, or a width without escapes
    _put(bad, 104, 8, 3)
    _put(bad, 122, 1, 0)
    assert _inspect(lib, _reseal(oracle, bad))[0] == HPDR_ERR_FORMAT
    bad = buf.copy()
    _put(bad, 104, 8, 0)
    _put(bad, 122, 1, 5)
    assert _inspect(lib, _reseal(oracle, bad))[0] == HPDR_ERR_FORMAT
    assert h["n_escapes"] <= h["N"]


@pytest.mark.parametrize("q", [0.0, -1.0, float("nan"), float("inf")])
def test_bin_widths_must_be_positive_and_finite(lib, oracle, q):
    buf = _compress(oracle, (33, 17, 9), np.float32, {})
    L = oracle.parse_header(buf)["L"]
    for level in (0, L):
        bad = buf.copy()
        _put_f64(bad, 128 + 8 * level, q)
        # q lies after the CRC-covered bytes: only the field check can reject it
        assert _inspect(lib, bad)[0] == HPDR_ERR_FORMAT, level


@pytest.mark.parametrize("shape,rate,dtype", [((64,), 8, np.float32), ((17, 9), 12, np.float64),
                                               ((9, 8, 7), 4, np.float32), ((5, 5, 5), 32, np.float64)])
def test_zfp_inspect(lib, oracle, shape, rate, dtype):
    buf = oracle.zfp_compress(_field(shape, dtype, 11), rate)
    st, dt, nd, dims, r = _zinspect(lib, buf)
    assert st == HPDR_OK and dims == shape and r == rate and dt == (0 if dtype == np.float32 else 1)
    assert nd == len(shape)
    for byte in range(64):
        bad = buf.copy()
        bad[byte] ^= np.uint8(1 << (byte % 8))
        assert _zinspect(lib, bad)[0] == HPDR_ERR_FORMAT, byte
    for n in (0, 63, 64, buf.size - 1):
        assert _zinspect(lib, buf, n)[0] == HPDR_ERR_FORMAT, n
