"""numpy front end of the C oracle (argument marshalling only).

TEST INFRASTRUCTURE ONLY.  Every function builds the oracle library on first
use (plain gcc) and calls it through ctypes.
"""
import ctypes as C

import numpy as np

from . import build as _build

__all__ = [
    "levels", "decompose", "recompose", "recompose_adjoint", "decompose_adjoint",
    "correction_norms", "bins", "bins_l2s", "l2s_weights", "quantize", "dequantize", "histogram",
    "code_lengths", "canonical_codes", "encode", "decode", "escape_width", "compress",
    "decompress", "inspect", "compress_bound", "crc32", "level_sizes",
    "parse_header", "zfp_bound", "zfp_compress", "zfp_decompress", "zfp_fwd_line", "zfp_inv_line",
    "zfp_order", "negabinary", "from_negabinary", "zfp_encode_planes", "zfp_decode_planes", "DTYPE_F32", "DTYPE_F64", "LINF", "L2", "L2_STAT", "ABS", "REL",
]

DTYPE_F32, DTYPE_F64 = 0, 1
LINF, L2, L2_STAT = 0, 1, 2
ABS, REL = 0, 1

_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        sz = C.POINTER(C.c_size_t)
        dp = C.POINTER(C.c_double)
        u8 = C.POINTER(C.c_uint8)
        u16 = C.POINTER(C.c_uint16)
        u32 = C.POINTER(C.c_uint32)
        u64 = C.POINTER(C.c_uint64)
        i64 = C.POINTER(C.c_int64)
        sig = {
            "oracle_levels": [C.c_int, sz, C.POINTER(C.c_int), sz],
            "oracle_decompose": [C.c_int, sz, dp, dp],
            "oracle_recompose": [C.c_int, sz, dp, dp],
            "oracle_decompose_c": [C.c_int, sz, dp, dp, dp],
            "oracle_recompose_c": [C.c_int, sz, dp, dp, dp],
            "oracle_correction_norms_c": [C.c_int, sz, dp, dp],
            "oracle_bins_c": [C.c_int, sz, dp, C.c_double, C.c_double, C.c_double, dp],
            "oracle_bins_l2s_c": [C.c_int, sz, dp, C.c_double, C.c_double, C.c_double, dp],
            "oracle_l2s_weights_c": [C.c_int, sz, dp, dp, dp],
            "oracle_recompose_adjoint": [C.c_int, sz, dp, dp],
            "oracle_recompose_adjoint_c": [C.c_int, sz, dp, dp, dp],
            "oracle_decompose_adjoint_c": [C.c_int, sz, dp, dp, dp],
            "oracle_decompose_adjoint": [C.c_int, sz, dp, dp],
            "oracle_correction_norms": [C.c_int, sz, dp],
            "oracle_bins": [C.c_int, sz, C.c_double, C.c_double, C.c_double, dp],
            "oracle_quantize": [C.c_int, sz, dp, dp, C.c_int, C.c_uint32, u16, u64, u64, i64,
                                C.c_uint64],
            "oracle_dequantize": [C.c_int, sz, u16, dp, C.c_uint32, C.c_uint64, u64, i64, dp],
            "oracle_histogram": [u16, C.c_uint64, C.c_uint32, u64],
            "oracle_code_lengths": [u64, C.c_uint32, u8],
            "oracle_canonical_codes": [u8, C.c_uint32, u64],
            "oracle_encode": [u16, C.c_uint64, u8, u64, C.c_uint32, i64, C.c_int, u32, C.c_uint64, u64,
                              u64],
            "oracle_decode": [u32, C.c_uint64, u64, C.c_uint64, C.c_uint32, u8, C.c_uint32, u16,
                              C.c_int, i64, C.c_uint64, u64],
            "oracle_escape_bits": [C.c_int64],
            "oracle_compress_c": [C.c_int, sz, dp, dp, C.c_int, C.c_double, C.c_int, C.c_int,
                                  C.c_uint32, C.c_uint32, C.POINTER(C.c_uint8), C.c_uint64,
                                  C.POINTER(C.c_uint64)],
            "oracle_compress": [C.c_int, sz, dp, C.c_int, C.c_double, C.c_int, C.c_int,
                                C.c_uint32, C.c_uint32, u8, C.c_uint64, u64],
            "oracle_decompress": [u8, C.c_uint64, dp, C.c_uint64],
            "oracle_inspect": [u8, C.c_uint64, C.POINTER(C.c_int), C.POINTER(C.c_int), u64],
        }
        for name, args in sig.items():
            f = getattr(_lib, name)
            f.argtypes = args
            f.restype = C.c_int
        _lib.oracle_compress_bound.argtypes = [C.c_int, sz, C.c_uint32, C.c_uint32]
        _lib.oracle_compress_bound.restype = C.c_uint64
        _lib.oracle_crc32.argtypes = [u8, C.c_uint64]
        _lib.oracle_zfp_bound.argtypes = [C.c_int, sz, C.c_int, C.c_uint32]
        _lib.oracle_zfp_bound.restype = C.c_uint64
        _lib.oracle_zfp_compress.argtypes = [C.c_int, sz, dp, C.c_int, C.c_uint32, u8, C.c_uint64, u64]
        _lib.oracle_zfp_compress.restype = C.c_int
        _lib.oracle_zfp_decompress.argtypes = [u8, C.c_uint64, dp, C.c_uint64]
        _lib.oracle_zfp_decompress.restype = C.c_int
        _lib.oracle_zfp_fwd_line.argtypes = [i64, C.c_int]
        _lib.oracle_zfp_fwd_line.restype = None
        _lib.oracle_zfp_inv_line.argtypes = [i64, C.c_int]
        _lib.oracle_zfp_inv_line.restype = None
        _lib.oracle_zfp_order.argtypes = [C.c_int, C.POINTER(C.c_int)]
        _lib.oracle_zfp_order.restype = None
        _lib.oracle_negabinary.argtypes = [C.c_int64, C.c_int]
        _lib.oracle_negabinary.restype = C.c_uint64
        _lib.oracle_from_negabinary.argtypes = [C.c_uint64, C.c_int]
        _lib.oracle_from_negabinary.restype = C.c_int64
        _lib.oracle_zfp_encode_planes.argtypes = [u64, C.c_int, C.c_int, u32, C.c_uint64, C.c_uint64]
        _lib.oracle_zfp_encode_planes.restype = None
        _lib.oracle_zfp_decode_planes.argtypes = [u64, C.c_int, C.c_int, u32, C.c_uint64, C.c_uint64]
        _lib.oracle_zfp_decode_planes.restype = None
        _lib.oracle_crc32.restype = C.c_uint32
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _zdims(shape):
    """dims of a fixed-rate ZFP field: 1..3 sizes, each >= 1"""
    d = len(shape)
    if not 1 <= d <= 3 or any(int(s) < 1 for s in shape):
        raise ValueError("dims must be 1..3 sizes, each >= 1: %r" % (shape,))
    return d, (C.c_size_t * 3)(*[int(s) for s in shape] + [1] * (3 - d))


def _dims(shape):
    d = len(shape)
    if not 1 <= d <= 3 or any(int(s) < 2 for s in shape):
        raise ValueError("dims must be 1..3 sizes, each >= 2: %r" % (shape,))
    return d, (C.c_size_t * 3)(*[int(s) for s in shape] + [1] * (3 - d))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("%s failed with status %d" % (what, rc))


def levels(shape):
    """Return (L, m) with m[k][l] the node count of dim k on level l."""
    d, dims = _dims(shape)
    L = C.c_int()
    _check(_L().oracle_levels(d, dims, C.byref(L), None), "levels")
    m = np.zeros(3 * (L.value + 1), dtype=np.uint64)
    _check(_L().oracle_levels(d, dims, C.byref(L), m.ctypes.data_as(C.POINTER(C.c_size_t))),
           "levels")
    return L.value, m.reshape(3, L.value + 1)[:d].astype(np.int64)


def level_sizes(shape):
    """Node count N_l of every level l = 0..L (N_L = number of elements)."""
    L, m = levels(shape)
    return [int(np.prod(m[:, l])) for l in range(L + 1)]


def _field_op(fn, x, shape, what):
    d, dims = _dims(shape)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    if x.size != int(np.prod(shape)):
        raise ValueError("size mismatch")
    out = np.empty_like(x)
    _check(fn(d, dims, _p(x, C.c_double), _p(out, C.c_double)), what)
    return out


def _coords(shape, coords):
    """Concatenated node coordinates (dimension 0 first) or None; accepts a
    sequence of per-dimension arrays or one flat array."""
    if coords is None:
        return None
    if isinstance(coords, (list, tuple)):
        if len(coords) != len(shape) or any(len(c) != n for c, n in zip(coords, shape)):
            raise ValueError("one coordinate array per dimension, of the dimension's length")
        coords = np.concatenate([np.asarray(c, dtype=np.float64) for c in coords])
    coords = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1)
    if coords.size != int(sum(shape)):
        raise ValueError("coords must hold sum(shape) values")
    return coords


def decompose(u, coords=None):
    """Level-major coefficient stream (FP64) of the field u (Alg. 1); coords:
    node coordinates of every dimension (default: node i at coordinate i)."""
    u = np.asarray(u)
    co = _coords(u.shape, coords)
    if co is None:
        return _field_op(_L().oracle_decompose, u, u.shape, "decompose")
    return _field_op(lambda d, dims, x, o: _L().oracle_decompose_c(d, dims, _p(co, C.c_double), x, o),
                     u, u.shape, "decompose")


def recompose(coef, shape, coords=None):
    co = _coords(shape, coords)
    if co is None:
        return _field_op(_L().oracle_recompose, coef, shape, "recompose").reshape(shape)
    return _field_op(lambda d, dims, x, o: _L().oracle_recompose_c(d, dims, _p(co, C.c_double), x, o),
                     coef, shape, "recompose").reshape(shape)


def recompose_adjoint(g_u, coords=None):
    g_u = np.asarray(g_u)
    co = _coords(g_u.shape, coords)
    if co is None:
        return _field_op(_L().oracle_recompose_adjoint, g_u, g_u.shape, "recompose_adjoint")
    return _field_op(lambda d, dims, x, o: _L().oracle_recompose_adjoint_c(d, dims, _p(co, C.c_double), x, o),
                     g_u, g_u.shape, "recompose_adjoint")


def decompose_adjoint(g_coef, shape, coords=None):
    co = _coords(shape, coords)
    if co is None:
        return _field_op(_L().oracle_decompose_adjoint, g_coef, shape, "decompose_adjoint").reshape(shape)
    return _field_op(lambda d, dims, x, o: _L().oracle_decompose_adjoint_c(d, dims, _p(co, C.c_double), x, o),
                     g_coef, shape, "decompose_adjoint").reshape(shape)


def correction_norms(shape, coords=None):
    d, dims = _dims(shape)
    L, _ = levels(shape)
    c = np.zeros(L + 1)
    co = _coords(shape, coords)
    _check(_L().oracle_correction_norms_c(d, dims, None if co is None else _p(co, C.c_double),
                                          _p(c, C.c_double)), "correction_norms")
    return c


def bins_l2s(shape, tau_abs, norm_inf, eps, coords=None):
    """Statistical L2 bins (mode 2): q_l = sqrt(12 tau'^2 T / ((L+1) S_l))."""
    d, dims = _dims(shape)
    L, _ = levels(shape)
    q = np.zeros(L + 1)
    co = _coords(shape, coords)
    _check(_L().oracle_bins_l2s_c(d, dims, None if co is None else _p(co, C.c_double), float(tau_abs),
                                  float(norm_inf), float(eps), _p(q, C.c_double)), "bins_l2s")
    return q


def l2s_weights(shape, coords=None):
    """(S[0..L], T): the mass-matrix diagonal summed over each level's new
    nodes (all of level 0's), and over all finest nodes."""
    d, dims = _dims(shape)
    L, _ = levels(shape)
    S = np.zeros(L + 1)
    T = np.zeros(1)
    co = _coords(shape, coords)
    _check(_L().oracle_l2s_weights_c(d, dims, None if co is None else _p(co, C.c_double), _p(S, C.c_double),
                                     _p(T, C.c_double)), "l2s_weights")
    return S, float(T[0])


def bins(shape, tau_abs, norm_inf, eps, coords=None):
    d, dims = _dims(shape)
    L, _ = levels(shape)
    q = np.zeros(L + 1)
    co = _coords(shape, coords)
    _check(_L().oracle_bins_c(d, dims, None if co is None else _p(co, C.c_double), float(tau_abs),
                              float(norm_inf), float(eps), _p(q, C.c_double)), "bins")
    return q


def quantize(coef, shape, q, D=8192, precision=64):
    """Symbols (uint16) and outliers (stream index, code) of a coefficient stream."""
    d, dims = _dims(shape)
    coef = np.ascontiguousarray(coef, dtype=np.float64).reshape(-1)
    q = np.ascontiguousarray(q, dtype=np.float64)
    sym = np.empty(coef.size, dtype=np.uint16)
    nout = C.c_uint64()
    _check(_L().oracle_quantize(d, dims, _p(coef, C.c_double), _p(q, C.c_double), precision, D,
                                _p(sym, C.c_uint16), C.byref(nout), None, None, 0), "quantize")
    idx = np.zeros(max(nout.value, 1), dtype=np.uint64)
    k = np.zeros(max(nout.value, 1), dtype=np.int64)
    _check(_L().oracle_quantize(d, dims, _p(coef, C.c_double), _p(q, C.c_double), precision, D,
                                _p(sym, C.c_uint16), C.byref(nout), _p(idx, C.c_uint64),
                                _p(k, C.c_int64), nout.value), "quantize")
    return sym, idx[:nout.value], k[:nout.value]


def dequantize(sym, shape, q, D, out_idx, out_k):
    d, dims = _dims(shape)
    sym = np.ascontiguousarray(sym, dtype=np.uint16)
    q = np.ascontiguousarray(q, dtype=np.float64)
    out_idx = np.ascontiguousarray(out_idx, dtype=np.uint64)
    out_k = np.ascontiguousarray(out_k, dtype=np.int64)
    coef = np.empty(sym.size)
    _check(_L().oracle_dequantize(d, dims, _p(sym, C.c_uint16), _p(q, C.c_double), D,
                                  out_idx.size, _p(out_idx, C.c_uint64), _p(out_k, C.c_int64),
                                  _p(coef, C.c_double)), "dequantize")
    return coef


def histogram(sym, D):
    sym = np.ascontiguousarray(sym, dtype=np.uint16)
    h = np.zeros(D, dtype=np.uint64)
    _check(_L().oracle_histogram(_p(sym, C.c_uint16), sym.size, D, _p(h, C.c_uint64)), "histogram")
    return h


def code_lengths(hist):
    hist = np.ascontiguousarray(hist, dtype=np.uint64)
    ln = np.zeros(hist.size, dtype=np.uint8)
    _check(_L().oracle_code_lengths(_p(hist, C.c_uint64), hist.size, _p(ln, C.c_uint8)),
           "code_lengths")
    return ln


def canonical_codes(lengths):
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    code = np.zeros(lengths.size, dtype=np.uint64)
    _check(_L().oracle_canonical_codes(_p(lengths, C.c_uint8), lengths.size,
                                       _p(code, C.c_uint64)), "canonical_codes")
    return code


def encode(sym, lengths, K=1024, esc_k=None, esc_width=None):
    """Huffman-encode symbols: returns (words uint32, chunk table uint64, total bits).
    esc_k: None for plain symbols; else the integer codes of the escapes (symbol 0)
    in stream order, each written after its codeword as zigzag(k) in esc_width
    bits (default: the largest bit length among them)."""
    sym = np.ascontiguousarray(sym, dtype=np.uint16)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    code = canonical_codes(lengths)
    bits = int(lengths[sym].astype(np.uint64).sum())
    ek, ew = None, 0
    if esc_k is not None:
        ek = np.ascontiguousarray(esc_k, dtype=np.int64)
        ew = escape_width(ek) if esc_width is None else int(esc_width)
        bits += int(ek.size) * ew
        if ek.size == 0:
            ek = np.zeros(1, dtype=np.int64)
    nw = (bits + 31) // 32
    words = np.zeros(max(nw, 1), dtype=np.uint32)
    nch = (sym.size + K - 1) // K
    chunk = np.zeros(max(nch, 1), dtype=np.uint64)
    tb = C.c_uint64()
    _check(_L().oracle_encode(_p(sym, C.c_uint16), sym.size, _p(lengths, C.c_uint8),
                              _p(code, C.c_uint64), K, _p(ek, C.c_int64) if ek is not None else None,
                              ew, _p(words, C.c_uint32), words.size, _p(chunk, C.c_uint64),
                              C.byref(tb)), "encode")
    return words[:nw], chunk[:nch], tb.value


def escape_width(esc_k):
    """Largest bit length of zigzag(k) over the escapes (|k| < 2^62); 0 if none."""
    k = np.asarray(esc_k, dtype=np.int64)
    if k.size == 0:
        return 0
    z = np.where(k >= 0, 2 * k.astype(np.uint64), 2 * (-(k + 1)).astype(np.uint64) + 1)
    return int(max(int(x).bit_length() for x in (z.max(),)))


def decode(words, chunk, N, K, lengths, esc_width=None):
    """Decode N symbols.  With esc_width given (a container stream, symbol 0
    the quantizer's escape) also returns the escapes' codes in stream order,
    each read as zigzag(k) in esc_width bits (0: the stream has no escapes)."""
    words = np.ascontiguousarray(words, dtype=np.uint32)
    chunk = np.ascontiguousarray(chunk, dtype=np.uint64)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    sym = np.zeros(N, dtype=np.uint16)
    ek = np.zeros(max(N, 1), dtype=np.int64)
    ne = C.c_uint64()
    w = words if words.size else np.zeros(1, dtype=np.uint32)
    _check(_L().oracle_decode(_p(w, C.c_uint32), words.size, _p(chunk, C.c_uint64), N, K,
                              _p(lengths, C.c_uint8), lengths.size, _p(sym, C.c_uint16),
                              int(esc_width or 0), _p(ek, C.c_int64), ek.size, C.byref(ne)),
           "decode")
    if esc_width is not None:
        return sym, ek[:ne.value].copy()
    return sym


def compress_bound(shape, D=8192, K=1024):
    d, dims = _dims(shape)
    return int(_L().oracle_compress_bound(d, dims, D, K))


def compress(u, tol, tol_kind=REL, mode=LINF, D=8192, K=1024, dtype=None, coords=None):
    """Container bytes of the field u (dtype defaults to u's own: f32 or f64);
    coords: node coordinates (recorded in the container)."""
    u = np.asarray(u)
    if dtype is None:
        dtype = DTYPE_F32 if u.dtype == np.float32 else DTYPE_F64
    d, dims = _dims(u.shape)
    x = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    cap = compress_bound(u.shape, D, K)
    out = np.zeros(cap, dtype=np.uint8)
    nb = C.c_uint64()
    co = _coords(u.shape, coords)
    _check(_L().oracle_compress_c(d, dims, None if co is None else _p(co, C.c_double), _p(x, C.c_double),
                                  dtype, float(tol), tol_kind, mode, D, K, _p(out, C.c_uint8), cap,
                                  C.byref(nb)), "compress")
    return out[:nb.value].copy()


def inspect(buf):
    buf = np.ascontiguousarray(np.frombuffer(bytes(buf), dtype=np.uint8))
    dt, d = C.c_int(), C.c_int()
    dims = np.zeros(3, dtype=np.uint64)
    _check(_L().oracle_inspect(_p(buf, C.c_uint8), buf.size, C.byref(dt), C.byref(d),
                               _p(dims, C.c_uint64)), "inspect")
    return dt.value, tuple(int(x) for x in dims[:d.value])


def decompress(buf):
    """FP64 reconstruction of a container (shape from the header)."""
    buf = np.ascontiguousarray(np.frombuffer(bytes(buf), dtype=np.uint8))
    _, shape = inspect(buf)
    n = int(np.prod(shape))
    u = np.empty(n)
    _check(_L().oracle_decompress(_p(buf, C.c_uint8), buf.size, _p(u, C.c_double), n),
           "decompress")
    return u.reshape(shape)


# ---- fixed-rate ZFP (Alg. 3) ---------------------------------------------

def zfp_bound(shape, rate, dtype=DTYPE_F32):
    d, dims = _zdims(shape)
    return int(_L().oracle_zfp_bound(d, dims, int(dtype), int(rate)))


def zfp_compress(u, rate, dtype=None):
    """Fixed-rate container bytes of u (dtype defaults to u's: f32 or f64)."""
    u = np.asarray(u)
    if dtype is None:
        dtype = DTYPE_F32 if u.dtype == np.float32 else DTYPE_F64
    d, dims = _zdims(u.shape)
    x = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    cap = zfp_bound(u.shape, rate, dtype)
    if cap == 0:
        raise ValueError("zfp: invalid rate %r for %d dimensions" % (rate, d))
    out = np.zeros(cap, dtype=np.uint8)
    nb = C.c_uint64()
    _check(_L().oracle_zfp_compress(d, dims, _p(x, C.c_double), int(dtype), int(rate), _p(out, C.c_uint8), cap,
                                    C.byref(nb)), "zfp_compress")
    return out[:nb.value].copy()


def zfp_decompress(buf):
    b = np.ascontiguousarray(np.frombuffer(bytes(buf), dtype=np.uint8))
    d = int.from_bytes(bytes(b[12:16]), "little")
    shape = tuple(int.from_bytes(bytes(b[16 + 8 * k:24 + 8 * k]), "little") for k in range(d))
    u = np.empty(int(np.prod(shape)))
    _check(_L().oracle_zfp_decompress(_p(b, C.c_uint8), b.size, _p(u, C.c_double), u.size), "zfp_decompress")
    return u.reshape(shape)


def zfp_fwd_line(a):
    x = np.ascontiguousarray(a, dtype=np.int64).copy()
    _L().oracle_zfp_fwd_line(_p(x, C.c_int64), 1)
    return x


def zfp_inv_line(a):
    x = np.ascontiguousarray(a, dtype=np.int64).copy()
    _L().oracle_zfp_inv_line(_p(x, C.c_int64), 1)
    return x


def zfp_order(d):
    perm = (C.c_int * (4 ** d))()
    _L().oracle_zfp_order(d, perm)
    return list(perm)


def negabinary(q, P):
    return int(_L().oracle_negabinary(int(q), int(P)))


def from_negabinary(u, P):
    return int(_L().oracle_from_negabinary(int(u), int(P)))


def zfp_encode_planes(u, P, maxbits):
    u = np.ascontiguousarray(u, dtype=np.uint64)
    w = np.zeros((maxbits + 31) // 32, dtype=np.uint32)
    _L().oracle_zfp_encode_planes(_p(u, C.c_uint64), u.size, P, _p(w, C.c_uint32), 0, maxbits)
    return w


def zfp_decode_planes(words, B, P, maxbits):
    w = np.ascontiguousarray(words, dtype=np.uint32)
    u = np.zeros(B, dtype=np.uint64)
    _L().oracle_zfp_decode_planes(_p(u, C.c_uint64), B, P, _p(w, C.c_uint32), 0, maxbits)
    return u


def crc32(data):
    b = np.ascontiguousarray(np.frombuffer(bytes(data), dtype=np.uint8))
    return int(_L().oracle_crc32(_p(b, C.c_uint8), b.size))


def parse_header(buf):
    """Header fields and section views of a version-3 container (plain byte reads)."""
    b = bytes(buf)
    u32 = lambda o: int.from_bytes(b[o:o + 4], "little")  # noqa: E731
    u64 = lambda o: int.from_bytes(b[o:o + 8], "little")  # noqa: E731
    f64 = lambda o: float(np.frombuffer(b[o:o + 8], dtype="<f8")[0])  # noqa: E731
    h = dict(magic=b[:4], version=u32(4), dtype=u32(8), ndim=u32(12),
             dims=tuple(u64(16 + 8 * k) for k in range(u32(12))), L=u32(40), mode=u32(44),
             tol_kind=u32(48) & 0xFF, has_coords=bool(u32(48) & 0x100), D=u32(52), K=u32(56),
             s_lo=u32(60), tol=f64(64),
             tau_abs=f64(72), norm_inf=f64(80), norm_rms=f64(88), N=u64(96),
             n_escapes=u64(104), total_bits=u64(112), s_hi=u32(120) & 0xFFFF,
             esc_width=(u32(120) >> 16) & 0xFF, crc=u32(124))
    a16 = lambda x: (x + 15) & ~15  # noqa: E731
    L = h["L"]
    off_q = 128
    nco = sum(h["dims"]) if h["has_coords"] else 0
    off_co = off_q + 8 * (L + 1)
    off_len = a16(off_co + 8 * nco)
    off_chunk = a16(off_len + h["s_hi"] - h["s_lo"] + 1)
    nch = (h["N"] + h["K"] - 1) // h["K"]
    off_bits = a16(off_chunk + 8 * nch)
    nw = (h["total_bits"] + 31) // 32
    arr = np.frombuffer(b, dtype=np.uint8)
    h["q"] = arr[off_q:off_q + 8 * (L + 1)].view("<f8").copy()
    h["coords"] = arr[off_co:off_co + 8 * nco].view("<f8").copy() if nco else None
    ln = np.zeros(h["D"], dtype=np.uint8)
    ln[h["s_lo"]:h["s_hi"] + 1] = arr[off_len:off_len + h["s_hi"] - h["s_lo"] + 1]
    h["lengths"] = ln
    h["chunk"] = arr[off_chunk:off_chunk + 8 * nch].view("<u8").copy()
    h["words"] = arr[off_bits:off_bits + 4 * nw].view("<u4").copy()
    h["total_bytes"] = off_bits + 4 * nw
    return h
