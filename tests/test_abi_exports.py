"""The C ABI library loads without a GPU and exports every entry point that
include/hpdr.h declares.  Only host-side entries are called (no device work):
the status strings, the launch counter and the container size bound."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "hpdr.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w ]*?[\s*]+(hpdr_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_06322_gb300 import build
    path = build.build()       # no-op when up to date; nvcc cross-compiles without a GPU
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("hpdr_compress", "hpdr_decompress", "hpdr_recompose_adjoint", "hpdr_decompose",
                 "hpdr_recompose", "hpdr_decompose_adjoint", "hpdr_compress_batched",
                 "hpdr_compress_host_streamed", "hpdr_decompress_host_streamed",
                 "hpdr_huffman_encode", "hpdr_huffman_decode", "hpdr_inspect",
                 "hpdr_compress_bound", "hpdr_ctx_create", "hpdr_ctx_destroy",
                 "hpdr_status_string", "hpdr_decompose_noalloc"):
        assert must in names, must


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entries(lib):
    lib.hpdr_status_string.restype = C.c_char_p
    lib.hpdr_status_string.argtypes = [C.c_int]
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert lib.hpdr_status_string(code)
    lib.hpdr_launch_count.restype = C.c_ulonglong
    assert lib.hpdr_launch_count() >= 0
    lib.hpdr_compress_bound.restype = C.c_size_t
    lib.hpdr_compress_bound.argtypes = [C.c_int, C.POINTER(C.c_size_t), C.c_int, C.c_void_p]
    dims = (C.c_size_t * 3)(65, 65, 65)
    b32 = lib.hpdr_compress_bound(3, dims, 0, None)
    b64 = lib.hpdr_compress_bound(3, dims, 1, None)
    # at least the header plus ceil(log2 D) = 13 bits per symbol, and finite
    assert 128 + 65 ** 3 * 13 // 8 <= b32 <= b64 < 64 * 65 ** 3
    bad = (C.c_size_t * 3)(65, 1, 65)
    assert lib.hpdr_compress_bound(3, bad, 0, None) == 0


def test_zfp_bound_matches_the_oracle(lib):
    """The fixed-rate container size is exact and host-only: it must equal the
    oracle's for every dimension count, type and rate, and both must reject
    the same rates (rate * 4^d not a multiple of 32, or out of 1..256)."""
    import oracle
    lib.hpdr_zfp_bound.restype = C.c_size_t
    lib.hpdr_zfp_bound.argtypes = [C.c_int, C.POINTER(C.c_size_t), C.c_int, C.c_uint32]
    for shape in [(1,), (7,), (1000,), (5, 9), (65, 33), (1, 1, 1), (33, 17, 9), (513, 513, 513)]:
        dims = (C.c_size_t * 3)(*(list(shape) + [1] * (3 - len(shape))))
        for dtype in (0, 1):
            for rate in (1, 2, 3, 4, 7, 8, 12, 16, 64, 136, 256, 257, 0):
                got = lib.hpdr_zfp_bound(len(shape), dims, dtype, rate)
                assert got == oracle.zfp_bound(shape, rate, dtype), (shape, dtype, rate)
                if got:
                    nb = 1
                    for s in shape:
                        nb *= (s + 3) // 4
                    assert got == 64 + nb * rate * 4 ** len(shape) // 8
