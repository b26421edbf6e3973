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
