"""Argument checks of the Python binding, without a GPU.

Several C entry points take no size for a buffer whose element count follows
from the shape (hpdr_decompose, hpdr_recompose, the adjoints, the Huffman
decoder), so the binding checks every tensor before the call: a tensor that
is too small, of the wrong type, not contiguous or on the wrong side (host or
device) raises here instead of reaching a kernel.  The checks are plain
Python; they run on CPU tensors with the CUDA-tensor test replaced by a
contiguity test, and every failing case raises before the library is used."""
import pytest
import torch

from paper_2503_06322_gb300 import hpdr


@pytest.fixture
def cpu_as_device(monkeypatch):
    """Let CPU tensors stand for device tensors, and make any use of the
    library an error: the checks must decide before it is reached."""
    def as_dev(t, what):
        if not (isinstance(t, torch.Tensor) and t.is_contiguous()):
            raise TypeError("%s must be a contiguous CUDA tensor" % what)
        return t

    def no_lib():
        raise AssertionError("the library was reached")

    monkeypatch.setattr(hpdr, "_dev_tensor", as_dev)
    monkeypatch.setattr(hpdr, "lib", no_lib)
    return hpdr


def test_missing_library_is_an_error(monkeypatch, tmp_path):
    monkeypatch.setattr(hpdr, "LIB_PATH", str(tmp_path / "libhpdr.so"))
    monkeypatch.setattr(hpdr, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        hpdr.lib()


@pytest.mark.parametrize("call", [
    lambda: hpdr.hpdr_compress(torch.zeros(9, 9), 1e-3),
    lambda: hpdr.hpdr_decompress(torch.zeros(300, dtype=torch.uint8)),
    lambda: hpdr.hpdr_decompose(torch.zeros(9, 9)),
    lambda: hpdr.hpdr_recompose(torch.zeros(81), (9, 9)),
    lambda: hpdr.hpdr_recompose_adjoint(torch.zeros(9, 9)),
    lambda: hpdr.hpdr_decompose_adjoint(torch.zeros(81), (9, 9)),
    lambda: hpdr.hpdr_decompose_noalloc(torch.zeros(9, 9)),
    lambda: hpdr.hpdr_huffman_encode(torch.zeros(100, dtype=torch.int16)),
    lambda: hpdr.hpdr_lossless_compress(torch.zeros(100, dtype=torch.uint8)),
    lambda: hpdr.hpdr_zfp_compress(torch.zeros(64), 8),
    lambda: hpdr.hpdr_compress_batched([torch.zeros(9, 9)], [1e-3]),
], ids=["compress", "decompress", "decompose", "recompose", "recompose_adjoint", "decompose_adjoint",
        "noalloc", "huffman_encode", "lossless", "zfp", "batched"])
def test_host_tensors_are_refused_by_device_entries(call):
    with pytest.raises(TypeError, match="CUDA tensor"):
        call()


def test_device_buffer_checks(cpu_as_device):
    H = cpu_as_device
    dev = torch.device("cpu")
    t = torch.zeros(10, dtype=torch.float32)
    assert H._dev_buf(t, "t", dev, torch.float32, 10) is t
    assert H._dev_buf(t, "t", dev, 4, 3) is t
    with pytest.raises(TypeError, match="float64"):
        H._dev_buf(t, "t", dev, torch.float64)
    with pytest.raises(TypeError, match="8-byte"):
        H._dev_buf(t, "t", dev, 8)
    with pytest.raises(ValueError, match="11 are needed"):
        H._dev_buf(t, "t", dev, torch.float32, 11)
    with pytest.raises(ValueError, match="the call runs on"):
        H._dev_buf(t, "t", torch.device("meta"))
    with pytest.raises(TypeError, match="contiguous"):
        H._dev_buf(torch.zeros(4, 4).t(), "t", dev)


def test_shape_mismatches_raise_before_the_call(cpu_as_device):
    H = cpu_as_device
    u = torch.zeros(9, 9)
    with pytest.raises(ValueError, match="80 elements, 81"):
        H.hpdr_decompose(u, out=torch.zeros(80))
    with pytest.raises(TypeError, match="float32"):
        H.hpdr_decompose(u, out=torch.zeros(81, dtype=torch.float64))
    with pytest.raises(ValueError, match="80 elements, 81"):
        H.hpdr_decompose_noalloc(u, out=torch.zeros(80))
    with pytest.raises(ValueError, match="coef holds 80"):
        H.hpdr_recompose(torch.zeros(80), (9, 9))
    with pytest.raises(ValueError, match="80 elements, 81"):
        H.hpdr_recompose(torch.zeros(81), (9, 9), out=torch.zeros(80))
    with pytest.raises(ValueError, match="80 elements, 81"):
        H.hpdr_recompose_adjoint(u, out=torch.zeros(80))
    with pytest.raises(ValueError, match="grad_coef holds 82"):
        H.hpdr_decompose_adjoint(torch.zeros(82), (9, 9))
    with pytest.raises(TypeError, match="uint8"):
        H.hpdr_compress(u, 1e-3, out=torch.zeros(1000))
    with pytest.raises(ValueError, match="result holds 1"):
        H.hpdr_compress_async(u, 1e-3, torch.zeros(1000, dtype=torch.uint8), torch.zeros(1, dtype=torch.int64))
    with pytest.raises(TypeError, match="8-byte"):
        H.hpdr_decompress_async(torch.zeros(1000, dtype=torch.uint8), u, torch.zeros(2, dtype=torch.int32))
    with pytest.raises(TypeError, match="2-byte"):
        H.hpdr_huffman_encode(torch.zeros(100, dtype=torch.int32))
    with pytest.raises(ValueError, match="at least one field"):
        H.hpdr_compress_batched([], [])


def test_huffman_decode_buffers_are_sized(cpu_as_device):
    H = cpu_as_device
    N, K, D, bits = 5000, 1024, 256, 40000
    words = torch.zeros((bits + 31) // 32, dtype=torch.int32)
    chunk = torch.zeros((N + K - 1) // K, dtype=torch.int64)
    lengths = torch.zeros(D, dtype=torch.uint8)
    ok = dict(words=words, total_bits=bits, chunk=chunk, N=N, lengths=lengths, D=D, K=K)
    for key, bad, msg in [("words", words[:-1], "words holds"), ("chunk", chunk[:-1], "chunk holds"),
                          ("lengths", lengths[:-1], "lengths holds"),
                          ("lengths", torch.zeros(D, dtype=torch.int16), "uint8"),
                          ("chunk", torch.zeros(5, dtype=torch.int32), "8-byte"),
                          ("out", torch.zeros(N - 1, dtype=torch.int16), "out holds")]:
        kw = dict(ok)
        kw[key] = bad
        with pytest.raises((TypeError, ValueError), match=msg):
            H.hpdr_huffman_decode(**kw)
    with pytest.raises(AssertionError, match="library was reached"):
        H.hpdr_huffman_decode(**ok)     # every check passes: the next step is the library


def test_host_streamed_buffers_are_host_tensors(cpu_as_device):
    H = cpu_as_device
    with pytest.raises(TypeError, match="CPU tensor"):
        H._host_buf(torch.zeros(4, 4).t(), "out")
    with pytest.raises(H.HpdrError):
        H.hpdr_decompress_host_streamed(torch.zeros(10, dtype=torch.uint8))
