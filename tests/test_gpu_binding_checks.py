"""The binding's buffer checks on real device tensors: a tensor that the
library would read or write past its end, or one of the wrong type or on the
wrong side, raises before the call, and the context stays usable."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2503_06322_gb300 import hpdr
    hpdr.lib()
    return hpdr


def test_device_buffers_are_checked(H):
    dev = torch.device("cuda:0")
    u = torch.randn(33, 17, device=dev)
    with pytest.raises(ValueError):
        H.hpdr_decompose(u, out=torch.empty(u.numel() - 1, device=dev))
    with pytest.raises(TypeError):
        H.hpdr_decompose(u, out=torch.empty(u.numel(), dtype=torch.float64, device=dev))
    with pytest.raises(ValueError):
        H.hpdr_recompose(torch.empty(u.numel() - 1, device=dev), u.shape)
    with pytest.raises(TypeError):
        H.hpdr_decompose(u, out=torch.empty(u.numel()))              # a host tensor
    buf = H.hpdr_compress(u, 1e-3).clone()
    with pytest.raises(TypeError):
        H.hpdr_decompress(buf, out=torch.empty(u.shape, dtype=torch.float64, device=dev))
    with pytest.raises(ValueError):
        H.hpdr_decompress(buf, out=torch.empty(u.numel() - 1, device=dev))
    lengths, chunk, words, bits = H.hpdr_huffman_encode(torch.randint(0, 200, (5000,), dtype=torch.int16,
                                                                     device=dev), D=256)
    with pytest.raises(ValueError):
        H.hpdr_huffman_decode(words[:-1], bits, chunk, 5000, lengths, D=256)
    with pytest.raises(TypeError):
        H.hpdr_compress_host_streamed(u.cpu(), 1e-3, out=torch.empty(1 << 20, dtype=torch.uint8, device=dev))
    # valid calls still work after the refusals
    c = H.hpdr_decompose(u)
    assert torch.allclose(H.hpdr_recompose(c, u.shape), u, atol=1e-5)
    r = H.hpdr_decompress(buf)
    assert (r - u).abs().max().item() <= 1e-3 * u.abs().max().item()
    dec = H.hpdr_huffman_decode(words, bits, chunk, 5000, lengths, D=256)
    assert dec.numel() == 5000
