"""Lossless key compression, the Huffman stage on its own (Sec. IV-B, Alg. 2):
the HPDL container's code lengths, chunk table and bitstream equal the
oracle's encoding of the same keys, byte for byte; the oracle decodes the
container's stream; round trips; a single key, one repeated key, every 16-bit
key; corrupted and truncated containers; short buffers."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _parse(buf):
    b = buf.cpu().numpy()
    hdr = b[:64].tobytes()
    u32 = lambda o: int.from_bytes(hdr[o:o + 4], "little")  # noqa: E731
    u64 = lambda o: int.from_bytes(hdr[o:o + 8], "little")  # noqa: E731
    assert hdr[:4] == b"HPDL" and u32(4) == 1
    kb, D, K = u32(8), u32(12), u32(16)
    n, bits, oc, ob = u64(24), u64(32), u64(40), u64(48)
    nch = -(-n // K)
    assert oc % 16 == 0 and ob % 16 == 0 and ob + 4 * ((bits + 31) // 32) == b.size
    lengths = b[64:64 + D]
    chunk = b[oc:oc + 8 * nch].view(np.uint64)
    words = b[ob:ob + 4 * ((bits + 31) // 32)].view(np.uint32)
    return kb, D, K, n, bits, lengths, chunk, words


def _keys(kind, n, rng):
    if kind == "u8":
        return np.clip(np.round(rng.laplace(128, 6, size=n)), 0, 255).astype(np.uint8)
    if kind == "u8-const":
        return np.full(n, 7, np.uint8)
    if kind == "u8-all":
        return np.tile(np.arange(256, dtype=np.uint8), n // 256)
    if kind == "u16":
        # negative codes wrap to the top of the range, so keys 0 and 65535 both occur
        return (np.round(rng.laplace(0, 40, size=n)).astype(np.int64) % 65536).astype(np.uint16)
    return np.tile(np.arange(65536, dtype=np.uint16), n // 65536)


@pytest.mark.parametrize("n,kind,K", [(1_000_003, "u8", 0), (1, "u8", 0), (5000, "u8-const", 128),
                                      (256 * 40, "u8-all", 256), (300_001, "u16", 0),
                                      (65536 * 3, "u16-all", 1024), (131072, "u16", 128)], ids=str)
def test_lossless_bit_exact_and_round_trip(oracle, n, kind, K):
    from paper_2503_06322_gb300 import hpdr
    keys = _keys(kind, n, np.random.default_rng(n))
    D = 256 if keys.dtype == np.uint8 else 65536
    t = torch.from_numpy(keys if keys.dtype == np.uint8 else keys.view(np.int16)).cuda()
    buf = hpdr.hpdr_lossless_compress(t, K=K)
    kb, Dh, Kh, nh, bits, lengths, chunk, words = _parse(buf)
    assert (kb, Dh, nh) == (keys.itemsize, D, n) and (K == 0 or Kh == K)
    k16 = keys.astype(np.uint16)
    ln = oracle.code_lengths(oracle.histogram(k16, D))
    w_ref, c_ref, b_ref = oracle.encode(k16, ln, K=Kh)
    assert np.array_equal(lengths, ln) and bits == b_ref
    assert np.array_equal(chunk, c_ref) and np.array_equal(words, w_ref)
    assert np.array_equal(oracle.decode(words, chunk, n, Kh, lengths), k16)
    back = hpdr.hpdr_lossless_decompress(buf).cpu().numpy()
    assert np.array_equal(back if keys.dtype == np.uint8 else back.view(np.uint16), keys)


def test_lossless_errors():
    from paper_2503_06322_gb300 import hpdr
    keys = torch.randint(0, 256, (10000,), dtype=torch.uint8, device="cuda")
    buf = hpdr.hpdr_lossless_compress(keys)
    bad = buf.clone()
    bad[16] ^= 1                       # the chunk size field: the CRC no longer matches
    with pytest.raises(hpdr.HpdrError) as e:
        hpdr.hpdr_lossless_decompress(bad)
    assert e.value.status == -4
    with pytest.raises(hpdr.HpdrError) as e:
        hpdr.hpdr_lossless_decompress(buf[:-4])
    assert e.value.status == -4
    with pytest.raises(hpdr.HpdrError) as e:
        hpdr.hpdr_lossless_compress(keys, out=torch.empty(200, dtype=torch.uint8, device="cuda"))
    assert e.value.status == -3
    with pytest.raises(hpdr.HpdrError) as e:
        hpdr.hpdr_lossless_decompress(buf, out=torch.empty(9999, dtype=torch.uint8, device="cuda"))
    assert e.value.status == -3
    assert torch.equal(hpdr.hpdr_lossless_decompress(buf), keys)
