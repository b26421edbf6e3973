"""GPU path against the FP64 oracle, element by element, through the C ABI.

Tolerances (the bar stated for this path):
  * decomposition coefficients: 1e-5 x max|coef| (FP32 data), 1e-12 (FP64);
  * quantization codes on identical inputs (the oracle quantizes the GPU's own
    coefficients with the container's bins, deciding in binary64): equal
    except at half-bin ties, at most 1e-5 of the elements;
  * Huffman encoder and decoder on the oracle's codes: bit-exact;
  * every reconstruction within the requested bound.
"""
import numpy as np
import pytest
import torch
from _codes import assert_codes_match_fp64

pytestmark = pytest.mark.gpu

SHAPES = [(2,), (3,), (33,), (1000,), (3, 2), (6, 5), (129, 129), (65, 33), (500, 50),
          (6, 5, 4), (9, 6, 5), (33, 17, 9), (70, 70, 70), (100, 7, 5), (65, 65, 65),
          (17, 100, 41), (300, 200), (100, 60, 40)]


@pytest.fixture(scope="module")
def H():
    from paper_2503_06322_gb300 import hpdr
    return hpdr


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def _field(shape, seed, dtype):
    from paper_2503_06322_gb300 import fields
    if len(shape) == 1:
        return (np.random.default_rng(seed).standard_normal(shape) * 2 + 0.5).astype(dtype)
    return fields.powerlaw_field(shape, seed=seed, dtype=dtype)


@pytest.mark.parametrize("shape", SHAPES, ids=str)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_decompose_parity(oracle, H, dev, shape, dtype):
    u = _field(shape, 1, dtype)
    got = H.hpdr_decompose(torch.from_numpy(u).to(dev)).cpu().numpy().astype(np.float64)
    ref = oracle.decompose(u.astype(np.float64))
    tol = 1e-5 if dtype == np.float32 else 1e-12
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("shape", SHAPES, ids=str)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_recompose_parity_and_identity(oracle, H, dev, shape, dtype):
    u = _field(shape, 2, dtype)
    coef = oracle.decompose(u.astype(np.float64))
    ct = torch.from_numpy(coef.astype(dtype)).to(dev)
    got = H.hpdr_recompose(ct, shape).cpu().numpy().astype(np.float64)
    ref = oracle.recompose(coef.astype(dtype).astype(np.float64), shape)
    tol = 1e-5 if dtype == np.float32 else 1e-12
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    ut = torch.from_numpy(u).to(dev)
    back = H.hpdr_recompose(H.hpdr_decompose(ut), shape).cpu().numpy().astype(np.float64)
    assert np.abs(back - u).max() <= tol * np.abs(u).max()


def _decode_container_symbols(oracle, buf):
    h = oracle.parse_header(buf)
    sym, esc = oracle.decode(h["words"], h["chunk"], h["N"], h["K"], h["lengths"], esc_width=h["esc_width"])
    return h, sym, esc


@pytest.mark.parametrize("shape,tol,D", [((129, 129), 1e-3, 8192), ((33, 17, 9), 1e-2, 8192),
                                         ((70, 70, 70), 1e-4, 8192), ((65, 33), 1e-3, 64),
                                         ((100, 7, 5), 1e-3, 8192), ((1000,), 1e-3, 8192),
                                         ((3, 2), 1e-2, 4), ((50000,), 1e-3, 8192), ((9000, 3), 1e-3, 8192)],
                         ids=str)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_codes_on_identical_inputs(oracle, H, dev, shape, tol, D, dtype):
    u = _field(shape, 3, dtype)
    ut = torch.from_numpy(u).to(dev)
    buf = H.hpdr_compress(ut, tol, dict_size=D).cpu().numpy()
    h, sym, esc = _decode_container_symbols(oracle, buf)
    coef = H.hpdr_decompose(ut).cpu().numpy().astype(np.float64)
    assert_codes_match_fp64(oracle, sym, esc, coef, shape, h["q"], D)
    assert h["n_escapes"] == esc.size
    # bins: same definition computed independently (correction norms differ only by rounding)
    eps = 2.0 ** -24 if dtype == np.float32 else 2.0 ** -53
    q_ref = oracle.bins(shape, tol * np.abs(u.astype(np.float64)).max(),
                        np.abs(u.astype(np.float64)).max(), eps)
    assert np.allclose(h["q"], q_ref, rtol=1e-12, atol=0)
    # the whole Huffman part of the container equals the oracle's encoding of its codes
    ln = oracle.code_lengths(oracle.histogram(sym, D))
    words, chunk, bits = oracle.encode(sym, ln, K=h["K"], esc_k=esc)
    assert np.array_equal(h["lengths"], ln)
    assert np.array_equal(h["chunk"], chunk) and h["total_bits"] == bits
    assert np.array_equal(h["words"], words)


@pytest.mark.parametrize("n,D,K,spread", [(20000, 8192, 1024, 300.0), (1, 16, 128, 1.0),
                                          (777, 256, 128, 0.0), (300000, 65536, 1024, 2000.0),
                                          (65536, 8192, 4096, 3.0), (5000, 64, 256, 40.0),
                                          (100000, 8192, 512, 500.0), (300000, 8192, 1024, 3000.0),
                                          # several warp groups of chunks (K < 1024 dividing 1024), ragged tails,
                                          # a K that does not divide 1024, and a one-symbol stream
                                          (100003, 8192, 128, 40.0), (262147, 8192, 256, 0.3),
                                          (50001, 4096, 384, 100.0), (70001, 256, 512, 0.0),
                                          (1048576, 8192, 256, 2.0), (33000, 8192, 512, 8000.0)])
def test_huffman_bit_exact(oracle, H, dev, n, D, K, spread):
    rng = np.random.default_rng(n)
    sym = np.clip(np.round(rng.laplace(D // 2, spread + 1e-9, size=n)), 1, D - 1).astype(np.uint16)
    ln_ref = oracle.code_lengths(oracle.histogram(sym, D))
    words_ref, chunk_ref, bits_ref = oracle.encode(sym, ln_ref, K=K)
    st = torch.from_numpy(sym.view(np.int16)).to(dev)
    ln, chunk, words, bits = H.hpdr_huffman_encode(st, D=D, K=K)
    assert np.array_equal(ln.cpu().numpy(), ln_ref)
    assert bits == bits_ref
    assert np.array_equal(chunk.cpu().numpy().view(np.uint64), chunk_ref)
    assert np.array_equal(words.cpu().numpy().view(np.uint32), words_ref)
    # GPU decodes the oracle's stream
    wt = torch.from_numpy(words_ref.view(np.int32).copy()).to(dev)
    ct = torch.from_numpy(chunk_ref.view(np.int64).copy()).to(dev)
    lt = torch.from_numpy(ln_ref).to(dev)
    dec = H.hpdr_huffman_decode(wt, bits_ref, ct, n, lt, D=D, K=K)
    assert np.array_equal(dec.cpu().numpy().view(np.uint16), sym)


@pytest.mark.parametrize("D,reps", [(8192, 3), (4096, 1), (16, 7)])
def test_huffman_equal_frequencies(oracle, H, dev, D, reps):
    """Every symbol equally frequent: all weights tie, so the order of the
    leaves and the two-queue tie rule decide every pick."""
    sym = np.tile(np.arange(D, dtype=np.uint16), reps)
    K = 1024
    ln_ref = oracle.code_lengths(oracle.histogram(sym, D))
    words_ref, chunk_ref, bits_ref = oracle.encode(sym, ln_ref, K=K)
    ln, chunk, words, bits = H.hpdr_huffman_encode(torch.from_numpy(sym.view(np.int16)).to(dev), D=D, K=K)
    assert np.array_equal(ln.cpu().numpy(), ln_ref) and bits == bits_ref
    assert np.array_equal(words.cpu().numpy().view(np.uint32), words_ref)
    dec = H.hpdr_huffman_decode(words, bits, chunk, sym.size, ln, D=D, K=K)
    assert np.array_equal(dec.cpu().numpy().view(np.uint16), sym)


@pytest.mark.parametrize("nsym,K", [(20, 1024), (35, 2048), (35, 256), (28, 128)])
def test_huffman_long_codewords(oracle, H, dev, nsym, K):
    """Fibonacci frequencies give codewords up to nsym - 1 bits: past the
    decoder's 15-bit table and, for 35 symbols, past 32 bits."""
    fib = [1, 1]
    while len(fib) < nsym:
        fib.append(fib[-1] + fib[-2])
    D = 64
    sym = np.repeat(np.arange(1, nsym + 1, dtype=np.uint16), fib)
    sym = sym[np.random.default_rng(nsym).permutation(sym.size)]
    n = sym.size
    ln_ref = oracle.code_lengths(oracle.histogram(sym, D))
    assert ln_ref.max() == nsym - 1
    words_ref, chunk_ref, bits_ref = oracle.encode(sym, ln_ref, K=K)
    st = torch.from_numpy(sym.view(np.int16)).to(dev)
    ln, chunk, words, bits = H.hpdr_huffman_encode(st, D=D, K=K)
    assert np.array_equal(ln.cpu().numpy(), ln_ref) and bits == bits_ref
    assert np.array_equal(words.cpu().numpy().view(np.uint32), words_ref)
    wt = torch.from_numpy(words_ref.view(np.int32).copy()).to(dev)
    ct = torch.from_numpy(chunk_ref.view(np.int64).copy()).to(dev)
    lt = torch.from_numpy(ln_ref).to(dev)
    dec = H.hpdr_huffman_decode(wt, bits_ref, ct, n, lt, D=D, K=K)
    assert np.array_equal(dec.cpu().numpy().view(np.uint16), sym)


# (129, 129, 129) and (300, 65, 65) give the level kernels segments of more
# planes than their ring of stages holds, so every stage is reused
@pytest.mark.parametrize("shape,tol,kind,mode", [((129, 129), 1e-3, 1, 0), ((65, 65, 65), 1e-2, 1, 0),
                                                 ((65, 65, 65), 1e-4, 1, 0), ((40, 30, 20), 1e-3, 1, 1),
                                                 ((500, 50), 0.01, 0, 0), ((2,), 1e-3, 1, 0),
                                                 ((129, 129, 129), 1e-3, 1, 0), ((300, 65, 65), 1e-3, 1, 0)],
                         ids=str)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_round_trips_within_bound(oracle, H, dev, shape, tol, kind, mode, dtype):
    u = _field(shape, 4, dtype)
    if shape == (129, 129):
        from paper_2503_06322_gb300 import fields
        u = fields.sinusoid_field_2d(dtype=dtype)
    ut = torch.from_numpy(u).to(dev)
    ud = u.astype(np.float64)
    nrm = np.abs(ud).max() if mode == 0 else np.sqrt((ud ** 2).mean())
    tau = tol * nrm if kind == 1 else tol
    buf = H.hpdr_compress(ut, tol, tol_kind=kind, mode=mode)
    bnp = buf.cpu().numpy()
    assert oracle.parse_header(bnp)["total_bytes"] == buf.numel()
    rec = H.hpdr_decompress(buf).cpu().numpy().astype(np.float64)
    assert np.abs(rec - ud).max() <= tau
    # cross decoding: oracle decodes the GPU container, GPU decodes the oracle's
    assert np.abs(oracle.decompress(bnp) - ud).max() <= tau
    obuf = oracle.compress(u, tol, tol_kind=kind, mode=mode)
    rec2 = H.hpdr_decompress(torch.from_numpy(obuf).to(dev)).cpu().numpy().astype(np.float64)
    assert np.abs(rec2 - ud).max() <= tau


def test_zero_and_constant_fields(H, dev):
    z = torch.zeros((17, 9, 5), device=dev)
    assert torch.equal(H.hpdr_decompress(H.hpdr_compress(z, 1e-3)), z)
    c = torch.full((33, 33), 2.5, device=dev)
    r = H.hpdr_decompress(H.hpdr_compress(c, 1e-3))
    assert (r - c).abs().max().item() <= 2.5e-3


def test_errors_are_reported(H, dev):
    u = torch.randn(129, 65, device=dev)
    with pytest.raises(H.HpdrError) as e:
        H.hpdr_compress(u, 1e-9)               # below the binary32 precision floor
    assert e.value.status == -1
    with pytest.raises(H.HpdrError) as e:
        H.hpdr_compress(u, 1e-3, out=torch.empty(64, dtype=torch.uint8, device=dev))
    assert e.value.status == -3
    buf = H.hpdr_compress(u, 1e-3).clone()
    bad = buf.clone()
    bad[20] ^= 1                                 # header byte -> CRC mismatch
    with pytest.raises(H.HpdrError) as e:
        H.hpdr_decompress(bad)
    assert e.value.status == -4
    with pytest.raises(H.HpdrError) as e:
        H.hpdr_decompress(buf[:100])
    assert e.value.status == -4
    # a chunk-table entry beyond the end of the bitstream
    import oracle as O
    h = O.parse_header(buf.cpu().numpy())
    nch = len(h["chunk"])
    off_chunk = 128 + 8 * (h["L"] + 1)
    off_chunk = (off_chunk + 15) & ~15
    off_chunk = (off_chunk + h["s_hi"] - h["s_lo"] + 1 + 15) & ~15
    assert nch >= 2
    bad = buf.clone()
    bad[off_chunk + 8:off_chunk + 16] = torch.tensor(
        list((h["total_bits"] + 5).to_bytes(8, "little")), dtype=torch.uint8, device=dev)
    with pytest.raises(H.HpdrError) as e:
        H.hpdr_decompress(bad)
    assert e.value.status == -4
    # heavy damage inside the bitstream: either rejected or a different field
    bad = buf.clone()
    mid = buf.numel() - 4 * len(h["words"]) // 2
    bad[mid:mid + 64] ^= 0x5A
    try:
        r = H.hpdr_decompress(bad)
        assert not torch.equal(r, H.hpdr_decompress(buf))
    except H.HpdrError as e2:
        assert e2.status == -4
    with pytest.raises(H.HpdrError):
        H.hpdr_compress(u, float("nan"))
    # the context is still usable after the errors
    r = H.hpdr_decompress(buf)
    assert (r - u).abs().max().item() <= 1e-3 * u.abs().max().item()
