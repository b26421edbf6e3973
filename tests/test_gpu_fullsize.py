"""Full-size workloads, in the launch configuration the benchmark times
(default dictionary and chunk size, one context, the current stream):

  * 513^3 FP32 power-law field at relative Linf bounds 1e-2, 1e-3, 1e-4;
  * 500 x 500 x 100 FP64 power-law field (non-dyadic, L = 7).

What the oracle can finish in tens of seconds is compared in full:
  * decomposition coefficients, every element (1e-5 x max|coef| for FP32,
    1e-12 for FP64);
  * quantization codes on identical inputs against the oracle's binary64
    decision (equal except at half-bin ties, at most 1e-5 of the elements; at
    1e-3 and at the tightest bound, 1e-4) and the whole Huffman part of the
    container, bit-exact (513^3 at 1e-3, the benchmark's bound);
  * cross decoding: the oracle's FP64 reconstruction of the GPU container
    against the GPU's own reconstruction;
  * the error bound, on every element of every reconstruction.
"""
import numpy as np
import pytest
import torch
from _codes import assert_codes_match_fp64

pytestmark = pytest.mark.gpu

BIG = (513, 513, 513)
F64 = (500, 500, 100)


@pytest.fixture(scope="module")
def H():
    from paper_2503_06322_gb300 import hpdr
    return hpdr


@pytest.fixture(scope="module")
def big():
    from paper_2503_06322_gb300 import fields
    assert torch.cuda.is_available()
    u = fields.powerlaw_field_torch(BIG, seed=1, device=torch.device("cuda:0"))
    torch.cuda.synchronize()
    return u, u.cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def f64field():
    from paper_2503_06322_gb300 import fields
    u = fields.powerlaw_field(F64, seed=2, dtype=np.float64)
    return torch.from_numpy(u).to("cuda:0"), u


def _parse(oracle, buf):
    h = oracle.parse_header(buf)
    assert h["magic"] == b"HPDR" and h["total_bytes"] == buf.size
    return h


def test_513_decompose_every_coefficient(oracle, H, big):
    u, ud = big
    coef = H.hpdr_decompose(u).cpu().numpy().astype(np.float64)
    ref = oracle.decompose(ud)
    assert np.abs(coef - ref).max() <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("tol", [1e-2, 1e-3, 1e-4])
def test_513_round_trip_bound_and_cross_decoding(oracle, H, big, tol):
    u, ud = big
    tau = tol * np.abs(ud).max()
    buf = H.hpdr_compress(u, tol)
    bnp = buf.cpu().numpy()
    h = _parse(oracle, bnp)
    assert h["L"] == 9 and h["N"] == ud.size and h["dims"] == BIG
    rec = H.hpdr_decompress(buf).cpu().numpy().astype(np.float64)
    err = np.abs(rec - ud).max()
    assert err <= tau
    orec = oracle.decompress(bnp)
    assert np.abs(orec - ud).max() <= tau
    # same codes, recomposed in FP32 on the GPU and in FP64 by the oracle
    assert np.abs(orec - rec).max() <= 1e-5 * np.abs(ud).max()


def test_513_codes_and_huffman_bit_exact(oracle, H, big):
    u, ud = big
    buf = H.hpdr_compress(u, 1e-3).cpu().numpy()
    h = _parse(oracle, buf)
    sym, esc = oracle.decode(h["words"], h["chunk"], h["N"], h["K"], h["lengths"], esc_width=h["esc_width"])
    coef = H.hpdr_decompose(u).cpu().numpy().astype(np.float64)
    assert_codes_match_fp64(oracle, sym, esc, coef, BIG, h["q"], h["D"])
    ln = oracle.code_lengths(oracle.histogram(sym, h["D"]))
    words, chunk, bits = oracle.encode(sym, ln, K=h["K"], esc_k=esc)
    assert np.array_equal(h["lengths"], ln)
    assert h["total_bits"] == bits and np.array_equal(h["chunk"], chunk)
    assert np.array_equal(h["words"], words)


def test_500x500x100_fp64_decompose(oracle, H, f64field):
    u, ud = f64field
    coef = H.hpdr_decompose(u).cpu().numpy()
    ref = oracle.decompose(ud)
    assert np.abs(coef - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("tol", [1e-2, 1e-3, 1e-4])
def test_500x500x100_fp64_round_trip(oracle, H, f64field, tol):
    u, ud = f64field
    tau = tol * np.abs(ud).max()
    buf = H.hpdr_compress(u, tol)
    bnp = buf.cpu().numpy()
    h = _parse(oracle, bnp)
    assert h["L"] == 7 and h["dtype"] == 1
    rec = H.hpdr_decompress(buf).cpu().numpy()
    assert np.abs(rec - ud).max() <= tau
    orec = oracle.decompress(bnp)
    assert np.abs(orec - ud).max() <= tau
    assert np.abs(orec - rec).max() <= 1e-12 * np.abs(ud).max()


def test_513_codes_against_fp64_decision_at_1e4(oracle, H, big):
    """At the tightest bound (codes in the thousands) the codes of the
    container still agree with the binary64 decision on the GPU's own
    coefficients everywhere but at half-bin ties (at most 1e-5 of the
    elements).  A binary32 decision fails this: at this bound it disagreed
    on 4.6e-4 of the elements."""
    u, ud = big
    buf = H.hpdr_compress(u, 1e-4).cpu().numpy()
    h = _parse(oracle, buf)
    sym, esc = oracle.decode(h["words"], h["chunk"], h["N"], h["K"], h["lengths"], esc_width=h["esc_width"])
    coef = H.hpdr_decompose(u).cpu().numpy().astype(np.float64)
    assert_codes_match_fp64(oracle, sym, esc, coef, BIG, h["q"], h["D"])
