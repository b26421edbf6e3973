"""Fixed-rate ZFP (Alg. 3) on the GPU against the oracle, through the C ABI.

Integer and byte work, so the bar is bit-exact: container bytes equal the
oracle's; decoding the oracle's containers gives the oracle's values; at the
513^3 bench size the words of the first two block planes equal the oracle's
container of those 8 planes (blocks are independent and dimension 0 is the
slowest block index)."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

CASES = [((1000,), 8), ((1000,), 16), ((7,), 32), ((1001,), 64), ((65, 33), 2), ((65, 33), 8), ((9, 6), 12),
         ((300, 200), 4), ((33, 17, 9), 1), ((33, 17, 9), 4), ((33, 17, 9), 8), ((5, 6, 7), 16),
         ((16, 16, 16), 32), ((70, 70, 70), 8), ((65, 65, 65), 12), ((20, 30, 40), 136)]


@pytest.fixture(scope="module")
def H():
    from paper_2503_06322_gb300 import hpdr
    return hpdr


def _field(shape, seed, dtype):
    from paper_2503_06322_gb300 import fields
    if len(shape) == 1:
        return np.random.default_rng(seed).standard_normal(shape).astype(dtype)
    u = fields.powerlaw_field(shape, seed=seed, dtype=dtype)
    if len(shape) == 2 and shape[0] >= 8 and shape[1] >= 4:
        u[:4, :4] = 0.0          # a zero block
        u[4:8, :4] = 2.25        # a constant block
    return u


@pytest.mark.parametrize("shape,rate", CASES, ids=str)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_containers_bit_exact_and_cross_decoding(H, shape, rate, dtype):
    u = _field(shape, 3, dtype)
    ob = oracle.zfp_compress(u, rate)
    gb = H.hpdr_zfp_compress(torch.from_numpy(u).cuda(), rate)
    assert gb.numel() == ob.size == H.zfp_bound(shape, rate, torch.from_numpy(u).dtype)
    assert np.array_equal(gb.cpu().numpy(), ob)
    od = oracle.zfp_decompress(ob).astype(dtype)
    gd = H.hpdr_zfp_decompress(torch.from_numpy(ob).cuda()).cpu().numpy()
    assert gd.shape == shape and np.array_equal(gd, od)


def test_full_size_first_block_planes(H):
    from paper_2503_06322_gb300 import fields
    u = fields.powerlaw_field_torch((513, 513, 513), seed=1, device="cuda")
    for rate in (8, 16):
        gb = H.hpdr_zfp_compress(u, rate)
        nblocks = 129 ** 3
        assert gb.numel() == 64 + nblocks * rate * 64 // 8
        per = rate * 64 // 8
        head = gb[64:64 + 2 * 129 * 129 * per].cpu().numpy()
        ob = oracle.zfp_compress(u[:8].cpu().numpy(), rate)
        assert np.array_equal(head, ob[64:])
        rec = H.hpdr_zfp_decompress(gb)
        err = (rec.double() - u.double()).pow(2).mean().sqrt().item() / u.double().std().item()
        assert err < (2e-2 if rate == 8 else 1e-4)


def test_errors(H):
    u = torch.zeros(10, device="cuda")
    with pytest.raises(ValueError):
        H.hpdr_zfp_compress(u, 4)                      # 4 x 4 bits is not a multiple of 32
    with pytest.raises(H.HpdrError) as e:
        H.hpdr_zfp_compress(u, 8, out=torch.empty(40, dtype=torch.uint8, device="cuda"))
    assert e.value.status == -3
    b = H.hpdr_zfp_compress(torch.ones(64, 64, device="cuda"), 8).clone()
    b[20] ^= 1                                         # header CRC
    with pytest.raises(H.HpdrError) as e:
        H.hpdr_zfp_decompress(b)
    assert e.value.status == -4
