"""Compression and decompression that never wait on the host.

hpdr_compress_async reports {container bytes, device status} through device
memory; hpdr_decompress_async parses the container header on the device.
Their results must equal the waiting calls' byte for byte, chains of them
must run without host synchronization, and a bad header must come back as a
FORMAT status (not as a fault or a wrong field).
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

FORMAT = -4


@pytest.fixture(scope="module")
def H():
    from paper_2503_06322_gb300 import hpdr
    return hpdr


@pytest.mark.parametrize("shape,dtype,tol", [((65, 65, 65), torch.float32, 1e-3), ((129, 129, 129), torch.float32, 1e-4),
                                             ((300, 200), torch.float32, 1e-2), ((40, 30, 20), torch.float64, 1e-3),
                                             ((1000,), torch.float32, 1e-3)], ids=str)
def test_async_equals_waiting_calls(H, shape, dtype, tol):
    from paper_2503_06322_gb300 import fields
    np_dtype = np.float32 if dtype == torch.float32 else np.float64
    if len(shape) == 1:
        u = torch.from_numpy(np.random.default_rng(5).standard_normal(shape).astype(np_dtype)).cuda()
    else:
        u = torch.from_numpy(fields.powerlaw_field(shape, seed=5, dtype=np_dtype)).cuda()
    ref = H.hpdr_compress(u, tol)
    cap = H.hpdr_compress_bound(shape, dtype)
    out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    res = torch.full((2,), -1, dtype=torch.int64, device="cuda")
    H.hpdr_compress_async(u, tol, out, res)
    rec = torch.full_like(u, float("nan"))
    dres = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    H.hpdr_decompress_async(out, rec, dres)
    torch.cuda.synchronize()
    nb, st = int(res[0]), int(res[1])
    assert st == 0 and nb == ref.numel()
    assert torch.equal(out[:nb], ref)
    assert int(dres[0]) == 0
    assert torch.equal(rec, H.hpdr_decompress(ref))


def test_async_chain_without_host_waits(H):
    """Ten compress -> decompress steps queued back to back, checked once."""
    from paper_2503_06322_gb300 import fields
    shape = (129, 65, 97)
    u = torch.from_numpy(fields.powerlaw_field(shape, seed=6)).cuda()
    cap = H.hpdr_compress_bound(shape, u.dtype)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    rec = torch.empty_like(u)
    res = torch.zeros((10, 2), dtype=torch.int64, device="cuda")
    dres = torch.zeros((10,), dtype=torch.int64, device="cuda")
    for i in range(10):
        H.hpdr_compress_async(u, 1e-3, out, res[i])
        H.hpdr_decompress_async(out, rec, dres[i:i + 1])
    torch.cuda.synchronize()
    assert (res[:, 1] == 0).all() and (dres == 0).all()
    assert (res[:, 0] == res[0, 0]).all()
    tau = 1e-3 * u.abs().max().item()
    assert (rec.double() - u.double()).abs().max().item() <= tau


def test_async_rejects_bad_headers(H):
    from paper_2503_06322_gb300 import fields
    shape = (65, 65, 65)
    u = torch.from_numpy(fields.powerlaw_field(shape, seed=7)).cuda()
    buf = H.hpdr_compress(u, 1e-3).clone()
    rec = torch.empty_like(u)
    res = torch.zeros((1,), dtype=torch.int64, device="cuda")
    # a flipped header byte (CRC)
    bad = buf.clone()
    bad[20] ^= 1
    H.hpdr_decompress_async(bad, rec, res)
    torch.cuda.synchronize()
    assert H.device_status(int(res[0])) == FORMAT
    # the wrong shape for this container
    other = torch.empty((65, 65, 64), dtype=torch.float32, device="cuda")
    res.zero_()
    H.hpdr_decompress_async(buf, other, res)
    torch.cuda.synchronize()
    assert H.device_status(int(res[0])) == FORMAT
    # a truncated buffer
    res.zero_()
    H.hpdr_decompress_async(buf[: buf.numel() // 2], rec, res)
    torch.cuda.synchronize()
    assert H.device_status(int(res[0])) == FORMAT
    # the context still works
    res.zero_()
    H.hpdr_decompress_async(buf, rec, res)
    torch.cuda.synchronize()
    assert int(res[0]) == 0 and torch.equal(rec, H.hpdr_decompress(buf))
