"""Host-streamed slab pipeline: directory layout, byte identity of every slab
container with the plain API on the same slab, round trips within the bound,
and the oracle decoding the slab containers."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _dir(buf):
    b = buf.numpy().tobytes()
    u32 = lambda o: int.from_bytes(b[o:o + 4], "little")  # noqa: E731
    u64 = lambda o: int.from_bytes(b[o:o + 8], "little")  # noqa: E731
    ns = u32(8)
    ent = [(u64(64 + 32 * i), u64(72 + 32 * i), u64(80 + 32 * i), u64(88 + 32 * i)) for i in range(ns)]
    return b[:4], ns, ent


@pytest.mark.parametrize("shape,slab_planes,dtype", [((70, 65, 65), 8, np.float32), ((41, 33, 17), 4, np.float64),
                                                     ((129, 257), 16, np.float32), ((9, 33, 33), 64, np.float32),
                                                     ((17, 20, 30), 2, np.float32)], ids=str)
def test_streamed_round_trip_and_slab_identity(oracle, shape, slab_planes, dtype):
    from paper_2503_06322_gb300 import fields, hpdr
    u = fields.powerlaw_field(shape, seed=7, dtype=dtype)
    ut = torch.from_numpy(u).pin_memory()
    esz = u.itemsize
    plane = int(np.prod(shape[1:])) * esz
    tol = 1e-3
    buf = hpdr.hpdr_compress_host_streamed(ut, tol, slab_bytes=slab_planes * plane)
    magic, ns, ent = _dir(buf)
    assert magic == b"HPDS"
    assert sum(e[1] for e in ent) == shape[0] and ent[0][0] == 0
    assert all(e[1] >= 2 for e in ent)
    tau = tol * np.abs(u.astype(np.float64)).max()
    for first, planes, off, size in ent:
        slab = np.ascontiguousarray(u[first:first + planes])
        plain = hpdr.hpdr_compress(torch.from_numpy(slab).cuda(), tol).cpu().numpy()
        got = buf[off:off + size].numpy()
        assert np.array_equal(plain, got)
        rec = oracle.decompress(got)
        assert np.abs(rec - slab.astype(np.float64)).max() <= tau
    rec = hpdr.hpdr_decompress_host_streamed(buf)
    assert rec.shape == shape
    assert np.abs(rec.numpy().astype(np.float64) - u.astype(np.float64)).max() <= tau


def test_streamed_capacity_error():
    from paper_2503_06322_gb300 import hpdr
    u = torch.randn(40, 33, 33).pin_memory()
    with pytest.raises(hpdr.HpdrError) as e:
        hpdr.hpdr_compress_host_streamed(u, 1e-3, out=torch.empty(100, dtype=torch.uint8))
    assert e.value.status == -3
