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


def _const_model(hpdr, growth):
    """Phi constant (gamma), Theta(t) = growth * gamma * t: every chunk is
    growth times the previous one (Alg. 4 with a saturated device)."""
    g = 1e11
    return hpdr.PipelineModel(alpha=0.0, beta=g, gamma=g, c_threshold=0.0, h2d=growth * g)


@pytest.mark.parametrize("shape,dtype,init_planes,limit_planes,expect",
                         [((70, 65, 65), np.float32, 2, 0, [2, 4, 8, 16, 32, 8]),
                          ((41, 33, 17), np.float64, 3, 10, [3, 6, 10, 10, 10, 2]),
                          ((100000,), np.float32, 4096, 40000, [4096, 8192, 16384, 32768, 38560])], ids=str)
def test_adaptive_round_trip_and_chunk_identity(oracle, shape, dtype, init_planes, limit_planes, expect):
    from paper_2503_06322_gb300 import fields, hpdr
    u = fields.powerlaw_field(shape, seed=9, dtype=dtype)
    ut = torch.from_numpy(u).pin_memory()
    plane = int(np.prod(shape[1:])) * u.itemsize
    m = _const_model(hpdr, 2.0)
    c_init, c_limit = init_planes * plane, limit_planes * plane
    assert hpdr.pipeline_plan(m, shape[0], plane, c_init, c_limit) == expect
    tol = 1e-3
    buf = hpdr.hpdr_compress_host_adaptive(ut, tol, m, c_init=c_init, c_limit=c_limit)
    magic, ns, ent = _dir(buf)
    assert magic == b"HPDS" and [e[1] for e in ent] == expect
    assert [e[0] for e in ent] == list(np.cumsum([0] + expect[:-1]))
    tau = tol * np.abs(u.astype(np.float64)).max()
    for first, planes, off, size in ent:
        slab = np.ascontiguousarray(u[first:first + planes])
        plain = hpdr.hpdr_compress(torch.from_numpy(slab).cuda(), tol).cpu().numpy()
        got = buf[off:off + size].numpy()
        assert np.array_equal(plain, got)
        assert np.abs(oracle.decompress(got) - slab.astype(np.float64)).max() <= tau
    rec = hpdr.hpdr_decompress_host_streamed(buf)
    assert np.abs(rec.numpy().astype(np.float64) - u.astype(np.float64)).max() <= tau


def test_pipeline_profile_and_adaptive_compression():
    from paper_2503_06322_gb300 import fields, hpdr
    shape = (129, 129, 129)
    u = fields.powerlaw_field(shape, seed=11, dtype=np.float32)
    ut = torch.from_numpy(u).pin_memory()
    plane = 129 * 129 * 4
    sizes = [2 * plane, 8 * plane, 32 * plane, 128 * plane]
    m = hpdr.pipeline_profile(ut, 1e-3, sizes, reps=2)
    assert m.gamma > 0 and m.h2d > 0 and m.c_threshold in sizes
    planes = hpdr.pipeline_plan(m, shape[0], plane, 4 * plane, 64 * plane)
    assert sum(planes) == 129 and min(planes) >= 2 and max(planes) <= 65
    buf = hpdr.hpdr_compress_host_adaptive(ut, 1e-3, m, c_init=4 * plane, c_limit=64 * plane)
    _, ns, ent = _dir(buf)
    assert [e[1] for e in ent] == planes
    rec = hpdr.hpdr_decompress_host_streamed(buf).numpy().astype(np.float64)
    assert np.abs(rec - u).max() <= 1e-3 * np.abs(u).max()
