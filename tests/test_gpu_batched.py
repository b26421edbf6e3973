"""Batched compression (one graph replay): every field's container is
byte-identical to the plain API on that field, and replays repeat it."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_batched_matches_plain_and_replays(oracle):
    from paper_2503_06322_gb300 import fields, hpdr
    shapes = fields.batch_shapes(count=24, seed=11, lo=17, hi=90)
    us, tols = [], []
    for i, (shape, tol) in enumerate(shapes):
        us.append(torch.from_numpy(fields.powerlaw_field(shape, seed=100 + i)).cuda())
        tols.append(tol)
    us.append(torch.from_numpy(fields.powerlaw_field((40, 30, 20), seed=99, dtype=np.float64)).cuda())
    tols.append(1e-3)
    out, offs, sizes = hpdr.hpdr_compress_batched(us, tols)
    for i, (u, tol) in enumerate(zip(us, tols)):
        plain = hpdr.hpdr_compress(u, tol)
        got = out[offs[i]:offs[i] + sizes[i]]
        assert sizes[i] == plain.numel()
        assert torch.equal(got, plain)
        rec = hpdr.hpdr_decompress(got.clone())
        un = u.double()
        assert (rec.double() - un).abs().max().item() <= tol * un.abs().max().item()
    out2, offs2, sizes2 = hpdr.hpdr_compress_batched(us, tols, out=out)
    assert offs2 == offs and sizes2 == sizes
    assert hpdr.lib().hpdr_batched_streams(hpdr.context()) in (1, 2, 4, 8, 16)
    # one container through the oracle
    h = out[offs[3]:offs[3] + sizes[3]].cpu().numpy()
    u3 = us[3].cpu().numpy().astype(np.float64)
    assert np.abs(oracle.decompress(h) - u3).max() <= tols[3] * np.abs(u3).max()


def test_batched_full_draw_matches_plain():
    """The batching workload's own draw: 256 fields (seed 3), 2-D or 3-D,
    dims log-uniform in [17, 513], bounds from {1e-2, 1e-3, 1e-4}.  Large
    fields take the level kernels' multi-tile, multi-segment paths; every
    container must equal the plain API's, byte for byte, and decompress
    within its bound."""
    from paper_2503_06322_gb300 import fields, hpdr
    draw = fields.batch_shapes(count=256, seed=3)
    assert max(max(s) for s, _ in draw) >= 400
    us = [fields.powerlaw_field_torch(s, seed=1000 + i, device=torch.device("cuda:0")) for i, (s, _) in enumerate(draw)]
    tols = [t for _, t in draw]
    out, offs, sizes = hpdr.hpdr_compress_batched(us, tols)
    for i, (u, tol) in enumerate(zip(us, tols)):
        plain = hpdr.hpdr_compress(u, tol)
        assert sizes[i] == plain.numel(), i
        got = out[offs[i]:offs[i] + sizes[i]]
        assert torch.equal(got, plain), i
        if max(u.shape) >= 257:
            rec = hpdr.hpdr_decompress(got.clone())
            un = u.double()
            assert (rec.double() - un).abs().max().item() <= tol * un.abs().max().item(), i


def test_batched_cache_is_bounded():
    """A captured batch holds its buffers, so every new output buffer is a new
    capture; the context keeps the four most recently used ones and frees the
    rest (workspace, sizes, graph), and results stay byte-identical."""
    from paper_2503_06322_gb300 import fields, hpdr
    lib = hpdr.lib()
    us = [torch.from_numpy(fields.powerlaw_field((33 + 8 * i, 40, 17), seed=300 + i)).cuda() for i in range(5)]
    tols = [1e-3] * len(us)
    ref, offs_ref, sizes_ref = hpdr.hpdr_compress_batched(us, tols)
    outs = [torch.zeros_like(ref) for _ in range(7)]      # seven distinct output buffers
    free_at = []
    for out in outs:
        got, offs, sizes = hpdr.hpdr_compress_batched(us, tols, out=out)
        assert sizes == sizes_ref and offs == offs_ref
        for i in range(len(us)):
            assert torch.equal(got[offs[i]:offs[i] + sizes[i]], ref[offs_ref[i]:offs_ref[i] + sizes_ref[i]])
        assert 1 <= lib.hpdr_batched_cached(hpdr.context()) <= 4
        torch.cuda.synchronize()
        free_at.append(torch.cuda.mem_get_info()[0])
    # once four batches are held, each new capture frees as much as it takes
    assert abs(free_at[-1] - free_at[3]) < (16 << 20)
    # a buffer whose batch was evicted is captured again and still agrees
    got, offs, sizes = hpdr.hpdr_compress_batched(us, tols, out=outs[0])
    assert sizes == sizes_ref
    for i in range(len(us)):
        assert torch.equal(got[offs[i]:offs[i] + sizes[i]], ref[offs_ref[i]:offs_ref[i] + sizes_ref[i]])


def test_batched_large_alphabet_and_mixed_types():
    """An alphabet above the one-block codebook's limit (D = 16384) takes the
    per-field codebook in the batch's codebook phase; FP32 and FP64 fields
    whose coarse levels run in one launch per element type; a field too small
    for any coarse level (level 0 alone).  Every container equals the plain
    API's with the same dictionary."""
    from paper_2503_06322_gb300 import fields, hpdr
    shapes = [((70, 33, 40), np.float32), ((65, 65, 65), np.float64), ((300, 200), np.float32),
              ((3, 3), np.float32), ((129, 17), np.float64), ((2,), np.float32)]
    us = []
    for i, (sh, dt) in enumerate(shapes):
        if len(sh) == 1:
            us.append(torch.from_numpy(np.random.default_rng(i).standard_normal(sh).astype(dt)).cuda())
        else:
            us.append(torch.from_numpy(fields.powerlaw_field(sh, seed=400 + i, dtype=dt)).cuda())
    tols = [1e-3, 1e-4, 1e-2, 1e-3, 1e-3, 1e-3]
    for D in (16384, 8192):
        out, offs, sizes = hpdr.hpdr_compress_batched(us, tols, dict_size=D)
        for i, (u, tol) in enumerate(zip(us, tols)):
            plain = hpdr.hpdr_compress(u, tol, dict_size=D)
            assert sizes[i] == plain.numel(), (D, i)
            assert torch.equal(out[offs[i]:offs[i] + sizes[i]], plain), (D, i)
