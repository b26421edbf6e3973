"""Adaptive chunk sizing of the host-device pipeline (Sec. V-C, Alg. 4):
the throughput-model fit and the chunk plan, host-only entries of the C ABI
(no device work), against worked examples and closed forms."""
import pytest

MB = 1 << 20


@pytest.fixture(scope="module")
def H():
    from paper_2503_06322_gb300 import build, hpdr
    build.build()
    return hpdr


def test_fit_recovers_a_piecewise_model(H):
    # Phi(C) = min(alpha C + beta, gamma), profiled at 1 MB .. 1 GB
    alpha, beta, gamma = 1e3, 1e10, 2e11
    sizes = [float((1 << k) * MB) for k in range(11)]
    tp = [min(alpha * c + beta, gamma) for c in sizes]
    m = H.pipeline_fit(sizes, tp, h2d=5e10, f=0.1)
    # saturated from the first size with throughput >= 0.9 gamma: 256 MB
    assert m.c_threshold == 256 * MB and m.gamma == gamma and m.h2d == 5e10
    assert m.alpha == pytest.approx(alpha, rel=1e-9) and m.beta == pytest.approx(beta, rel=1e-9)


def test_fit_order_and_degenerate_cases(H):
    # input order does not matter
    m1 = H.pipeline_fit([4 * MB, 1 * MB, 2 * MB], [3e9, 1e9, 2e9], h2d=1e9, f=0.1)
    m2 = H.pipeline_fit([1 * MB, 2 * MB, 4 * MB], [1e9, 2e9, 3e9], h2d=1e9, f=0.1)
    assert m1.as_dict() == m2.as_dict()
    # three points on a line below the saturated largest chunk (3e9 / 2e9 < 0.9)
    assert m2.c_threshold == 4 * MB and m2.gamma == 3e9
    assert m2.alpha == pytest.approx(1e9 / MB) and m2.beta == pytest.approx(0.0, abs=1e-3)
    # one chunk: constant model
    m = H.pipeline_fit([8 * MB], [5e9], h2d=1e9)
    assert (m.alpha, m.beta, m.gamma, m.c_threshold) == (0.0, 5e9, 5e9, 8 * MB)
    # one smaller chunk: the line through it and (c_threshold, gamma)
    m = H.pipeline_fit([2 * MB, 6 * MB], [1e9, 3e9], h2d=1e9, f=0.1)
    assert m.c_threshold == 6 * MB
    assert m.alpha * 2 * MB + m.beta == pytest.approx(1e9) and m.alpha * 6 * MB + m.beta == pytest.approx(3e9)
    # every chunk within f of gamma: all saturated
    m = H.pipeline_fit([1 * MB, 2 * MB], [9.5e9, 1e10], h2d=1e9, f=0.1)
    assert m.c_threshold == 1 * MB and (m.alpha, m.beta) == (0.0, 1e10)
    for bad in (([], [], 1e9, 0.1), ([MB], [0.0], 1e9, 0.1), ([MB], [1e9], 0.0, 0.1), ([MB], [1e9], 1e9, 1.0)):
        with pytest.raises(H.HpdrError):
            H.pipeline_fit(bad[0], bad[1], h2d=bad[2], f=bad[3])


def _const(H, growth, gamma=1e11):
    return H.PipelineModel(alpha=0.0, beta=gamma, gamma=gamma, c_threshold=0.0, h2d=growth * gamma)


def test_plan_worked_examples(H):
    # Theta(C / gamma) = 2 C: each chunk doubles until the data runs out
    assert H.pipeline_plan(_const(H, 2.0), 100, MB, 3 * MB) == [3, 6, 12, 24, 48, 7]
    # ... up to C_limit
    assert H.pipeline_plan(_const(H, 2.0), 100, MB, 3 * MB, 20 * MB) == [3, 6, 12, 20, 20, 20, 19]
    # a single plane left joins the last chunk
    assert H.pipeline_plan(_const(H, 2.0), 10, MB, 3 * MB) == [3, 7]
    # a copy slower than the compression shrinks the chunks, to two planes at least
    assert H.pipeline_plan(_const(H, 0.5), 20, MB, 8 * MB) == [8, 4, 2, 2, 2, 2]
    # C_init below two planes, and above the whole field
    assert H.pipeline_plan(_const(H, 1.0), 9, MB, 1) == [2, 2, 2, 3]
    assert H.pipeline_plan(_const(H, 1.0), 9, MB, 100 * MB) == [9]


def test_plan_with_a_linear_phi(H):
    # below the threshold Phi(C) = alpha C: C / Phi(C) = 1 / alpha seconds for
    # every chunk, so every next chunk is Theta(1 / alpha) = h2d / alpha bytes
    m = H.PipelineModel(alpha=1e3, beta=0.0, gamma=1e12, c_threshold=1e15, h2d=8e3 * MB)
    assert H.pipeline_plan(m, 50, MB, 2 * MB) == [2, 8, 8, 8, 8, 8, 8]
    # above the threshold: Phi = gamma, so the chunk grows by h2d / gamma
    m = H.PipelineModel(alpha=1e3, beta=0.0, gamma=1e9, c_threshold=1.0, h2d=3e9)
    assert H.pipeline_plan(m, 60, MB, 2 * MB) == [2, 6, 18, 34]


def test_plan_rejects_bad_arguments(H):
    with pytest.raises(H.HpdrError):
        H.pipeline_plan(_const(H, 2.0), 1, MB, MB)
    with pytest.raises(H.HpdrError):
        H.pipeline_plan(H.PipelineModel(alpha=0.0, beta=1.0, gamma=0.0, c_threshold=0.0, h2d=1.0), 10, MB, MB)


def test_streamed_bound_of_a_plan(H):
    import torch
    shape = (20, 33, 17)
    planes = [2, 4, 8, 6]
    b = H.streamed_bound_plan(shape, torch.float32, planes)
    parts = [(H.hpdr_compress_bound((p, 33, 17), torch.float32) + 15) // 16 * 16 for p in planes]
    assert b == (64 + 32 * 4 + 15) // 16 * 16 + sum(parts)
    for bad in ([2, 4, 8, 5], [1, 4, 8, 7]):
        with pytest.raises(H.HpdrError):
            H.streamed_bound_plan(shape, torch.float32, bad)


def test_lossless_bound(H):
    # n = 1000 byte keys, automatic K = 256: 4 chunks; table at a16(64 + 256) = 320,
    # bitstream at a16(320 + 32) = 352, at most 8 bits per key
    assert H.lossless_bound(1000, 1) == 352 + 4 * 250
    # 16-bit keys: a 65536-byte length table, at most 16 bits per key
    assert H.lossless_bound(1000, 2, 128) == (64 + 65536 + 8 * 8 + 15) // 16 * 16 + 4 * 500
    for bad in ((0, 1, 0), (10, 3, 0), (10, 1, 100)):
        with pytest.raises(H.HpdrError):
            H.lossless_bound(*bad)
