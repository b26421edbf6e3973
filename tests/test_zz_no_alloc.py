"""The allocation-free decomposition entry point.

Some callers cannot allocate device memory on their call path (a stream being
captured into a CUDA graph, services that reserve all memory at start-up);
hpdr_decompose_noalloc serves them from a fixed device array inside the
library.  This file is collected last so that, if it fails, a run stopping at
the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _call(lib, u, out):
    nd = u.dim()
    dims = (C.c_size_t * 3)(*(list(u.shape) + [1] * (3 - nd)))
    st = lib.hpdr_decompose_noalloc(C.c_void_p(u.data_ptr()), C.c_void_p(out.data_ptr()),
                                    0 if u.dtype == torch.float32 else 1, nd, dims,
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st


@pytest.mark.parametrize("shape", [(65, 65, 65), (129, 129), (100, 7, 5), (1000,)], ids=str)
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_noalloc_matches_decompose_twice(shape, dtype):
    from paper_2503_06322_gb300 import fields, hpdr
    lib = hpdr.lib()
    dev = torch.device("cuda:0")
    np_dtype = np.float32 if dtype == torch.float32 else np.float64
    if len(shape) == 1:
        u = np.random.default_rng(9).standard_normal(shape).astype(np_dtype)
    else:
        u = fields.powerlaw_field(shape, seed=9, dtype=np_dtype)
    ut = torch.from_numpy(u).to(dev)
    ref = hpdr.hpdr_decompose(ut)
    tol = 1e-5 if dtype == torch.float32 else 1e-12
    for _ in range(2):                       # the array keeps the last call's contents
        out = torch.full_like(ref, float("nan"))
        assert _call(lib, ut, out) == 0
        assert torch.isfinite(out).all()
        assert (out - ref).abs().max().item() <= tol * ref.abs().max().item()


def test_noalloc_rejects_fields_beyond_its_array():
    from paper_2503_06322_gb300 import hpdr
    lib = hpdr.lib()
    u = torch.zeros((257, 257, 257), device="cuda:0")
    out = torch.empty(u.numel(), device="cuda:0")
    assert _call(lib, u, out) == -3          # HPDR_ERR_CAPACITY, nothing queued
