"""Failure detection on the GPU without a fault: a bounded device wait that
runs out.

The level kernels of compression and decompression stream planes through a
ring of shared-memory stages filled by bulk asynchronous copies and wait on
mbarriers for them.  Every wait gives up after a number of polls, records
DS_TIMEOUT, waits (with its own long bound) for the copies it has in flight
and returns; the call then returns HPDR_ERR_TIMEOUT.  Setting the poll limit
to zero makes the first wait give up at once, so the path runs with every
copy completing normally: nothing stalls, nothing faults, and the context
stays usable -- the same calls afterwards give the same bytes as before.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TIMEOUT = -5


@pytest.fixture(scope="module")
def H():
    from paper_2503_06322_gb300 import hpdr
    return hpdr


@pytest.mark.parametrize("shape", [(65, 65, 65), (257, 257), (70, 33, 40)], ids=str)
def test_wait_that_runs_out_returns_timeout_and_context_recovers(H, shape):
    from paper_2503_06322_gb300 import fields
    lib = H.lib()
    u = torch.from_numpy(fields.powerlaw_field(shape, seed=3)).to("cuda:0")
    ref = H.hpdr_compress(u, 1e-3).clone()
    rec_ref = H.hpdr_decompress(ref)
    prev = lib.hpdr_debug_set_wait_limit(0)
    try:
        with pytest.raises(H.HpdrError) as e:
            H.hpdr_compress(u, 1e-3)
        assert e.value.status == TIMEOUT
        with pytest.raises(H.HpdrError) as e:
            H.hpdr_decompress(ref)
        assert e.value.status == TIMEOUT
    finally:
        assert lib.hpdr_debug_set_wait_limit(prev) == 0
    assert lib.hpdr_debug_set_wait_limit(-1) == prev
    torch.cuda.synchronize()
    again = H.hpdr_compress(u, 1e-3)
    assert torch.equal(again, ref)
    rec = H.hpdr_decompress(again)
    assert torch.equal(rec, rec_ref)
    tau = 1e-3 * u.abs().max().item()
    assert (rec.double() - u.double()).abs().max().item() <= tau
