"""px_filter_noalloc: the allocation-free filter entry point.

It serves callers that cannot allocate device memory (and so cannot pass a
workspace): its scratch is a static device array inside libpx.so. These tests
call it through the C ABI and check that its output equals px_filter's on two
calls in a row, and that sizes beyond its static scratch are refused on the host.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import pxdata


def test_noalloc_rejects_rows_beyond_its_scratch_on_the_host():
    import paper_2606_24647_gb300 as pxm
    L = pxm.load()
    col = pxm.px_col(pxm.PX_I32, 0, 0x7f0000000000)
    limit = 134217728
    r = L.px_filter_noalloc(ctypes.byref(col), limit + 1, None, 0, 1, 0x7f0000001000, 0x7f0000002000, None, None)
    assert r == pxm.PX_ERR_UNSUPPORTED
    assert "px_filter" in pxm.last_error()


@pytest.mark.gpu
def test_noalloc_matches_px_filter_on_two_calls_in_a_row(px):
    L = px.load()
    g = pxdata.rng(900)
    stream = torch.cuda.current_stream()
    cases = [(pxdata.random_column(g, 300_001, np.int32, 0, 2556), 895, 1662),
             (pxdata.random_column(g, 70_003, np.int64, -1000, 1000), -10, 500)]
    for col_np, lo, hi in cases:
        col = torch.from_numpy(col_np).cuda()
        n = col.numel()
        want_sel, want_n = px.px_filter(col, lo, hi)
        sel = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        nsel = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        c = px.px_col(px.PX_I64 if col.dtype == torch.int64 else px.PX_I32, 0, col.data_ptr())
        r = L.px_filter_noalloc(ctypes.byref(c), n, None, lo, hi, sel.data_ptr(), nsel.data_ptr(),
                                status.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert r == px.PX_OK, px.last_error()
        torch.cuda.synchronize()
        assert int(status.item()) == px.PX_OK
        m = int(want_n.item())
        assert int(nsel.item()) == m
        assert torch.equal(sel[:m], want_sel[:m])
