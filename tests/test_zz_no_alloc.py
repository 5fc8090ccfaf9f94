"""px_filter_noalloc: the allocation-free filter entry point.

It serves callers that cannot allocate device memory (and so cannot pass a
workspace): its scratch is a static device array inside libpx.so. These tests
call it through the C ABI and check its selection against the CPU oracle's
filter and against px_filter's on two calls in a row (a case with more tiles
than one round of the tile-count scan included, so the scan's carry runs inside
the static array), and that sizes beyond its static scratch are refused on the
host. This file is collected last so that a run stopping at the first failure
has already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import pxdata


def test_noalloc_rejects_rows_beyond_its_scratch_on_the_host():
    import paper_2606_24647_gb300 as pxm
    L = pxm.load()
    col = pxm.px_col(pxm.PX_I32, 0, 0x7f0000000000)
    limit = 134217728
    r = L.px_filter_noalloc(ctypes.byref(col), limit + 1, None, 0, 1, 0x7f0000001000, 0x7f0000002000, None, None)
    assert r == pxm.PX_ERR_UNSUPPORTED
    assert "px_filter" in pxm.last_error()


_TYPES = {np.int8: 1, np.int32: 4, np.int64: 8}


@pytest.mark.gpu
def test_noalloc_matches_the_oracle_and_px_filter_on_two_calls_in_a_row(px):
    L = px.load()
    g = pxdata.rng(900)
    stream = torch.cuda.current_stream()
    # 17.5M int8 rows = 8545 tiles of 2048: more than one 8192-count round of the scan
    cases = [(pxdata.random_column(g, 300_001, np.int32, 0, 2556), 895, 1662),
             (pxdata.random_column(g, 70_003, np.int64, -1000, 1000), -10, 500),
             (pxdata.random_column(g, 17_500_001, np.int8, -128, 127), -40, 77)]
    for col_np, lo, hi in cases:
        want = oracle.filter(col_np, lo, hi)
        col = torch.from_numpy(col_np).cuda()
        n = col.numel()
        ref_sel, ref_n = px.px_filter(col, lo, hi)
        c = px.px_col(_TYPES[col_np.dtype.type], 0, col.data_ptr())
        for _ in range(2):  # the static scratch keeps the previous call's contents
            sel = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            nsel = torch.full((1,), -1, dtype=torch.int64, device="cuda")
            status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
            r = L.px_filter_noalloc(ctypes.byref(c), n, None, lo, hi, sel.data_ptr(), nsel.data_ptr(),
                                    status.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
            assert r == px.PX_OK, px.last_error()
            torch.cuda.synchronize()
            assert int(status.item()) == px.PX_OK
            m = int(nsel.item())
            assert m == want.size
            assert np.array_equal(sel[:m].cpu().numpy(), want)
            assert m == int(ref_n.item()) and torch.equal(sel[:m], ref_sel[:m])
