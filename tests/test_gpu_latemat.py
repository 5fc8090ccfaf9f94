"""GPU parity of late materialization: px_gather against plain indexing, and the
selective wide join run eagerly and late-materialized against the oracle's
unpartitioned join + group-by (both plans must give the same, exact answer)."""
import numpy as np
import pytest
import torch

import oracle
import pxdata
from gpu_helpers import count, dev, host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [0, 1, 1023, 4096, 100_003])
def test_gather_parity(px, n):
    g = pxdata.rng(700 + n % 97)
    m = 50_000
    cols = [pxdata.random_column(g, m, t) for t in (np.int64, np.int32, np.int8)]
    idx = g.integers(0, m, size=max(n, 1), dtype=np.int32)[:n] if n else np.zeros(0, np.int32)
    out = px.px_gather([dev(c) for c in cols], dev(idx) if n else torch.zeros(1, dtype=torch.int32, device="cuda"),
                       n=n)
    for c, o in zip(cols, out):
        np.testing.assert_array_equal(host(o, n), c[idx])


def test_gather_device_count_and_bad_index(px):
    g = pxdata.rng(710)
    a = pxdata.random_column(g, 1000, np.int64)
    idx = g.integers(0, 1000, size=500, dtype=np.int32)
    d_n = torch.tensor([300], dtype=torch.int64, device="cuda")
    out = px.px_gather([dev(a)], dev(idx), d_n=d_n)
    np.testing.assert_array_equal(host(out[0], 300), a[idx[:300]])
    idx[7] = 1000  # out of range
    ws = px.Workspace(1 << 12)
    px.px_gather([dev(a)], dev(idx), ws=ws)
    assert ws.status() == px.PX_ERR_INVALID


@pytest.mark.parametrize("late", [False, True])
def test_wide_join_eager_and_late_match_oracle(px, late):
    from paper_2606_24647_gb300.pipelines import WideJoinPipeline
    d = pxdata.wide_at_scale(20_000, 400_000, nattr=10_000, build_attr_below=1_000)
    want = oracle.pipeline_wide_join(d)
    dd = {k: dev(v) for k, v in d.items()}
    p = WideJoinPipeline(dd, late=late, nparts=64, nattr_bound=1_000)
    r = p.run()
    assert p.ws.status() == px.PX_OK
    fin = r["final"]
    n = count(fin["ngroups"])
    assert n == want["ngroups"]
    k = host(fin["keys"][0], n).astype(np.int64)
    o = np.argsort(k)
    np.testing.assert_array_equal(k[o], want["keys"][0])
    for a in range(3):
        np.testing.assert_array_equal(host(fin["aggs"][a], n)[o], want["aggs"][a])
