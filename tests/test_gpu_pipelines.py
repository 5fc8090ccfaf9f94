"""GPU parity of the three workload pipelines against the oracle.

Reduced sizes are compared element by element with the oracle's pipelines. At the
full workload sizes (1M-row plain batch; 200k x 6M plain join; 2M x 60M skewed
join at 64 partitions, the launch configuration the bench times) the small ones
are compared in full, and the large ones on sampled rows the oracle computes one
by one plus closed forms of the generators (every fact key names exactly one
dimension row, so each group's SUM/COUNT is a lookup-and-add over the fact rows).
"""
import numpy as np
import pytest
import torch

import oracle
import pxdata
from gpu_helpers import assert_groups_equal, count, dev, host
from paper_2606_24647_gb300.pipelines import AtScalePipeline, JoinPipeline, PlainPipeline

pytestmark = pytest.mark.gpu


def _to_dev(d):
    return {k: dev(v) for k, v in d.items()}


@pytest.mark.parametrize("n", [1, 5000, 1_000_000])
def test_plain_pipeline(px, n):
    d = pxdata.plain(n, 0)
    p = PlainPipeline(_to_dev(d), pxdata.CFG1_DATE_LO, pxdata.CFG1_DATE_HI, nparts=8)
    r = p.run()
    assert p.ws.status() == px.PX_OK
    w = oracle.pipeline_plain(d, pxdata.CFG1_DATE_LO, pxdata.CFG1_DATE_HI, 8)
    m = count(r["nsel"])
    assert m == w["sel"].size
    np.testing.assert_array_equal(host(r["sel"], m), w["sel"])
    np.testing.assert_array_equal(host(r["offsets"]), w["offsets"])
    for name in PlainPipeline.NAMES:
        np.testing.assert_array_equal(host(r["parts"][name], m), w["parts"][name])
    assert_groups_equal(r["groups"], w["groups"], 2)


def test_plain_pipeline_repeatable(px):
    d = pxdata.plain(300_000, 0)
    p = PlainPipeline(_to_dev(d), pxdata.CFG1_DATE_LO, pxdata.CFG1_DATE_HI, nparts=8)
    a = [t.clone() for t in p.run()["groups"]["aggs"]]
    for _ in range(3):
        b = p.run()["groups"]["aggs"]
        ng = count(p.run()["groups"]["ngroups"])
        for x, y in zip(a, b):
            # group order may differ between runs; compare sorted multisets
            assert sorted(host(x, ng).tolist()) == sorted(host(y, ng).tolist())
    assert p.ws.status() == px.PX_OK


@pytest.mark.parametrize("sizes", [(2_000, 60_000), (200_000, 6_000_000)])
def test_join_pipeline(px, sizes):
    nd, nf = sizes
    d = pxdata.plain_join(nd, nf)
    p = JoinPipeline(_to_dev(d), pxdata.CFG2_DATE_LO, pxdata.CFG2_DATE_HI)
    r = p.run()
    assert p.ws.status() == px.PX_OK
    w = oracle.pipeline_join(d, pxdata.CFG2_DATE_LO, pxdata.CFG2_DATE_HI)
    m = count(r["join"]["nout"])
    assert m == w["probe_rows"].size == count(r["nsel"])
    np.testing.assert_array_equal(host(r["join"]["cols"][0], m), d["amount"][w["probe_rows"]])
    np.testing.assert_array_equal(host(r["join"]["cols"][1], m), d["attr"][w["build_rows"]])
    assert_groups_equal(r["groups"], w["groups"], 1)


def test_at_scale_pipeline_small(px):
    d = pxdata.plain_at_scale(20_000, 600_000, nattr=1000)
    p = AtScalePipeline(_to_dev(d), nparts=64, nattr_bound=1000)
    r = p.run()
    assert p.ws.status() == px.PX_OK
    w = oracle.pipeline_at_scale(d, 64)
    np.testing.assert_array_equal(host(r["dim_offsets"]), w["dim_offsets"])
    np.testing.assert_array_equal(host(r["fact_offsets"]), w["fact_offsets"])
    np.testing.assert_array_equal(host(r["join"]["out_seg"]), w["join_offsets"])
    assert_groups_equal(r["partial"], w["partial"], 1, segmented=True)
    assert_groups_equal(r["final"], w["final"], 1)


def test_at_scale_pipeline_full_size(px):
    """60M-row Zipf fact x 2M dim, 64 partitions: the configuration the bench times."""
    d = pxdata.plain_at_scale()
    nf, nd = d["fk"].size, d["pk"].size
    p = AtScalePipeline(_to_dev(d), nparts=64)
    r = p.run()
    assert p.ws.status() == px.PX_OK
    # Exchange: the partition of every distinct key comes from the oracle one by one;
    # offsets must equal the per-partition row counts, and whole segments (the
    # hottest partition and two others) must hold exactly the input rows of that
    # partition in input order (stability).
    uniq, inv, cnt = np.unique(d["fk"], return_inverse=True, return_counts=True)
    part_u = oracle.part_of_array(uniq, 0, 64)
    want_foff = np.concatenate([[0], np.cumsum(np.bincount(part_u, weights=cnt, minlength=64).astype(np.int64))])
    np.testing.assert_array_equal(host(r["fact_offsets"]), want_foff)
    part_pk = oracle.part_of_array(d["pk"], 0, 64)
    want_doff = np.concatenate([[0], np.cumsum(np.bincount(part_pk, minlength=64))])
    np.testing.assert_array_equal(host(r["dim_offsets"]), want_doff)
    part_row = part_u[inv]
    hot = int(np.argmax(np.diff(want_foff)))
    for q in sorted({hot, 0, 63}):
        mask = part_row == q
        a, b = int(want_foff[q]), int(want_foff[q + 1])
        for c, name in enumerate(["fk", "amount", "date"]):
            np.testing.assert_array_equal(host(p.fparts[c][a:b]), d[name][mask])
        m = part_pk == q
        for c, name in enumerate(["pk", "attr"]):
            np.testing.assert_array_equal(host(p.dparts[c][int(want_doff[q]):int(want_doff[q + 1])]), d[name][m])
    # Join: every fact row matches once (pk is a permutation), so nout = nf.
    assert count(r["join"]["nout"]) == nf
    # Final groups: closed form via the permutation (attr of fk = attr[pos_of_pk[fk]]).
    pos = np.empty(nd + 1, np.int64)
    pos[d["pk"]] = np.arange(nd)
    attr_of = d["attr"][pos[d["fk"]]]
    sums = np.bincount(attr_of, weights=d["amount"].astype(np.float64), minlength=10_000)
    cnts = np.bincount(attr_of, minlength=10_000)
    fin = r["final"]
    ng = count(fin["ngroups"])
    keys = host(fin["keys"][0], ng)
    order = np.argsort(keys)
    keys = keys[order]
    np.testing.assert_array_equal(keys, np.nonzero(cnts)[0])
    np.testing.assert_array_equal(host(fin["aggs"][1], ng)[order], cnts[keys])
    np.testing.assert_array_equal(host(fin["aggs"][0], ng)[order], sums[keys].astype(np.int64))
    # Partial groups sum to the final ones and count every joined row.
    pc = host(r["partial"]["aggs"][1], count(r["partial"]["ngroups"]))
    assert int(pc.sum()) == nf


@pytest.mark.parametrize("which", ["plain", "join"])
def test_pipelines_replayed_from_a_cuda_graph(px, which):
    # Two copies of the pipeline captured back to back in one CUDA graph (how the
    # bench streams the small workloads): every replay gives the oracle's result.
    if which == "plain":
        ds = [pxdata.plain(200_000, s) for s in (0, 1)]
        pipes = [PlainPipeline(_to_dev(d), pxdata.CFG1_DATE_LO, pxdata.CFG1_DATE_HI, nparts=8) for d in ds]
        wants = [oracle.pipeline_plain(d, pxdata.CFG1_DATE_LO, pxdata.CFG1_DATE_HI, 8) for d in ds]
    else:
        ds = [pxdata.plain_join(20_000, 600_000, seed=s) for s in (2, 3)]
        pipes = [JoinPipeline(_to_dev(d), pxdata.CFG2_DATE_LO, pxdata.CFG2_DATE_HI) for d in ds]
        wants = [oracle.pipeline_join(d, pxdata.CFG2_DATE_LO, pxdata.CFG2_DATE_HI) for d in ds]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for p in pipes:
            p.run(side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        outs = [p.run() for p in pipes]
    for _ in range(2):
        for o in outs:  # poison the outputs: the replay must rewrite them
            for t in o["groups"]["aggs"]:
                t.fill_(-1)
        graph.replay()
        torch.cuda.synchronize()
        for p, o, w, d in zip(pipes, outs, wants, ds):
            assert p.ws.status() == px.PX_OK
            if which == "plain":
                m = count(o["nsel"])
                np.testing.assert_array_equal(host(o["sel"], m), w["sel"])
                np.testing.assert_array_equal(host(o["offsets"]), w["offsets"])
                for name in PlainPipeline.NAMES:
                    np.testing.assert_array_equal(host(o["parts"][name], m), w["parts"][name])
                assert_groups_equal(o["groups"], w["groups"], 2)
            else:
                m = count(o["join"]["nout"])
                assert m == w["probe_rows"].size
                np.testing.assert_array_equal(host(o["join"]["cols"][1], m), d["attr"][w["build_rows"]])
                assert_groups_equal(o["groups"], w["groups"], 1)
