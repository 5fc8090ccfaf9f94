"""GPU parity of the three workload pipelines against the oracle.

Reduced sizes and the full workload sizes (1M-row plain batch; 200k x 6M plain
join; 2M x 60M skewed join at 64 partitions, the launch configuration the bench
times) are all compared element by element with the oracle's pipelines.
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
    """60M-row Zipf fact x 2M dim, 64 partitions: the configuration the bench times,
    compared element by element with the oracle's pipeline on the same input: both
    exchanges (offsets and every column of every partition, in order), the join
    (output segment offsets and every joined row), the Partial groups with their
    segments and the Final groups."""
    d = pxdata.plain_at_scale()
    nf, nd = d["fk"].size, d["pk"].size
    p = AtScalePipeline(_to_dev(d), nparts=64)
    r = p.run()
    assert p.ws.status() == px.PX_OK
    w = oracle.pipeline_at_scale(d, 64)
    np.testing.assert_array_equal(host(r["dim_offsets"]), w["dim_offsets"])
    np.testing.assert_array_equal(host(r["fact_offsets"]), w["fact_offsets"])
    for c in range(3):
        np.testing.assert_array_equal(host(p.fparts[c], nf), w["fact_parts"][c])
    for c in range(2):
        np.testing.assert_array_equal(host(p.dparts[c], nd), w["dim_parts"][c])
    m = count(r["join"]["nout"])
    assert m == w["probe_rows"].size == nf  # every fact key names one dimension row
    np.testing.assert_array_equal(host(r["join"]["out_seg"]), w["join_offsets"])
    np.testing.assert_array_equal(host(p.jout[0], m), w["fact_parts"][1][w["probe_rows"]])
    np.testing.assert_array_equal(host(p.jout[1], m), w["dim_parts"][1][w["build_rows"]])
    assert_groups_equal(r["partial"], w["partial"], 1, segmented=True)
    assert_groups_equal(r["final"], w["final"], 1)


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
