"""Host logic of bench.py that runs without a GPU: the group-set comparison the
small workloads use to check graph replays against the eager pipeline, and the
reference arm's line for workloads it does not cover."""
import contextlib
import io
import json

import pytest
import torch


def _groups(keys, aggs):
    return {"ngroups": torch.tensor([len(keys[0])], dtype=torch.int64),
            "keys": [torch.tensor(k) for k in keys], "aggs": [torch.tensor(a, dtype=torch.int64) for a in aggs]}


def test_same_groups_ignores_group_order_only():
    import bench
    a = _groups([[0, 1, 3], [1, 0, 1]], [[10, 20, 30], [1, 2, 3]])
    b = _groups([[3, 0, 1], [1, 1, 0]], [[30, 10, 20], [3, 1, 2]])     # same groups, other order
    assert bench._same_groups(a, b)
    c = _groups([[3, 0, 1], [1, 1, 0]], [[30, 10, 21], [3, 1, 2]])     # one sum differs
    assert not bench._same_groups(a, c)
    d = _groups([[0, 1, 3], [1, 0, 0]], [[10, 20, 30], [1, 2, 3]])     # one key differs
    assert not bench._same_groups(a, d)
    e = _groups([[0, 1], [1, 0]], [[10, 20], [1, 2]])                  # a group missing
    assert not bench._same_groups(a, e)


def test_same_groups_reads_only_the_first_ngroups_rows():
    import bench
    a = _groups([[5, 6]], [[1, 2]])
    b = _groups([[6, 5, 99]], [[2, 1, -7]])
    b["ngroups"] = torch.tensor([2], dtype=torch.int64)
    assert bench._same_groups(a, b)


@pytest.mark.parametrize("workload", ["plain", "plain-join", "fragments", "serve", "late-mat"])
def test_reference_arm_line_for_uncovered_workloads(workload):
    import bench
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.main(["--workload", workload, "--impl", "reference"]) == 0
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unavailable"]


def test_small_workload_algorithmic_bytes_count_each_column_once():
    import bench
    n = {"rows": 1000, "sel": 980}
    b = bench._small_alg_bytes("plain", n)
    assert set(b) == {"px_filter", "px_partition", "px_groupby_agg"}
    assert b["px_filter"] == 4 * 1000 + 4 * 980           # date read, selection written
    assert b["px_partition"] == (4 + 30 + 30) * 980       # selection, 30-byte rows in and out
    assert b["px_groupby_agg"] == (1 + 1 + 8 + 8) * 980   # flag, status, price, qty
    j = bench._small_alg_bytes("plain-join", {"rows": 6000, "dim": 200, "sel": 1800, "out": 1800})
    assert j["px_join_probe"] == 20 * 6000 + 12 * 1800 and j["px_join_build"] == 40 * 200
