"""The oracle against hand-worked examples stored under tests/golden/."""
import json
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")


def _load():
    with open(GOLDEN) as f:
        return json.load(f)


def test_filter_hand_example():
    g = _load()["filter"]
    sel = oracle.filter(np.array(g["date"], np.int32), g["lo"], g["hi"])
    assert sel.tolist() == g["expected_sel"]


def test_groupby_hand_example():
    g = _load()["groupby_q1"]
    flag, status = np.array(g["flag"], np.int8), np.array(g["status"], np.int8)
    price, qty = np.array(g["price"], np.int64), np.array(g["qty"], np.int64)
    r = oracle.groupby([flag, status], [(oracle.SUM, price, None), (oracle.SUM_MUL, price, qty),
                                        (oracle.SUM, qty, None), (oracle.COUNT, None, None)])
    e = g["expected"]
    assert [list(t) for t in zip(r["keys"][0].tolist(), r["keys"][1].tolist())] == e["keys"]
    assert r["aggs"][0].tolist() == e["sum_price"]
    assert r["aggs"][1].tolist() == e["sum_price_qty"]
    assert r["aggs"][2].tolist() == e["sum_qty"]
    assert r["aggs"][3].tolist() == e["count"]


def test_join_hand_example():
    g = _load()["join_agg"]
    pk, fk = np.array(g["pk"], np.int64), np.array(g["fk"], np.int64)
    pr, br, _ = oracle.join(pk, fk)
    assert [list(p) for p in zip(pr.tolist(), br.tolist())] == g["expected_pairs"]
    attr = np.array(g["attr"], np.int32)[br]
    amount = np.array(g["amount"], np.int64)[pr]
    r = oracle.groupby([attr], [(oracle.SUM, amount, None), (oracle.COUNT, None, None)])
    e = g["expected_groups"]
    assert r["keys"][0].tolist() == e["attr"]
    assert r["aggs"][0].tolist() == e["sum_amount"] and r["aggs"][1].tolist() == e["count"]
