"""Helpers shared by the GPU parity tests (test side only)."""
import numpy as np
import torch


def dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t: torch.Tensor, n=None) -> np.ndarray:
    a = t.cpu().numpy()
    return a if n is None else a[:n]


def count(t: torch.Tensor) -> int:
    return int(t.cpu().item())


def sorted_groups(keys, aggs, n, seg=None):
    """GPU group-by output (unspecified order) -> arrays sorted by (seg, keys...)."""
    ks = [host(k, n).astype(np.int64) for k in keys]
    ag = [host(a, n) for a in aggs]
    sk = host(seg, n).astype(np.int64) if seg is not None else np.zeros(n, np.int64)
    order = np.lexsort(tuple(reversed([sk] + ks))) if n else np.zeros(0, np.int64)
    return sk[order], [k[order] for k in ks], [a[order] for a in ag]


def assert_groups_equal(gpu, oracle_res, nkeys, segmented=False):
    n = count(gpu["ngroups"])
    assert n == oracle_res["ngroups"]
    seg, ks, ag = sorted_groups(gpu["keys"], gpu["aggs"], n, gpu.get("seg") if segmented else None)
    if segmented:
        np.testing.assert_array_equal(seg, oracle_res["seg"].astype(np.int64))
    for k in range(nkeys):
        np.testing.assert_array_equal(ks[k], oracle_res["keys"][k])
    for a in range(len(ag)):
        np.testing.assert_array_equal(ag[a], oracle_res["aggs"][a])
