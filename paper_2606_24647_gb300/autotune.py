"""Grid-search autotuner for the launch configurations of px_fragments_run and
px_partition.

The fused fragment kernel has four knobs (threads per block, rows per thread per
tile, rows per work item - the fan-out of a fragment into work items - and
resident blocks per SM); the exchange has two (rows per thread of its tiles, and
resident blocks per SM). Every configuration computes the same results; they differ only in
speed, and the best one depends on the GPU and on the workload. The tuner times
each point of a small grid on the caller's own inputs with CUDA events and keeps
the fastest, caching it per GPU (name, compute capability, SM count) and
workload in a JSON file so later runs skip the search.
"""
from __future__ import annotations

import json
import os

GRID = [(t, i, c, b) for t in (256, 512) for i in (2, 4) for c in (0, 16384, 65536, 262144) for b in (1, 2, 4, 8)]
# px_partition: (rows per thread, most resident blocks per SM; 0 = as many as fit);
# rows per thread wider than the columns allow are narrowed by the library.
PARTITION_GRID = [(4, 0), (4, 3), (4, 2), (8, 0), (8, 2)]


def cache_path() -> str:
    return os.environ.get("PX_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "px_gb300", "tune.json"))


def gpu_key(name: str, major: int, minor: int, sms: int) -> str:
    return f"{name}|sm_{major}{minor}|{sms}SM"


def search(time_fn, grid=GRID) -> tuple:
    """The grid point with the smallest time_fn(point) (seconds); ties keep the
    earlier point. time_fn may raise for a point that cannot run; it is skipped."""
    best, best_t = None, float("inf")
    for point in grid:
        try:
            t = time_fn(point)
        except Exception:  # a configuration this GPU cannot launch
            continue
        if t < best_t:
            best, best_t = point, t
    if best is None:
        raise RuntimeError("no configuration of the grid could run")
    return best


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(entries: dict, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(entries, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def cached_or_search(key: str, workload: str, time_fn, grid=GRID, path: str | None = None,
                     force: bool = False) -> tuple:
    """The cached best point for (GPU key, workload name), else search and cache it."""
    entries = load_cache(path)
    slot = f"{key}|{workload}"
    if not force and slot in entries:
        return tuple(entries[slot])
    best = search(time_fn, grid)
    entries[slot] = list(best)
    store_cache(entries, path)
    return best


def tune_fragments(batch, workload: str, reps: int = 3, grid=GRID, force: bool = False) -> tuple:
    """Best launch configuration for a FragmentBatch on the current GPU (cached)."""
    import torch

    stream = torch.cuda.current_stream()

    def time_fn(point):
        return _time_calls(lambda: batch.run(stream, config=point), reps)

    return cached_or_search(_gpu_key(), workload, time_fn, grid, force=force)


def _gpu_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return gpu_key(p.name, p.major, p.minor, p.multi_processor_count)


def _time_calls(run, reps: int) -> float:
    import torch
    stream = torch.cuda.current_stream()
    run()  # warm-up (also surfaces launch errors)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        run()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1000.0 / reps


def tune_partition(cols, key_col: int, nparts: int, workload: str, reps: int = 5, grid=PARTITION_GRID,
                   force: bool = False) -> tuple:
    """Best (rows per thread, blocks per SM) for px_partition of these columns into
    nparts partitions on the current GPU (cached per GPU and workload)."""
    import torch

    from . import Workspace, load, px_partition
    L = load()
    n = cols[0].numel()
    out = [torch.empty(max(n, 1), dtype=c.dtype, device=c.device) for c in cols]
    off = torch.empty(nparts + 1, dtype=torch.int64, device=cols[0].device)
    ws = Workspace(L.px_partition_ws_bytes(n, nparts))

    def time_fn(point):
        return _time_calls(lambda: px_partition(cols, key_col, nparts, out=out, offsets=off, config=point, ws=ws),
                           reps)

    return cached_or_search(_gpu_key(), f"partition|{workload}", time_fn, grid, force=force)
