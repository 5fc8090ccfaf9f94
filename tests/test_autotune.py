"""Host logic of the launch-configuration autotuner (no GPU): the grid search
picks the fastest runnable point, the per-GPU cache round-trips, and a cached
entry skips the search."""
import json

from paper_2606_24647_gb300 import autotune


def test_grid_points_are_valid_configurations():
    for t, i, c, b in autotune.GRID:
        assert t in (256, 512) and i in (2, 4) and 1 <= b <= 8
        assert c % (t * i) == 0


def test_search_picks_fastest_and_skips_failures():
    times = {p: 1.0 + 0.01 * k for k, p in enumerate(autotune.GRID)}
    fastest = autotune.GRID[7]
    times[fastest] = 0.5
    broken = autotune.GRID[3]

    def time_fn(p):
        if p == broken:
            raise RuntimeError("cannot launch")
        return times[p]

    assert autotune.search(time_fn) == fastest
    times[broken] = 0.1  # would win, but raises
    assert autotune.search(time_fn) == fastest


def test_cache_round_trip_and_reuse(tmp_path):
    path = str(tmp_path / "tune.json")
    key = autotune.gpu_key("NVIDIA GB300", 10, 3, 152)
    calls = []

    def time_fn(p):
        calls.append(p)
        return 1.0 if p != autotune.GRID[5] else 0.2

    best = autotune.cached_or_search(key, "w", time_fn, path=path)
    assert best == autotune.GRID[5] and len(calls) == len(autotune.GRID)
    with open(path) as f:
        assert json.load(f)[f"{key}|w"] == list(best)
    calls.clear()
    assert autotune.cached_or_search(key, "w", time_fn, path=path) == best
    assert calls == []  # served from the cache
    assert autotune.cached_or_search(key, "w", time_fn, path=path, force=True) == best
    assert len(calls) == len(autotune.GRID)


def test_unreadable_cache_is_empty(tmp_path):
    p = tmp_path / "bad.json"
    p.write_text("{not json")
    assert autotune.load_cache(str(p)) == {}


def test_partition_grid_points_are_valid_configurations():
    assert len(set(autotune.PARTITION_GRID)) == len(autotune.PARTITION_GRID)
    for items, bps in autotune.PARTITION_GRID:
        assert items in (2, 4, 8) and 0 <= bps <= 32


def test_partition_and_fragment_entries_share_one_cache_without_clashing(tmp_path):
    path = str(tmp_path / "tune.json")
    key = autotune.gpu_key("NVIDIA GB300", 10, 3, 152)
    a = autotune.cached_or_search(key, "partition|fact", lambda p: 1.0 if p != (4, 3) else 0.1,
                                  grid=autotune.PARTITION_GRID, path=path)
    b = autotune.cached_or_search(key, "fragments512x1", lambda p: 1.0 if p != autotune.GRID[2] else 0.1, path=path)
    assert a == (4, 3) and b == autotune.GRID[2]
    entries = autotune.load_cache(path)
    assert entries[f"{key}|partition|fact"] == [4, 3] and entries[f"{key}|fragments512x1"] == list(autotune.GRID[2])
