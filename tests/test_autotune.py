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
