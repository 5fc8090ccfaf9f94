"""Host logic of the serving loop (no GPU): FIFO admission under the memory
budget, the seeded Poisson arrival process and the latency percentiles."""
import math

import numpy as np
import pytest

from paper_2606_24647_gb300 import serving


def test_admission_budget_fifo_and_release():
    a = serving.Admission(100)
    a.admit(60)
    assert a.fits(40) and not a.fits(41)
    with pytest.raises(RuntimeError):
        a.admit(41)
    a.admit(40)
    assert a.used == 100 and a.peak == 100
    a.release(60)
    assert a.used == 40
    with pytest.raises(ValueError):
        a.admit(101)  # can never fit
    with pytest.raises(RuntimeError):
        a.release(41)


def test_poisson_arrivals_are_seeded_and_have_the_rate():
    t1 = serving.poisson_arrivals(1000.0, 20000, seed=5)
    t2 = serving.poisson_arrivals(1000.0, 20000, seed=5)
    np.testing.assert_array_equal(t1, t2)
    assert np.all(np.diff(t1) >= 0)
    rate = t1.size / t1[-1]
    assert 950 < rate < 1050  # 20k draws: ~0.7 % standard error
    gaps = np.diff(t1)
    assert abs(gaps.std() / gaps.mean() - 1) < 0.05  # exponential gaps: CV = 1
    assert np.all(serving.poisson_arrivals(math.inf, 7, seed=1) == 0)


def test_percentiles():
    p = serving.percentiles([0.001 * i for i in range(1, 101)])
    assert abs(p["p50_ms"] - 50.5) < 1e-9 and abs(p["p99_ms"] - 99.01) < 1e-9
    assert serving.percentiles([])["p50_ms"] is None
