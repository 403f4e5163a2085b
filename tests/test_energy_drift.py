"""The drift measure on synthetic energy traces: a linear H(t) gives its slope
times the length; switch steps (force field changed between consecutive
steps) are removed from the series and reported separately."""
import numpy as np
import pytest

from paper_2412_18271_b300.energy_drift import nve_drift


def test_linear_trace_gives_slope_times_length():
    n, N = 1000, 10
    H = 5.0 + 2e-6 * np.arange(n)          # per atom
    r = nve_drift(H * N, np.zeros(n), N)
    assert r["drift"] == pytest.approx(2e-6 * n, rel=1e-9)
    assert r["drift_excluding_switches"] == r["drift"]


def test_switch_jumps_are_removed_and_counted():
    n, N = 2000, 4
    rng = np.random.default_rng(1)
    H = 1.0 + 1e-7 * rng.normal(size=n)     # conserved up to noise
    plain = np.zeros(n, dtype=bool)
    plain[500:800] = True                    # two switches: entering at 500, leaving at 800
    H = H + np.where(plain, 0.3, 0.0)        # the plain potential sits 0.3 per atom higher
    fb = np.cumsum(plain.astype(np.int64))
    r = nve_drift(H * N, np.zeros(n), N, fallbacks=fb, fallbacks_at_start=0)
    assert r["switch_steps"] == 2
    assert r["plain_steps"] == 300
    assert abs(r["switch_dH_per_atom"]) < 1e-5             # +0.3, then -0.3
    assert r["drift_excluding_switches"] < 1e-5
    assert r["drift"] > 1e-3                                 # the raw fit sees the plateau


def test_start_count_sets_the_first_step():
    n = 100
    fb = np.arange(1, n + 1)                 # every step fell back
    r = nve_drift(np.ones(n), np.zeros(n), 1, fallbacks=fb, fallbacks_at_start=0)
    assert r["plain_steps"] == n and r["switch_steps"] == 0
