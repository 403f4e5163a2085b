"""NVE energy drift of a trajectory's energy trace, with the steps where the
learned path's force field switched (plain fallback on or off) taken out.

Drift: |slope of the least-squares line through H(t)/N| times the run length
(kcal/mol/atom over the run).  When every trace entry is one step apart and
the cumulative count of fallback evaluations is known beside each entry
(mdpf_get_trace_fallbacks), each step's force field is known: a step whose
force field differs from its predecessor's is a switch step, and its change
of H (the difference of two potentials, not integration error) is removed
from the series and reported on its own.  Host-side arithmetic on the trace
only; the trace itself comes from the device.
"""
from __future__ import annotations

import numpy as np


def nve_drift(U, K, n_atoms: int, fallbacks=None, fallbacks_at_start: int = 0) -> dict:
    """U, K: the trace (kcal/mol), one entry per step; fallbacks: the cumulative fallback count
    beside each entry, or None (no switches); fallbacks_at_start: the count before the first
    traced step.  Returns drift, drift_excluding_switches, switch_steps, switch_dH_per_atom,
    plain_steps (steps run on the plain force field), steps."""
    H = (np.asarray(U, dtype=np.float64) + np.asarray(K, dtype=np.float64)) / n_atoms
    n = H.size
    out = {"steps": int(n), "drift": None, "drift_excluding_switches": None, "switch_steps": 0,
           "switch_dH_per_atom": 0.0, "plain_steps": 0}
    if n < 3:
        return out
    t = np.arange(n, dtype=np.float64)
    out["drift"] = float(abs(np.polyfit(t, H, 1)[0]) * n)
    if fallbacks is None:
        out["drift_excluding_switches"] = out["drift"]
        return out
    fb = np.asarray(fallbacks, dtype=np.int64)
    plain = np.diff(np.concatenate([[int(fallbacks_at_start)], fb])) > 0   # step k ran on the plain field
    switch = plain[1:] != plain[:-1]                                          # entry k + 1 vs entry k
    dH = np.diff(H)
    Hx = np.concatenate([[H[0]], H[0] + np.cumsum(np.where(switch, 0.0, dH))])
    out["drift_excluding_switches"] = float(abs(np.polyfit(t, Hx, 1)[0]) * n)
    out["switch_steps"] = int(switch.sum())
    out["switch_dH_per_atom"] = float(dH[switch].sum())
    out["plain_steps"] = int(plain.sum())
    return out
