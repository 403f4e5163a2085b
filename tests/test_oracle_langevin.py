"""Pins of the oracle's Langevin dynamics (BAOAB with Philox4x32-10 normals).

  - the generator against the published known-answer vectors (tests/golden);
  - the normals' mean, variance and cross-correlation;
  - the zero-friction limit is velocity Verlet;
  - free particles follow the exact Ornstein-Uhlenbeck velocity variance
    (1 - c1^(2t)) kB T / m;
  - a molecule under the thermostat reaches equipartition, <K> = 3N kB T / 2.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_18271_b300 import synth
from tests import tiny

KB = 0.0019872041
ACC = 4.184e-4
HERE = os.path.dirname(os.path.abspath(__file__))


def _kat():
    rows = []
    for line in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        c, k, o = (part.split() for part in line.split("|"))
        rows.append(([int(x, 16) for x in c], [int(x, 16) for x in k], [int(x, 16) for x in o]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert O.philox4x32_10(ctr, key) == out


def test_normals_are_standard_and_uncorrelated():
    z = np.array([O.langevin_normals(7, step, atom) for step in range(40) for atom in range(500)])
    assert abs(z.mean()) < 4 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 4 * np.sqrt(2.0 / z.size)
    c = np.corrcoef(z.T)
    assert np.abs(c - np.eye(3)).max() < 4 / np.sqrt(len(z))
    # different steps, atoms and seeds give different numbers
    assert not np.array_equal(O.langevin_normals(7, 0, 0), O.langevin_normals(7, 1, 0))
    assert not np.array_equal(O.langevin_normals(7, 0, 0), O.langevin_normals(7, 0, 1))
    assert not np.array_equal(O.langevin_normals(7, 0, 0), O.langevin_normals(8, 0, 0))


def test_zero_friction_is_velocity_verlet():
    s = synth.workload("mol64")
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=0)
    plain = O.Plain(s)
    xl, vl, Ul, Kl = plain.langevin(s.pos, v0, 0.5, 50, gamma_ps=1e-14, temp_K=300.0, seed=1)
    xv, vv, Uv, Kv, _ = plain.vv(s.pos, v0, 0.5, 50)
    assert np.abs(xl - xv).max() < 1e-9
    assert np.abs(vl - vv).max() < 1e-9


def test_free_particles_follow_the_ornstein_uhlenbeck_variance():
    n = 600
    pos = np.stack([np.arange(n) * 40.0, np.zeros(n), np.zeros(n)], 1)
    s = tiny.isolated(n, element=np.zeros(n, dtype=np.int32))
    s.lj_eps[:] = 0.0
    gamma, dt, T, steps = 5.0, 0.5, 300.0, 100
    x, v, _, _ = O.Plain(s).langevin(pos, np.zeros((n, 3)), dt, steps, gamma_ps=gamma, temp_K=T, seed=3)
    c1 = np.exp(-gamma * 1e-3 * dt)
    expect = (1.0 - c1 ** (2 * steps)) * KB * T * ACC / s.mass[0]
    var = (v ** 2).mean()
    assert abs(var / expect - 1.0) < 4 * np.sqrt(2.0 / v.size)


def test_thermostat_reaches_equipartition():
    s = synth.workload("mol64")
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=0)
    T = 300.0
    _, _, U, K = O.Plain(s).langevin(s.pos, v0, 0.5, 20000, gamma_ps=10.0, temp_K=T, seed=11)
    k_mean = K[5000:].mean()
    assert abs(k_mean / (1.5 * s.n_atoms * KB * T) - 1.0) < 0.06
