"""Pins of the oracle's Maxwell-Boltzmann initial velocities (counter-based
normals, centre-of-mass and angular momentum removed, kinetic energy set to
(3N - 6) kB T / 2) against what the definition fixes: conservation quantities,
the exact kinetic energy, the Maxwell-Boltzmann shape per mass (equipartition
between light and heavy atoms, normal scaled components), reproducibility."""
import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_2412_18271_b300 import synth

KB = 0.0019872041
ACC = 4.184e-4


def _momenta(mass, pos, v):
    m = mass[:, None]
    com = (m * pos).sum(0) / mass.sum()
    P = (m * v).sum(0)
    L = (m * np.cross(pos - com, v)).sum(0)
    K = 0.5 * (m * v * v).sum() / ACC
    return P, L, K


@pytest.mark.parametrize("name,T", [("mol64", 300.0), ("mol256", 50.0), ("cluster2048", 300.0)])
def test_zero_momenta_and_exact_kinetic_energy(name, T):
    s = synth.workload(name)
    v = O.init_velocities(s.mass, s.pos, T, seed=11)
    P, L, K = _momenta(s.mass, s.pos, v)
    scale = np.abs(s.mass[:, None] * v).sum()
    assert np.abs(P).max() <= 1e-13 * scale
    assert np.abs(L).max() <= 1e-12 * scale * np.abs(s.pos).max()
    assert K == pytest.approx(0.5 * (3 * s.n_atoms - 6) * KB * T, rel=1e-12)


def test_maxwell_boltzmann_shape_per_mass():
    # 20,000 atoms of two masses 16x apart, far apart (no effect of the rotation removal on the shape):
    # sqrt(m / (kB T)) v must be standard normal for both, and both must carry the same mean kinetic energy
    n = 20000
    mass = np.where(np.arange(n) % 2 == 0, 1.008, 15.999)
    pos = np.random.default_rng(0).uniform(-500, 500, size=(n, 3))
    T = 300.0
    v = O.init_velocities(mass, pos, T, seed=3)
    z = v * np.sqrt(mass / (KB * T * ACC))[:, None]
    for sel in (mass < 2, mass > 2):
        assert stats.kstest(z[sel].ravel(), "norm").pvalue > 1e-3
    ke = 0.5 * (mass[:, None] * v * v).sum(1) / ACC
    assert ke[mass < 2].mean() == pytest.approx(ke[mass > 2].mean(), rel=0.03)
    assert ke.mean() == pytest.approx(1.5 * KB * T * (3 * n - 6) / (3 * n), rel=1e-9)


def test_reproducible_and_seeded():
    s = synth.workload("mol64")
    a = O.init_velocities(s.mass, s.pos, 300.0, seed=5)
    b = O.init_velocities(s.mass, s.pos, 300.0, seed=5)
    c = O.init_velocities(s.mass, s.pos, 300.0, seed=6)
    assert np.array_equal(a, b)
    assert not np.allclose(a, c)


def test_small_and_degenerate_systems():
    m2 = np.array([1.008, 12.011])
    v = O.init_velocities(m2, np.array([[0.0, 0, 0], [1.1, 0, 0]]), 300.0, seed=1)
    P, _, K = _momenta(m2, np.array([[0.0, 0, 0], [1.1, 0, 0]]), v)
    assert np.abs(P).max() < 1e-15 and K == pytest.approx(0.5 * KB * 300.0, rel=1e-12)
    # collinear atoms: the inertia tensor is singular; the rotation step is skipped, nothing is NaN
    m3 = np.array([1.008, 12.011, 15.999])
    x3 = np.array([[0.0, 0, 0], [1.1, 0, 0], [2.3, 0, 0]])
    v3 = O.init_velocities(m3, x3, 300.0, seed=1)
    assert np.all(np.isfinite(v3))
    P, _, K = _momenta(m3, x3, v3)
    assert np.abs(P).max() < 1e-14 and K == pytest.approx(0.5 * 3 * KB * 300.0, rel=1e-12)
    v1 = O.init_velocities(np.array([1.008]), np.zeros((1, 3)), 300.0, seed=1)
    assert np.all(v1 == 0.0)
