"""Pins of the FP64 oracle's plain force field and integrator against facts
that do not come from the oracle itself: closed forms, finite differences,
conservation laws, symmetry, hand enumeration and the exact discrete solution
of velocity Verlet for a harmonic oscillator."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_18271_b300 import synth
from tests import tiny

KE = O.COULOMB_K


# ------------------------------------------------------------ exclusions / angles

def test_exclusions_hand_enumerated():
    #   0 - 1 - 3 - 4
    #       |
    #       2
    bonds = [(0, 1), (1, 2), (1, 3), (3, 4)]
    off, idx = O.exclusions(5, np.array(bonds))
    got = [sorted(idx[off[i]:off[i + 1]].tolist()) for i in range(5)]
    assert got == [[1, 2, 3], [0, 2, 3, 4], [0, 1, 3], [0, 1, 2, 4], [1, 3]]
    # rows come back ascending and without repeats
    for i in range(5):
        row = idx[off[i]:off[i + 1]].tolist()
        assert row == sorted(set(row))


def test_exclusions_star_and_chain():
    # star: every leaf is 1-3 to every other leaf
    off, idx = O.exclusions(5, np.array([(0, 1), (0, 2), (0, 3), (0, 4)]))
    assert idx[off[0]:off[1]].tolist() == [1, 2, 3, 4]
    assert idx[off[2]:off[3]].tolist() == [0, 1, 3, 4]
    # chain of 6: 1-4 pairs stay in the nonbonded sum
    off, idx = O.exclusions(6, np.array([(i, i + 1) for i in range(5)]))
    assert idx[off[0]:off[1]].tolist() == [1, 2]
    assert idx[off[3]:off[4]].tolist() == [1, 2, 4, 5]
    # no bonds: nothing excluded
    off, idx = O.exclusions(3, np.zeros((0, 2), dtype=np.int32))
    assert off.tolist() == [0, 0, 0, 0] and idx.size == 0


def test_angles_hand_enumerated():
    bonds = [(0, 1), (1, 2), (1, 3), (3, 4)]
    ang = O.angles(5, np.array(bonds)).tolist()
    assert ang == [[0, 1, 2], [0, 1, 3], [2, 1, 3], [1, 3, 4]]
    assert O.angles(4, np.array([(0, 1), (0, 2), (0, 3)])).tolist() == [[1, 0, 2], [1, 0, 3], [2, 0, 3]]


# ------------------------------------------------------------ closed forms

@pytest.mark.parametrize("ei,ej", [(0, 0), (1, 3), (2, 1)])
def test_lj_minimum_closed_form(ei, ej):
    sigma = (2.6, 3.1, 2.9, 3.4)
    eps = (0.07, 0.18, 0.11, 0.15)
    sij = 0.5 * (sigma[ei] + sigma[ej])
    eij = math.sqrt(eps[ei] * eps[ej])
    rmin = 2 ** (1 / 6) * sij
    s = tiny.system([[0, 0, 0], [rmin, 0, 0]], [ei, ej], sigma=sigma, eps=eps)
    e, f, t = O.Plain(s).energy_forces(s.pos)
    assert e == pytest.approx(-eij, rel=1e-13)
    assert np.abs(f).max() < 1e-12
    # E(sigma) = 0 and the repulsive force at r = sigma is 24 eps / sigma
    s.pos[1, 0] = sij
    e, f, _ = O.Plain(s).energy_forces(s.pos)
    assert abs(e) < 1e-14
    assert f[1, 0] == pytest.approx(24 * eij / sij, rel=1e-12)
    assert f[0, 0] == pytest.approx(-24 * eij / sij, rel=1e-12)


def test_coulomb_closed_form():
    r = 4.7
    s = tiny.system([[0, 0, 0], [0, r, 0]], [0, 0], charge=[0.3, -0.45], eps=(0, 0, 0, 0))
    e, f, t = O.Plain(s).energy_forces(s.pos)
    assert e == pytest.approx(KE * 0.3 * -0.45 / r, rel=1e-14)
    # attraction: atom 1 pulled toward atom 0
    assert f[1, 1] == pytest.approx(-KE * 0.3 * 0.45 / r ** 2, rel=1e-13)
    assert t["lj"] == 0.0


def test_bond_closed_form():
    s = tiny.system([[0, 0, 0], [1.3, 0, 0]], [1, 1], bonds=[(0, 1)], r0=[1.1], k=300.0, charge=[1.0, -1.0])
    e, f, t = O.Plain(s).energy_forces(s.pos)
    # bonded pair is excluded: no LJ, no Coulomb
    assert t["lj"] == 0 and t["coulomb"] == 0
    assert e == pytest.approx(0.5 * 300 * 0.2 ** 2, rel=1e-13)
    assert f[0, 0] == pytest.approx(300 * 0.2, rel=1e-13)
    assert f[1, 0] == pytest.approx(-300 * 0.2, rel=1e-13)
    s.pos[1, 0] = 1.1
    e, f, _ = O.Plain(s).energy_forces(s.pos)
    assert e == 0.0 and np.abs(f).max() < 1e-12


def test_angle_closed_form():
    # right angle at the vertex: E = k/2 (pi/2 - theta0)^2 ; 1-3 pair excluded
    th0 = 109.5
    s = tiny.system([[1.2, 0, 0], [0, 0, 0], [0, 1.4, 0]], [0, 1, 0], bonds=[(0, 1), (1, 2)], r0=[1.2, 1.4],
                    charge=[0.5, 0, -0.5], theta0_deg=th0, angle_k=50.0)
    e, f, t = O.Plain(s).energy_forces(s.pos)
    d = math.pi / 2 - math.radians(th0)
    assert t["angle"] == pytest.approx(0.5 * 50 * d * d, rel=1e-13)
    assert t["lj"] == 0 and t["coulomb"] == 0 and t["bond"] == 0
    # the angular force on an end atom is perpendicular to its bond, magnitude k*dtheta/r
    assert f[0, 0] == pytest.approx(0, abs=1e-12)
    assert abs(f[0, 1]) == pytest.approx(50 * abs(d) / 1.2, rel=1e-12)
    # at theta0 the force vanishes
    a = math.radians(th0)
    s.pos[2] = [1.4 * math.cos(a), 1.4 * math.sin(a), 0]
    e, f, _ = O.Plain(s).energy_forces(s.pos)
    assert e == pytest.approx(0, abs=1e-20) and np.abs(f).max() < 1e-9


# ------------------------------------------------------------ FD / conservation / symmetry

@pytest.fixture(scope="module")
def mol64():
    return synth.workload("mol64")


def test_forces_central_differences(mol64):
    p = O.Plain(mol64)
    x = mol64.pos
    _, f, _ = p.energy_forces(x)
    h = 1e-4
    fd = np.zeros_like(f)
    for i in range(mol64.n_atoms):
        for c in range(3):
            xp = x.copy(); xp[i, c] += h
            xm = x.copy(); xm[i, c] -= h
            fd[i, c] = -(p.energy_forces(xp)[0] - p.energy_forces(xm)[0]) / (2 * h)
    # O(h^2) truncation: relative RMS error well below 1e-6
    rel = np.sqrt(((fd - f) ** 2).mean()) / np.sqrt((f ** 2).mean())
    assert rel < 1e-6, rel


def test_net_force_and_torque_vanish(mol64):
    p = O.Plain(mol64)
    _, f, _ = p.energy_forces(mol64.pos)
    scale = np.abs(f).sum()
    assert np.abs(f.sum(axis=0)).max() < 1e-10 * scale
    tau = np.cross(mol64.pos, f).sum(axis=0)
    assert np.abs(tau).max() < 1e-10 * scale * np.abs(mol64.pos).max()


def _rotation(seed):
    q = np.random.default_rng(seed).normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a*a+b*b-c*c-d*d, 2*(b*c-a*d), 2*(b*d+a*c)],
                     [2*(b*c+a*d), a*a-b*b+c*c-d*d, 2*(c*d-a*b)],
                     [2*(b*d-a*c), 2*(c*d+a*b), a*a-b*b-c*c+d*d]])


def test_rotation_translation_invariance(mol64):
    p = O.Plain(mol64)
    e0, f0, _ = p.energy_forces(mol64.pos)
    R = _rotation(7)
    y = mol64.pos @ R.T + np.array([13.0, -4.0, 2.5])
    e1, f1, _ = p.energy_forces(y)
    assert e1 == pytest.approx(e0, rel=1e-11)
    np.testing.assert_allclose(f1, f0 @ R.T, rtol=0, atol=1e-9 * np.abs(f0).max())


def test_permutation_invariance(mol64):
    s = mol64
    perm = np.random.default_rng(3).permutation(s.n_atoms)   # new index k holds old atom perm[k]
    inv = np.argsort(perm)
    t = tiny.system(s.pos[perm], s.element[perm], bonds=inv[s.bonds], r0=s.bond_r0, charge=s.charge[perm],
                    sigma=s.lj_sigma, eps=s.lj_eps)
    e0, f0, _ = O.Plain(s).energy_forces(s.pos)
    e1, f1, _ = O.Plain(t).energy_forces(t.pos)
    assert e1 == pytest.approx(e0, rel=1e-12)
    np.testing.assert_allclose(f1, f0[perm], rtol=0, atol=1e-10 * np.abs(f0).max())


# ------------------------------------------------------------ velocity Verlet

def test_vv_harmonic_diatomic_exact_discrete_solution():
    m1, m2, k, r0, dt = 1.008, 15.999, 300.0, 1.0, 0.5
    d0 = 0.05
    s = tiny.system([[0, 0, 0], [r0 + d0, 0, 0]], [0, 3], bonds=[(0, 1)], r0=[r0], k=k, mass=[m1, m2])
    p = O.Plain(s)
    mu = m1 * m2 / (m1 + m2)
    w2 = k * O.ACC / mu
    wt = math.acos(1 - 0.5 * w2 * dt * dt)
    x = s.pos.copy()
    v = np.zeros((2, 3))
    for n in range(1, 201):
        x, v, U, K, _ = p.vv(x, v, dt, 1)
        r = x[1, 0] - x[0, 0]
        assert r - r0 == pytest.approx(d0 * math.cos(n * wt), abs=1e-13)
    # centre of mass stays put
    com = (m1 * x[0] + m2 * x[1]) / (m1 + m2)
    assert abs(com[0] - m2 * (r0 + d0) / (m1 + m2)) < 1e-13


def test_vv_time_reversible_and_momentum(mol64):
    p = O.Plain(mol64)
    v0 = synth.velocities(mol64.mass, mol64.pos, 300.0, seed=0)
    x1, v1, U, K, _ = p.vv(mol64.pos, v0, 0.5, 100)
    x2, v2, _, _, _ = p.vv(x1, -v1, 0.5, 100)
    assert np.abs(x2 - mol64.pos).max() < 1e-9
    assert np.abs(v2 + v0).max() < 1e-9
    mom0 = (mol64.mass[:, None] * v0).sum(axis=0)
    mom1 = (mol64.mass[:, None] * v1).sum(axis=0)
    assert np.abs(mom1 - mom0).max() < 1e-12


def test_vv_energy_conservation(mol64):
    p = O.Plain(mol64)
    v0 = synth.velocities(mol64.mass, mol64.pos, 300.0, seed=0)
    _, _, U, K, _ = p.vv(mol64.pos, v0, 0.5, 1000)
    H = U + K
    # fluctuation of H is a small fraction of the kinetic-energy scale, and there is no secular drift
    assert np.std(H) < 0.01 * np.mean(K)
    slope = np.polyfit(np.arange(H.size), H, 1)[0] * H.size / mol64.n_atoms
    assert abs(slope) < 2e-3
