"""Seeded synthetic gas-phase systems: molecules, clusters, initial velocities.

This module draws random numbers and builds geometry; it computes none of the
force field, integrator, features or network that the library and the oracle
evaluate.  Both sides read the arrays it returns, so neither can feed the
other its inputs.

Recipe (the workloads of the benchmark configurations, restated):

* A molecule of ``n`` atoms is a random bonded tree: atom ``i >= 1`` bonds to a
  parent drawn uniformly from the atoms ``j < i`` that have fewer than four
  bonds (a tetrahedral centre at most, so every pair of bonds at an atom can
  sit at 109.5 deg).  Elements H/C/N/O are drawn i.i.d.
  with probabilities 0.5/0.3/0.1/0.1.  Bond lengths ``r0 ~ U[1.0, 1.5]`` A,
  bond constant 300 kcal/mol/A^2; one harmonic angle per pair of bonds that
  share an atom, k = 50 kcal/mol/rad^2, theta0 = 109.5 deg.  Charges
  ``U[-0.5, 0.5]`` e, shifted so each molecule is neutral.
* Per system (per seed) each element gets ``sigma ~ U[2.5, 3.5]`` A and
  ``eps ~ U[0.05, 0.2]`` kcal/mol.
* Geometry is built atom by atom: a child sits at its bond length from its
  parent, at 109.5 deg to the parent's own parent bond, at the azimuth (out of
  48 tried) that keeps it farthest from every atom already placed.  The
  coordinates are then cleaned up by least squares on distances only (bonded
  pairs at r0 with weight 100, pairs sharing an atom at the 109.5 deg
  law-of-cosines distance with weight 50, all other pairs of the molecule at
  least 3.2 A apart with weight 50); no force field is evaluated.
* A cluster places ``m`` such molecules, each with its own random tree, with
  a uniform random rotation and a centre drawn uniformly in a ball of the given
  radius; a placement is rejected if an atom leaves the ball or comes closer
  than 3.0 A to an atom of another molecule.
* Velocities are Maxwell-Boltzmann at T, with the centre-of-mass momentum and
  the total angular momentum removed and the kinetic energy rescaled to
  ``(3N - 6) kB T / 2``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.spatial import cKDTree

ELEMENTS = ("H", "C", "N", "O")
MASS = np.array([1.008, 12.011, 14.007, 15.999])
ELEMENT_P = np.array([0.5, 0.3, 0.1, 0.1])
KB = 0.0019872041          # kcal/mol/K
ACC = 4.184e-4             # (kcal/mol/A/amu) -> A/fs^2 ; also kcal/mol -> amu A^2/fs^2
BOND_K = 300.0
ANGLE_K = 50.0
ANGLE_THETA0_DEG = 109.5


@dataclasses.dataclass
class System:
    """A gas-phase system in the units A, fs, amu, e, kcal/mol."""
    element: np.ndarray      # int32 [N]
    mass: np.ndarray         # f64 [N]
    charge: np.ndarray       # f64 [N]
    bonds: np.ndarray        # int32 [nb, 2]
    bond_r0: np.ndarray      # f64 [nb]
    bond_k: np.ndarray       # f64 [nb]
    angle_k: float
    angle_theta0_deg: float
    lj_sigma: np.ndarray     # f64 [4] per element
    lj_eps: np.ndarray       # f64 [4] per element
    pos: np.ndarray          # f64 [N, 3]
    molecule: np.ndarray     # int32 [N] molecule index

    @property
    def n_atoms(self) -> int:
        return int(self.element.shape[0])


MAX_DEGREE = 4


def _tree(rng, n):
    elem = rng.choice(4, size=n, p=ELEMENT_P).astype(np.int32)
    parent = np.full(n, -1, dtype=np.int64)
    degree = np.zeros(n, dtype=np.int64)
    for i in range(1, n):
        free = np.nonzero(degree[:i] < MAX_DEGREE)[0]   # never empty: atom i - 1 has at most one bond yet
        p = int(free[rng.integers(0, free.size)])
        parent[i] = p
        degree[p] += 1
        degree[i] += 1
    r0 = rng.uniform(1.0, 1.5, size=n - 1)
    q = rng.uniform(-0.5, 0.5, size=n)
    q = q - q.mean()
    return elem, parent, r0, q


def _perp_basis(w):
    a = np.array([1.0, 0.0, 0.0]) if abs(w[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(w, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(w, e1)
    return e1, e2


def _random_unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def _place(rng, parent, r0, n_azimuth=48):
    """Distance-only construction of a tree's coordinates (no energy model)."""
    n = parent.shape[0]
    x = np.zeros((n, 3))
    children = [[] for _ in range(n)]
    th0 = math.radians(ANGLE_THETA0_DEG)
    for i in range(1, n):
        p = int(parent[i])
        r = r0[i - 1]
        if parent[p] >= 0:
            ref = int(parent[p])
        elif children[p]:
            ref = children[p][0]
        else:
            ref = -1
        if ref < 0:
            d = _random_unit(rng)
            x[i] = x[p] + r * d
        else:
            w = x[ref] - x[p]
            w /= np.linalg.norm(w)
            e1, e2 = _perp_basis(w)
            phi = rng.uniform(0, 2 * math.pi) + np.arange(n_azimuth) * (2 * math.pi / n_azimuth)
            dirs = (math.cos(th0) * w[None, :]
                    + math.sin(th0) * (np.cos(phi)[:, None] * e1[None, :] + np.sin(phi)[:, None] * e2[None, :]))
            cand = x[p][None, :] + r * dirs                       # [K, 3]
            others = [j for j in range(i) if j != p]
            if others:
                dist = np.linalg.norm(cand[:, None, :] - x[others][None, :, :], axis=-1).min(axis=1)
                k = int(np.argmax(dist))
            else:
                k = 0
            x[i] = cand[k]
        children[p].append(i)
    return x


def _geometry_terms(n, bonds, r0):
    """Target distances of the geometric clean-up: bonded pairs at r0, pairs
    sharing an atom at the law-of-cosines distance for 109.5 deg, every other
    pair at least CONTACT_MIN apart."""
    nbr = [[] for _ in range(n)]
    for b, (i, j) in enumerate(bonds):
        nbr[i].append((j, r0[b]))
        nbr[j].append((i, r0[b]))
    c0 = math.cos(math.radians(ANGLE_THETA0_DEG))
    tgt = {}
    for b, (i, j) in enumerate(bonds):
        tgt[(min(i, j), max(i, j))] = (r0[b], 100.0)
    for v in range(n):
        for p in range(len(nbr[v])):
            for q in range(p + 1, len(nbr[v])):
                (a, ra), (b, rb) = nbr[v][p], nbr[v][q]
                tgt[(min(a, b), max(a, b))] = (math.sqrt(ra * ra + rb * rb - 2 * ra * rb * c0), W_13)
    pi, pj = np.triu_indices(n, 1)
    key = {k: t for k, t in tgt.items()}
    d0 = np.full(pi.shape, CONTACT_MIN)
    w = np.full(pi.shape, 50.0)
    hinge = np.ones(pi.shape, dtype=bool)
    lin = {(int(a), int(b)): k for k, (a, b) in enumerate(zip(pi, pj))}
    for k, (t, wt) in key.items():
        m = lin[k]
        d0[m], w[m], hinge[m] = t, wt, False
    return pi, pj, d0, w, hinge


CONTACT_MIN = 3.2
W_13 = 50.0


def _relax(x, terms):
    """Least-squares geometric clean-up (L-BFGS) of one or several molecules.

    Objective: sum over listed pairs of w (r - d0)^2, where contact pairs only
    count while r < d0.  This is a distance-geometry penalty, not a force field."""
    from scipy.optimize import minimize
    pi, pj, d0, w, hinge = terms
    n = x.shape[0]

    def fun(flat):
        y = flat.reshape(n, 3)
        d = y[pj] - y[pi]
        r = np.sqrt((d * d).sum(axis=1))
        e = r - d0
        e = np.where(hinge & (e > 0), 0.0, e)
        val = (w * e * e).sum()
        coef = (2 * w * e / np.maximum(r, 1e-12))[:, None] * d
        g = np.stack([np.bincount(pj, coef[:, c], n) - np.bincount(pi, coef[:, c], n) for c in range(3)], axis=1)
        return val, g.ravel()

    res = minimize(fun, x.ravel(), jac=True, method="L-BFGS-B", options={"maxiter": 3000, "gtol": 1e-8})
    return res.x.reshape(n, 3)


def make_molecule_parts(rng, n):
    elem, parent, r0, q = _tree(rng, n)
    x = _place(rng, parent, r0)
    bonds = np.stack([parent[1:], np.arange(1, n)], axis=1).astype(np.int32)
    x = _relax(x, _geometry_terms(n, bonds, r0))
    return elem, bonds, r0, q, x


def _element_params(rng):
    sigma = rng.uniform(2.5, 3.5, size=4)
    eps = rng.uniform(0.05, 0.2, size=4)
    return sigma, eps


def molecule(n_atoms: int, seed: int) -> System:
    """One seeded gas-phase molecule (the 64-atom plain and 256-atom learned cases)."""
    rng = np.random.default_rng(seed)
    sigma, eps = _element_params(rng)
    elem, bonds, r0, q, x = make_molecule_parts(rng, n_atoms)
    x = x - x.mean(axis=0)
    return System(element=elem, mass=MASS[elem].copy(), charge=q, bonds=bonds, bond_r0=r0,
                  bond_k=np.full(r0.shape, BOND_K), angle_k=ANGLE_K, angle_theta0_deg=ANGLE_THETA0_DEG,
                  lj_sigma=sigma, lj_eps=eps, pos=x, molecule=np.zeros(n_atoms, dtype=np.int32))


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def cluster(n_molecules: int, atoms_per_molecule: int, radius: float, seed: int,
            min_sep: float = 3.0, max_tries: int = 20000) -> System:
    """Seeded cluster of independent random molecules inside a ball of ``radius`` A."""
    rng = np.random.default_rng(seed)
    sigma, eps = _element_params(rng)
    elems, bonds, r0s, qs, xs, mol = [], [], [], [], [], []
    placed = np.zeros((0, 3))
    tree = None
    offset = 0
    for m in range(n_molecules):
        elem, b, r0, q, x = make_molecule_parts(rng, atoms_per_molecule)
        x = x - x.mean(axis=0)
        for _ in range(max_tries):
            c = rng.normal(size=3)
            c *= radius * rng.uniform() ** (1.0 / 3.0) / np.linalg.norm(c)
            y = x @ _random_rotation(rng).T + c
            if np.any(np.linalg.norm(y, axis=1) > radius):
                continue
            if tree is not None:
                d, _ = tree.query(y, k=1, distance_upper_bound=min_sep)
                if np.any(np.isfinite(d)):
                    continue
            break
        else:
            raise RuntimeError("cluster: could not place molecule %d" % m)
        placed = np.concatenate([placed, y])
        tree = cKDTree(placed)
        elems.append(elem)
        bonds.append(b + offset)
        r0s.append(r0)
        qs.append(q)
        xs.append(y)
        mol.append(np.full(atoms_per_molecule, m, dtype=np.int32))
        offset += atoms_per_molecule
    elem = np.concatenate(elems)
    r0 = np.concatenate(r0s)
    return System(element=elem, mass=MASS[elem].copy(), charge=np.concatenate(qs),
                  bonds=np.concatenate(bonds).astype(np.int32), bond_r0=r0, bond_k=np.full(r0.shape, BOND_K),
                  angle_k=ANGLE_K, angle_theta0_deg=ANGLE_THETA0_DEG, lj_sigma=sigma, lj_eps=eps,
                  pos=np.concatenate(xs), molecule=np.concatenate(mol))


def velocities(mass: np.ndarray, pos: np.ndarray, temperature: float, seed: int) -> np.ndarray:
    """Maxwell-Boltzmann velocities [N,3] in A/fs with zero linear and angular momentum."""
    rng = np.random.default_rng(seed)
    n = mass.shape[0]
    sd = np.sqrt(KB * temperature * ACC / mass)
    v = rng.normal(size=(n, 3)) * sd[:, None]
    m = mass[:, None]
    v -= (m * v).sum(axis=0) / mass.sum()
    if n >= 3:
        com = (m * pos).sum(axis=0) / mass.sum()
        r = pos - com
        L = (m * np.cross(r, v)).sum(axis=0)
        inertia = np.zeros((3, 3))
        for k in range(n):
            inertia += mass[k] * (np.dot(r[k], r[k]) * np.eye(3) - np.outer(r[k], r[k]))
        omega = np.linalg.solve(inertia, L)
        v -= np.cross(omega[None, :], r)
    dof = max(3 * n - 6, 1)
    ke = 0.5 * (m * v * v).sum() / ACC
    target = 0.5 * dof * KB * temperature
    if ke > 0:
        v *= math.sqrt(target / ke)
    return v


# Named workloads: (builder, seed) for the five benchmark configurations.
def workload(name: str, trajectory: int = 0) -> System:
    if name == "mol64":          # plain force field, one 64-atom molecule
        return molecule(64, seed=0)
    if name == "cluster2048":    # plain force field, 64 x 32-atom molecules in a 60 A ball
        return cluster(64, 32, 60.0, seed=100 + trajectory)
    if name == "mol256":         # learned potential, one 256-atom molecule
        return molecule(256, seed=200)
    if name == "cluster16384":   # learned potential, 512 x 32-atom molecules in an 80 A ball
        return cluster(512, 32, 80.0, seed=400)
    raise KeyError(name)


WORKLOAD_VELOCITY_SEED = {"mol64": 0, "cluster2048": 100, "mol256": 200, "cluster16384": 400}
