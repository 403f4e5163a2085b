"""Hand-built tiny systems for closed-form checks."""
import numpy as np

from paper_2412_18271_b300 import synth


def system(pos, element, bonds=(), r0=None, k=300.0, charge=None, sigma=(3.0, 3.0, 3.0, 3.0),
           eps=(0.1, 0.1, 0.1, 0.1), angle_k=50.0, theta0_deg=109.5, mass=None):
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    n = pos.shape[0]
    element = np.asarray(element, dtype=np.int32)
    bonds = np.asarray(bonds, dtype=np.int32).reshape(-1, 2)
    nb = bonds.shape[0]
    if r0 is None:
        r0 = np.full(nb, 1.2)
    return synth.System(
        element=element,
        mass=np.asarray(mass if mass is not None else synth.MASS[element], dtype=np.float64),
        charge=np.asarray(charge if charge is not None else np.zeros(n), dtype=np.float64),
        bonds=bonds, bond_r0=np.asarray(r0, dtype=np.float64).reshape(nb),
        bond_k=np.full(nb, float(k)), angle_k=float(angle_k), angle_theta0_deg=float(theta0_deg),
        lj_sigma=np.asarray(sigma, dtype=np.float64), lj_eps=np.asarray(eps, dtype=np.float64),
        pos=pos, molecule=np.zeros(n, dtype=np.int32))


def isolated(n, element=None, charge=None):
    """n unbonded atoms (positions at the origin; callers pass their own)."""
    el = np.zeros(n, dtype=np.int32) if element is None else np.asarray(element, dtype=np.int32)
    return system(np.zeros((n, 3)), el, charge=charge)
