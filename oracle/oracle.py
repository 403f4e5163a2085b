"""Python face of the FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg import this module; the library's product path never does.  The
oracle shares no code with the CUDA sources.

The compiled part (``mdpf_oracle.c``) is built with ``gcc -O2
-ffp-contract=off`` so that FP32 expressions that must match bit for bit are
evaluated exactly as written.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mdpf_oracle.c")
LIB = os.path.join(HERE, "libmdpf_oracle.so")

ACC = 4.184e-4
COULOMB_K = 332.06371


def build(force: bool = False) -> str:
    """Compile the C oracle into ``libmdpf_oracle.so`` beside its source."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-std=c11", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


_lib = None


class OrcSystem(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("element", ctypes.c_void_p),
        ("mass", ctypes.c_void_p),
        ("charge", ctypes.c_void_p),
        ("n_bonds", ctypes.c_int32),
        ("bonds", ctypes.c_void_p),
        ("bond_r0", ctypes.c_void_p),
        ("bond_k", ctypes.c_void_p),
        ("n_angles", ctypes.c_int32),
        ("angles", ctypes.c_void_p),
        ("angle_k", ctypes.c_double),
        ("angle_theta0", ctypes.c_double),
        ("lj_sigma", ctypes.c_double * 4),
        ("lj_eps", ctypes.c_double * 4),
        ("coulomb_k", ctypes.c_double),
        ("excl_offset", ctypes.c_void_p),
        ("excl_idx", ctypes.c_void_p),
    ]


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.orc_exclusions.restype = ctypes.c_int
        _lib.orc_angles.restype = ctypes.c_int
        _lib.orc_plain_energy_forces.restype = ctypes.c_double
        _lib.orc_kinetic.restype = ctypes.c_double
        _lib.orc_vv_run.restype = None
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def exclusions(n_atoms: int, bonds: np.ndarray):
    """1-2 and 1-3 partners of every atom as CSR (offset [N+1], idx), rows ascending."""
    bonds = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 2)
    off = np.zeros(n_atoms + 1, dtype=np.int32)
    deg = np.bincount(bonds.ravel(), minlength=n_atoms) if bonds.size else np.zeros(n_atoms, dtype=np.int64)
    cap = int((deg * (deg + 1)).sum() + (deg.sum() * deg.max() if deg.size and deg.max() > 0 else 0)) + 1
    idx = np.zeros(cap, dtype=np.int32)
    tot = lib().orc_exclusions(n_atoms, bonds.shape[0], _p(bonds), _p(off), _p(idx), cap)
    if tot < 0:
        raise RuntimeError("orc_exclusions: capacity")
    return off, idx[:tot].copy()


def angles(n_atoms: int, bonds: np.ndarray) -> np.ndarray:
    """Angles (a, vertex, b) derived from the bond graph, in canonical order."""
    bonds = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 2)
    deg = np.bincount(bonds.ravel(), minlength=n_atoms) if bonds.size else np.zeros(n_atoms, dtype=np.int64)
    cap = int((deg * (deg - 1) // 2).sum()) + 1
    out = np.zeros((cap, 3), dtype=np.int32)
    na = lib().orc_angles(n_atoms, bonds.shape[0], _p(bonds), _p(out), cap)
    if na < 0:
        raise RuntimeError("orc_angles: capacity")
    return out[:na].copy()


class Plain:
    """The plain analytic force field of a ``synth.System`` evaluated in FP64."""

    def __init__(self, system, coulomb_k: float = COULOMB_K):
        s = system
        self.n = s.n_atoms
        self.element = np.ascontiguousarray(s.element, dtype=np.int32)
        self.mass = np.ascontiguousarray(s.mass, dtype=np.float64)
        self.charge = np.ascontiguousarray(s.charge, dtype=np.float64)
        self.bonds = np.ascontiguousarray(s.bonds, dtype=np.int32).reshape(-1, 2)
        self.bond_r0 = np.ascontiguousarray(s.bond_r0, dtype=np.float64)
        self.bond_k = np.ascontiguousarray(s.bond_k, dtype=np.float64)
        self.angles = angles(self.n, self.bonds)
        self.excl_offset, self.excl_idx = exclusions(self.n, self.bonds)
        if self.excl_idx.size == 0:
            self.excl_idx = np.zeros(1, dtype=np.int32)
        st = OrcSystem()
        st.n = self.n
        st.element = self.element.ctypes.data
        st.mass = self.mass.ctypes.data
        st.charge = self.charge.ctypes.data
        st.n_bonds = self.bonds.shape[0]
        st.bonds = self.bonds.ctypes.data
        st.bond_r0 = self.bond_r0.ctypes.data
        st.bond_k = self.bond_k.ctypes.data
        st.n_angles = self.angles.shape[0]
        st.angles = self.angles.ctypes.data if self.angles.size else 0
        st.angle_k = float(s.angle_k)
        st.angle_theta0 = float(np.radians(s.angle_theta0_deg))
        for e in range(4):
            st.lj_sigma[e] = float(s.lj_sigma[e])
            st.lj_eps[e] = float(s.lj_eps[e])
        st.coulomb_k = float(coulomb_k)
        st.excl_offset = self.excl_offset.ctypes.data
        st.excl_idx = self.excl_idx.ctypes.data
        self._st = st

    def energy_forces(self, pos):
        """(E, F [N,3], terms {bond, angle, lj, coulomb}) at positions ``pos`` [N,3] in A."""
        x = np.ascontiguousarray(pos, dtype=np.float64).reshape(self.n, 3)
        f = np.zeros((self.n, 3))
        terms = np.zeros(4)
        e = lib().orc_plain_energy_forces(ctypes.byref(self._st), _p(x), _p(f), _p(terms))
        return e, f, dict(zip(("bond", "angle", "lj", "coulomb"), terms.tolist()))

    def kinetic(self, vel):
        v = np.ascontiguousarray(vel, dtype=np.float64)
        return lib().orc_kinetic(self.n, _p(self.mass), _p(v))

    def vv(self, pos, vel, dt: float, n_steps: int):
        """Velocity Verlet; returns (x, v, U[n_steps], K[n_steps], F at final x)."""
        x = np.array(pos, dtype=np.float64, copy=True).reshape(self.n, 3)
        v = np.array(vel, dtype=np.float64, copy=True).reshape(self.n, 3)
        U = np.zeros(max(n_steps, 1))
        K = np.zeros(max(n_steps, 1))
        f = np.zeros((self.n, 3))
        lib().orc_vv_run(ctypes.byref(self._st), ctypes.c_double(dt), n_steps, _p(x), _p(v), _p(U), _p(K), _p(f))
        return x, v, U[:n_steps], K[:n_steps], f
