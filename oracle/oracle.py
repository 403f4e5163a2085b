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
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
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


def set_threads(n: int) -> int:
    """Threads of the oracle's O(N^2) and per-atom loops (1, the default, runs them serially as
    written; the CPU-baseline timing uses more).  Returns the count in effect."""
    L = lib()
    L.orc_set_threads.restype = ctypes.c_int
    return int(L.orc_set_threads(ctypes.c_int32(int(n))))


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

    def langevin(self, pos, vel, dt: float, n_steps: int, gamma_ps: float, temp_K: float, seed: int,
                 step0: int = 0):
        """BAOAB Langevin dynamics with Philox normals; returns (x, v, U[n_steps], K[n_steps])."""
        L = lib()
        L.orc_langevin_run.restype = None
        x = np.array(pos, dtype=np.float64, copy=True).reshape(self.n, 3)
        v = np.array(vel, dtype=np.float64, copy=True).reshape(self.n, 3)
        U = np.zeros(max(n_steps, 1))
        K = np.zeros(max(n_steps, 1))
        L.orc_langevin_run(ctypes.byref(self._st), ctypes.c_double(dt), n_steps, ctypes.c_double(gamma_ps),
                           ctypes.c_double(temp_K), ctypes.c_uint64(seed), ctypes.c_int64(step0), _p(x), _p(v),
                           _p(U), _p(K))
        return x, v, U[:n_steps], K[:n_steps]

    def vv(self, pos, vel, dt: float, n_steps: int):
        """Velocity Verlet; returns (x, v, U[n_steps], K[n_steps], F at final x)."""
        x = np.array(pos, dtype=np.float64, copy=True).reshape(self.n, 3)
        v = np.array(vel, dtype=np.float64, copy=True).reshape(self.n, 3)
        U = np.zeros(max(n_steps, 1))
        K = np.zeros(max(n_steps, 1))
        f = np.zeros((self.n, 3))
        lib().orc_vv_run(ctypes.byref(self._st), ctypes.c_double(dt), n_steps, _p(x), _p(v), _p(U), _p(K), _p(f))
        return x, v, U[:n_steps], K[:n_steps], f


# ---------------------------------------------------------------- learned potential

N_FEAT = 384
RC_LIST = 6.2           # neighbour-list radius (5.2 A cutoff + 1 A skin)


class OrcMLP(ctypes.Structure):
    _fields_ = [
        ("n_feat", ctypes.c_int32), ("h1", ctypes.c_int32), ("h2", ctypes.c_int32), ("alpha", ctypes.c_double),
        ("W1", ctypes.c_void_p * 4), ("b1", ctypes.c_void_p * 4), ("W2", ctypes.c_void_p * 4),
        ("b2", ctypes.c_void_p * 4), ("W3", ctypes.c_void_p * 4), ("b3", ctypes.c_double * 4),
        ("e0", ctypes.c_double * 4),
    ]


def _learned_lib():
    L = lib()
    for name in ("orc_mlp_energy", "orc_learned_energy_forces", "orc_core_energy_forces"):
        getattr(L, name).restype = ctypes.c_double
    L.orc_core_energy_forces.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_void_p]
    for name in ("orc_features", "orc_feature_forces", "orc_feature_jvp"):
        getattr(L, name).restype = None
    L.orc_neighbors.restype = ctypes.c_int
    return L


def neighbors(pos32, rc_list: float = RC_LIST, max_per_atom: int = 256):
    """Brute-force neighbour rows (list of ascending int arrays) with the FP32 predicate
    d2 = fl(fl(fl(dx*dx) + fl(dy*dy)) + fl(dz*dz)) < fl32(rc^2)."""
    x = np.ascontiguousarray(pos32, dtype=np.float32).reshape(-1, 3)
    n = x.shape[0]
    cnt = np.zeros(n, dtype=np.int32)
    idx = np.zeros((n, max_per_atom), dtype=np.int32)
    rc2 = np.float32(rc_list * rc_list)
    tot = _learned_lib().orc_neighbors(n, _p(x), ctypes.c_float(rc2), max_per_atom, _p(cnt), _p(idx))
    if tot < 0:
        raise RuntimeError("orc_neighbors: row longer than max_per_atom")
    return [idx[i, :cnt[i]].copy() for i in range(n)]


def features(element, pos):
    el = np.ascontiguousarray(element, dtype=np.int32)
    x = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    G = np.zeros((x.shape[0], N_FEAT))
    _learned_lib().orc_features(x.shape[0], _p(el), _p(x), _p(G))
    return G


def feature_forces(element, pos, w):
    """F = -sum_{i,f} w[i,f] dG[i,f]/dx."""
    el = np.ascontiguousarray(element, dtype=np.int32)
    x = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    w = np.ascontiguousarray(w, dtype=np.float64)
    F = np.zeros_like(x)
    _learned_lib().orc_feature_forces(x.shape[0], _p(el), _p(x), _p(w), _p(F))
    return F


def feature_jvp(element, pos, u):
    """Gdot[i,f] = sum_a dG[i,f]/dx_a . u_a."""
    el = np.ascontiguousarray(element, dtype=np.int32)
    x = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1, 3)
    Gd = np.zeros((x.shape[0], N_FEAT))
    _learned_lib().orc_feature_jvp(x.shape[0], _p(el), _p(x), _p(u), _p(Gd))
    return Gd


def core_energy_forces(pos, A: float, rc: float):
    """Repulsive core sum_{i<j, r<rc} A (1 - r/rc)^3 (rc/r): (E, F [N,3])."""
    x = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    F = np.zeros_like(x)
    E = _learned_lib().orc_core_energy_forces(x.shape[0], _p(x), float(A), float(rc), _p(F))
    return E, F


class Learned:
    """The learned potential of a ``model.Model`` evaluated in FP64 (weights taken as stored):
    the per-element MLP on the symmetry functions plus the model's repulsive core, if it has one."""

    def __init__(self, model):
        self.m = model
        self._arr = {}
        st = OrcMLP()
        st.n_feat, st.h1, st.h2, st.alpha = N_FEAT, model.W1.shape[1], model.W2.shape[1], float(model.alpha)
        for e in range(4):
            for name in ("W1", "b1", "W2", "b2", "W3"):
                a = np.ascontiguousarray(getattr(model, name)[e], dtype=np.float64)
                self._arr[(name, e)] = a
                getattr(st, name)[e] = a.ctypes.data
            st.b3[e] = float(model.b3[e])
            st.e0[e] = float(model.e0[e])
        self._st = st

    def mlp(self, element, G):
        """(E_total, E_i [N], dE/dG [N,384])."""
        el = np.ascontiguousarray(element, dtype=np.int32)
        G = np.ascontiguousarray(G, dtype=np.float64)
        n = el.shape[0]
        Ei = np.zeros(n)
        dG = np.zeros((n, N_FEAT))
        E = _learned_lib().orc_mlp_energy(ctypes.byref(self._st), n, _p(el), _p(G), _p(Ei), _p(dG))
        return E, Ei, dG

    def energy_forces(self, element, pos):
        """(E, F [N,3], G [N,384])."""
        el = np.ascontiguousarray(element, dtype=np.int32)
        x = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        F = np.zeros_like(x)
        G = np.zeros((x.shape[0], N_FEAT))
        E = _learned_lib().orc_learned_energy_forces(ctypes.byref(self._st), x.shape[0], _p(el), _p(x), _p(F), _p(G))
        if getattr(self.m, "core_rc", 0.0) > 0.0:
            Ec, Fc = core_energy_forces(x, self.m.core_a, self.m.core_rc)
            E += Ec
            F += Fc
        return E, F, G


# ---------------------------------------------------------------- training loss and gradient

def _grad_arrays(model):
    return {"W1": np.zeros((4,) + model.W1.shape[1:]), "b1": np.zeros((4, model.W1.shape[1])),
            "W2": np.zeros((4,) + model.W2.shape[1:]), "b2": np.zeros((4, model.W2.shape[1])),
            "W3": np.zeros((4, model.W2.shape[1])), "b3": np.zeros(4)}


def mlp_param_grad(model, element, G, U, c, out=None):
    """Parameter gradient of sum_i [c_i E_i - U_i . dE_i/dG_i] (accumulated into ``out``)."""
    L = _learned_lib()
    L.orc_mlp_param_grad.restype = None
    lrn = Learned(model)
    el = np.ascontiguousarray(element, dtype=np.int32)
    G = np.ascontiguousarray(G, dtype=np.float64)
    U = np.ascontiguousarray(U, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    g = _grad_arrays(model) if out is None else out
    L.orc_mlp_param_grad(ctypes.byref(lrn._st), el.shape[0], _p(el), _p(G), _p(U), _p(c),
                         _p(g["W1"]), _p(g["b1"]), _p(g["W2"]), _p(g["b2"]), _p(g["W3"]), _p(g["b3"]))
    return g


def train_loss_grad(model, frames, w_force: float = 10.0):
    """Force-matching loss over a batch of frames and its parameter gradient (FP64).

    frames: list of (element [N], pos [N,3], E_ref, F_ref [N,3]).
      L = (1/B) sum_f ((E_f - E_ref,f) / N_f)^2  +  w_force * mean over all force components (F - F_ref)^2
    Steps per frame: features G; energies and dE/dG; forces F = -J^T dE/dG (plus the
    model's repulsive core in E and F, which has no parameters); the loss terms;
    v = dL/dF; U = J v (feature JVP); then the MLP parameter
    gradient of sum_i [c E_i - U_i . dE_i/dG_i] with c = dL/dE_f.
    Returns (L, grads dict, per-frame (E, F)).
    """
    B = len(frames)
    n_comp = sum(3 * f[0].shape[0] for f in frames)
    lrn = Learned(model)
    loss = 0.0
    grads = _grad_arrays(model)
    outs = []
    for el, pos, e_ref, f_ref in frames:
        n = el.shape[0]
        G = features(el, pos)
        E, _, dG = lrn.mlp(el, G)
        F = feature_forces(el, pos, dG)
        if getattr(model, "core_rc", 0.0) > 0.0:   # no parameters, but part of E and F
            Ec, Fc = core_energy_forces(pos, model.core_a, model.core_rc)
            E += Ec
            F = F + Fc
        loss += ((E - e_ref) / n) ** 2 / B + w_force * float(((F - f_ref) ** 2).sum()) / n_comp
        c = np.full(n, 2.0 * (E - e_ref) / (n * n) / B)
        v = 2.0 * w_force * (F - f_ref) / n_comp
        U = feature_jvp(el, pos, v)
        mlp_param_grad(model, el, G, U, c, out=grads)
        outs.append((E, F))
    return loss, grads, outs


# ---------------------------------------------------------------- AdamW with cosine decay

def cosine_lr(t: int, lr_max: float, T: int) -> float:
    """lr_t = lr_max * (1 + cos(pi t / T)) / 2, t = 0 .. T (0 afterwards)."""
    if t >= T:
        return 0.0
    return lr_max * 0.5 * (1.0 + np.cos(np.pi * t / T))


def adamw_step(theta, grad, m, v, t: int, lr: float, betas=(0.9, 0.999), eps=1e-8, wd=0.01):
    """One AdamW update (decoupled weight decay) at step t (1-based), in place:
    m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2;  mh = m / (1 - b1^t);  vh = v / (1 - b2^t)
    theta = theta - lr (mh / (sqrt(vh) + eps) + wd theta)."""
    b1, b2 = betas
    m *= b1
    m += (1.0 - b1) * grad
    v *= b2
    v += (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    theta -= lr * (mh / (np.sqrt(vh) + eps) + wd * theta)
    return theta


# ---------------------------------------------------------------- counter-based normals

def philox4x32_10(ctr, key):
    """Philox4x32-10 of counter (4 x uint32) and key (2 x uint32) -> 4 x uint32."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    out = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, out)
    return [int(v) for v in out]


def init_velocities(mass, pos, temperature: float, seed: int):
    """Maxwell-Boltzmann velocities [N,3] (A/fs) from counter-based normals, zero linear and angular
    momentum, K = (3N - 6) kB T / 2."""
    m = np.ascontiguousarray(mass, dtype=np.float64)
    x = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    v = np.zeros_like(x)
    L = lib()
    L.orc_init_velocities.restype = None
    L.orc_init_velocities(ctypes.c_int32(m.shape[0]), _p(m), _p(x), ctypes.c_double(temperature),
                          ctypes.c_uint64(seed), _p(v))
    return v


def langevin_normals(seed: int, step: int, atom: int):
    z = (ctypes.c_double * 3)()
    lib().orc_langevin_normals(ctypes.c_uint64(seed), ctypes.c_int64(step), ctypes.c_int32(atom), z)
    return np.array(list(z))
