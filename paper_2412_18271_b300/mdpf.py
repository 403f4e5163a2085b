"""Thin ctypes binding of libmdpf (include/mdpf.h), same names as the C ABI.

Only argument marshalling happens here; every step of the path runs in the
CUDA kernels of the library.  There is no fallback: if ``libmdpf.so`` is
missing or cannot be loaded, loading the binding raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmdpf.so")

MDPF_OK = 0
ERRORS = {
    -1: "INVALID_ARG", -2: "CUDA", -3: "OOM", -4: "NEIGHBOR_OVERFLOW", -5: "NONFINITE", -6: "TIMEOUT",
    -7: "OUT_OF_RANGE", -8: "UNSUPPORTED", -9: "CALLBACK",
}
MDPF_STATUS_NONFINITE = 0x1
MDPF_STATUS_NEIGHBOR_OVERFLOW = 0x2
MDPF_STATUS_TIMEOUT = 0x4
MDPF_STATUS_OUT_OF_RANGE = 0x8
MDPF_MODE_PLAIN = 0
MDPF_MODE_LEARNED = 1
MDPF_MODE_CALLBACK = 2
FORCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
MDPF_PROF_NONBONDED = 0
MDPF_PROF_STEPPER = 1
MDPF_PROF_STEP = 2
MDPF_PROF_LEARN_NEIGHBORS = 3
MDPF_PROF_LEARN_FEATURES = 4
MDPF_PROF_LEARN_MLP = 5
MDPF_PROF_LEARN_ADJOINT = 6
MDPF_PROF_LEARN_FUSED = 7
MDPF_STEPPER_PERSISTENT = 0
MDPF_STEPPER_KERNELS = 1
MDPF_INTEGRATOR_VERLET = 0
MDPF_INTEGRATOR_LANGEVIN = 1
MDPF_MLP_TENSOR = 0
MDPF_MLP_SIMT = 1
MDPF_MLP_SIMT_FP32 = 2
MDPF_MLP_FUSED = 3

_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_f64 = ctypes.c_double


class MdpfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code
        self.name = ERRORS.get(code, "?")


class mdpf_topology(ctypes.Structure):
    _fields_ = [
        ("n_atoms", _i32), ("element", _vp), ("mass", _vp), ("charge", _vp),
        ("n_bonds", _i32), ("bonds", _vp), ("bond_r0", _vp), ("bond_k", _vp),
        ("angle_k", _f64), ("angle_theta0_deg", _f64),
        ("lj_sigma", _f64 * 4), ("lj_eps", _f64 * 4),
    ]


class mdpf_params(ctypes.Structure):
    _fields_ = [
        ("mode", _i32), ("dt_fs", _f64), ("coulomb_k", _f64), ("trace_capacity", _i32),
        ("record_every", _i32), ("max_frames", _i32), ("stepper", _i32), ("energy_every", _i32),
        ("model", _vp), ("model_bytes", ctypes.c_uint64), ("skin", _f64), ("rebuild_every", _i32),
        ("fallback", _i32), ("mlp_kernel", _i32),
        ("integrator", _i32), ("friction_per_ps", _f64), ("temperature_K", _f64), ("seed", ctypes.c_uint64),
        ("provider", _vp), ("provider_user", _vp), ("provider_pos", _vp), ("provider_energy", _vp),
        ("provider_forces", _vp),
    ]


class mdpf_train_params(ctypes.Structure):
    _fields_ = [("max_frames", _i32), ("atoms_per_frame", _i32), ("w_force", _f64), ("e0", _f64 * 4),
                ("core_a", _f64), ("core_rc", _f64)]


TRAIN_PARAMS_PER_ELEMENT = 131585


class mdpf_counters(ctypes.Structure):
    _fields_ = [
        ("steps", _i64), ("force_evals", _i64), ("frames", _i64), ("status", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32), ("potential", _f64), ("kinetic", _f64), ("h_initial", _f64),
        ("h_now", _f64), ("rebuilds", _i64), ("fallbacks", _i64), ("max_disp", _f64),
    ]


def load(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise ImportError("libmdpf.so not built at %s (run python -m paper_2412_18271_b300.build)" % path)
    lib = ctypes.CDLL(path)
    sig = {
        "mdpf_create": (ctypes.c_int, [ctypes.POINTER(mdpf_topology), ctypes.POINTER(mdpf_params), ctypes.POINTER(_vp)]),
        "mdpf_destroy": (None, [_vp]),
        "mdpf_last_error": (ctypes.c_char_p, [_vp]),
        "mdpf_sizes": (ctypes.c_int, [_vp, _vp, _vp]),
        "mdpf_compute": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
        "mdpf_compute_device": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
        "mdpf_set_state": (ctypes.c_int, [_vp, _vp, _vp]),
        "mdpf_get_state": (ctypes.c_int, [_vp, _vp, _vp]),
        "mdpf_step": (ctypes.c_int, [_vp, _i64]),
        "mdpf_step_async": (ctypes.c_int, [_vp, _i64, _vp]),
        "mdpf_get_counters": (ctypes.c_int, [_vp, ctypes.POINTER(mdpf_counters)]),
        "mdpf_init_velocities": (ctypes.c_int, [_vp, _f64, ctypes.c_uint64]),
        "mdpf_get_trace": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _vp]),
        "mdpf_get_frames": (ctypes.c_int, [_vp, _i64, _vp, _vp, _vp, _vp, _vp]),
        "mdpf_get_trace_fallbacks": (ctypes.c_int, [_vp, _vp, _i64, _vp]),
        "mdpf_get_exclusions": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp]),
        "mdpf_get_angles": (ctypes.c_int, [_vp, _vp, _i64, _vp]),
        "mdpf_debug_set_status": (ctypes.c_int, [_vp, ctypes.c_uint32]),
        "mdpf_debug_wait_timeout": (ctypes.c_int, [_vp, _i32]),
        "mdpf_debug_tc_probe": (ctypes.c_int, [_vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp]),
        "mdpf_set_profiling": (ctypes.c_int, [_vp, _i32]),
        "mdpf_get_profile": (ctypes.c_int, [_vp, _i32, _vp, _vp]),
        "mdpf_learned_neighbors": (ctypes.c_int, [_vp, _vp, _i32, _vp, _vp]),
        "mdpf_learned_features": (ctypes.c_int, [_vp, _vp, _vp]),
        "mdpf_learned_mlp": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
        "mdpf_learned_counters": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
        "mdpf_learned_jvp": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
        "mdpf_trainer_create": (ctypes.c_int, [ctypes.POINTER(mdpf_train_params), ctypes.POINTER(_vp)]),
        "mdpf_trainer_destroy": (None, [_vp]),
        "mdpf_trainer_last_error": (ctypes.c_char_p, [_vp]),
        "mdpf_trainer_loss_grad": (ctypes.c_int, [_vp, _vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp]),
        "mdpf_trainer_status": (ctypes.c_int, [_vp, _vp]),
        "mdpf_trainer_feature_range": (ctypes.c_int, [_vp, _vp, _vp]),
        "mdpf_adamw_step": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _i64, _f64, _f64, _f64, _f64, _f64, _vp]),
        "mdpf_pairs_noalloc": (ctypes.c_int, [_i32, _vp, _vp, _vp, ctypes.POINTER(_f64), ctypes.POINTER(_f64), _f64,
                                              _vp, _vp, _vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


class Context:
    """One mdpf context (a system on the current CUDA device)."""

    def __init__(self, system, mode: int = MDPF_MODE_PLAIN, dt_fs: float = 0.5, coulomb_k: float = 0.0,
                 trace_capacity: int = 0, record_every: int = 0, max_frames: int = 0,
                 stepper: int = MDPF_STEPPER_PERSISTENT, energy_every: int = 1, model: bytes | None = None,
                 skin: float = 0.0, rebuild_every: int = 0, fallback: bool = True,
                 mlp_kernel: int = MDPF_MLP_TENSOR, provider=None, provider_kind: str = "energy_forces",
                 friction_per_ps: float = 0.0, temperature_K: float = 300.0, seed: int = 0):
        """mode MDPF_MODE_LEARNED needs ``model`` (a packed model blob, see model.Model.pack).

        mode MDPF_MODE_CALLBACK needs ``provider``, a Python callable the library calls for every
        force evaluation with the positions as a CUDA float64 tensor [N, 3] (A):
          provider_kind "energy_forces": provider(pos) -> (energy, forces[N, 3]) (kcal/mol, kcal/mol/A);
          provider_kind "energy":        provider(pos) -> energy (a differentiable torch scalar); the
                                         forces are -d energy / d pos by torch autograd.
        Its work runs on the library's stream (torch's current stream inside the call).
        """
        L = lib()
        s = system
        self.n = int(s.element.shape[0])
        self._keep = dict(
            element=np.ascontiguousarray(s.element, dtype=np.int32),
            mass=np.ascontiguousarray(s.mass, dtype=np.float64),
            charge=np.ascontiguousarray(s.charge, dtype=np.float64),
            bonds=np.ascontiguousarray(s.bonds, dtype=np.int32).reshape(-1, 2),
            r0=np.ascontiguousarray(s.bond_r0, dtype=np.float64),
            k=np.ascontiguousarray(s.bond_k, dtype=np.float64),
        )
        kp = self._keep
        t = mdpf_topology()
        t.n_atoms = self.n
        t.element = kp["element"].ctypes.data
        t.mass = kp["mass"].ctypes.data
        t.charge = kp["charge"].ctypes.data
        t.n_bonds = kp["bonds"].shape[0]
        t.bonds = kp["bonds"].ctypes.data if kp["bonds"].size else None
        t.bond_r0 = kp["r0"].ctypes.data if kp["r0"].size else None
        t.bond_k = kp["k"].ctypes.data if kp["k"].size else None
        t.angle_k = float(s.angle_k)
        t.angle_theta0_deg = float(s.angle_theta0_deg)
        for e in range(4):
            t.lj_sigma[e] = float(s.lj_sigma[e])
            t.lj_eps[e] = float(s.lj_eps[e])
        p = mdpf_params()
        p.mode = mode
        p.dt_fs = dt_fs
        p.coulomb_k = coulomb_k
        p.trace_capacity = trace_capacity
        p.record_every = record_every
        p.max_frames = max_frames
        p.stepper = stepper
        p.energy_every = energy_every
        if model is not None:
            self._model = ctypes.create_string_buffer(bytes(model), len(model))
            p.model = ctypes.addressof(self._model)
            p.model_bytes = len(model)
        p.skin = skin
        p.rebuild_every = rebuild_every
        p.fallback = 1 if fallback else 0
        p.mlp_kernel = mlp_kernel
        if friction_per_ps > 0.0:   # Langevin (BAOAB); zero friction keeps velocity Verlet
            p.integrator = MDPF_INTEGRATOR_LANGEVIN
            p.friction_per_ps = friction_per_ps
            p.temperature_K = temperature_K
            p.seed = seed
        if mode == MDPF_MODE_CALLBACK:
            self._setup_provider(p, provider, provider_kind)
        h = _vp()
        rc = L.mdpf_create(ctypes.byref(t), ctypes.byref(p), ctypes.byref(h))
        if rc != MDPF_OK:
            raise MdpfError(rc, L.mdpf_last_error(None).decode())
        self._h = h
        self.dt_fs = dt_fs
        self.record_every = record_every
        self.max_frames = max_frames

    # -- external force provider
    def _setup_provider(self, p, provider, kind):
        import torch
        if provider is None or kind not in ("energy", "energy_forces"):
            raise ValueError("callback mode needs provider= and provider_kind 'energy' or 'energy_forces'")
        dev = torch.device("cuda", torch.cuda.current_device())
        self._prov_pos = torch.zeros((self.n, 3), dtype=torch.float64, device=dev)
        self._prov_energy = torch.zeros(1, dtype=torch.float64, device=dev)
        self._prov_forces = torch.zeros((self.n, 3), dtype=torch.float32, device=dev)
        self._prov_error = None

        def call(user, stream):
            try:
                with torch.cuda.stream(torch.cuda.ExternalStream(stream)):
                    if kind == "energy":
                        with torch.enable_grad():
                            x = self._prov_pos.detach().clone().requires_grad_(True)
                            e = provider(x)
                            (g,) = torch.autograd.grad(e, x)
                        self._prov_forces.copy_(-g)
                    else:
                        e, f = provider(self._prov_pos)
                        self._prov_forces.copy_(f)
                    self._prov_energy.copy_(torch.as_tensor(e, dtype=torch.float64, device=dev).detach().reshape(1))
                return 0
            except Exception as exc:   # reported to the caller as MdpfError CALLBACK
                self._prov_error = exc
                return 1

        self._prov_fn = FORCE_FN(call)   # kept alive with the context
        p.provider = ctypes.cast(self._prov_fn, _vp)
        p.provider_user = None
        p.provider_pos = self._prov_pos.data_ptr()
        p.provider_energy = self._prov_energy.data_ptr()
        p.provider_forces = self._prov_forces.data_ptr()

    @property
    def provider_error(self):
        """The exception the provider raised in the last failed call, if any."""
        return getattr(self, "_prov_error", None)

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            lib().mdpf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc):
        if rc != MDPF_OK:
            err = MdpfError(rc, lib().mdpf_last_error(self._h).decode())
            cause = getattr(self, "_prov_error", None) if rc == -9 else None
            if cause is not None:
                self._prov_error = None
                raise err from cause
            raise err

    @property
    def handle(self):
        return self._h

    # -- the provider contract
    def compute(self, pos):
        """(E, F[N,3], terms) at host positions pos[N,3] (FP64)."""
        x = np.ascontiguousarray(pos, dtype=np.float64).reshape(self.n, 3)
        e = ctypes.c_double()
        f = np.zeros((self.n, 3))
        terms = np.zeros(4)
        self._check(lib().mdpf_compute(self._h, _ptr(x), ctypes.byref(e), _ptr(f), _ptr(terms)))
        return e.value, f, dict(zip(("bond", "angle", "lj", "coulomb"), terms.tolist()))

    def compute_device(self, d_pos: int, d_energy: int, d_forces: int, stream: int = 0):
        """Device-pointer form (addresses as ints, e.g. tensor.data_ptr())."""
        self._check(lib().mdpf_compute_device(self._h, _vp(d_pos), _vp(d_energy), _vp(d_forces), _vp(stream)))

    def set_state(self, pos, vel):
        x = np.ascontiguousarray(pos, dtype=np.float64).reshape(self.n, 3)
        v = np.ascontiguousarray(vel, dtype=np.float64).reshape(self.n, 3)
        self._check(lib().mdpf_set_state(self._h, _ptr(x), _ptr(v)))

    def init_velocities(self, temperature_K: float, seed: int):
        """Maxwell-Boltzmann velocities for the current positions, drawn on the device."""
        self._check(lib().mdpf_init_velocities(self._h, float(temperature_K), ctypes.c_uint64(int(seed))))

    def get_state(self, pos=None, vel=None):
        x = np.zeros((self.n, 3)) if pos is None else pos
        v = np.zeros((self.n, 3)) if vel is None else vel
        self._check(lib().mdpf_get_state(self._h, _ptr(x), _ptr(v)))
        return x, v

    def step(self, n_steps: int):
        self._check(lib().mdpf_step(self._h, int(n_steps)))

    def step_async(self, n_steps: int, stream: int = 0):
        self._check(lib().mdpf_step_async(self._h, int(n_steps), _vp(stream)))

    def counters(self) -> dict:
        c = mdpf_counters()
        self._check(lib().mdpf_get_counters(self._h, ctypes.byref(c)))
        return {k: getattr(c, k) for k, _ in mdpf_counters._fields_ if k != "reserved"}

    def trace(self, max_n: int = 1 << 20, with_steps: bool = False):
        cap = max_n
        U = np.zeros(cap)
        K = np.zeros(cap)
        st = np.zeros(cap, dtype=np.int64)
        n = ctypes.c_int64()
        self._check(lib().mdpf_get_trace(self._h, _ptr(U), _ptr(K), _ptr(st), cap, ctypes.byref(n)))
        if with_steps:
            return U[:n.value], K[:n.value], st[:n.value]
        return U[:n.value], K[:n.value]

    def trace_fallbacks(self, max_n: int = 1 << 20):
        """Cumulative fallback evaluations beside each energy-trace entry (learned mode)."""
        fb = np.zeros(max_n, dtype=np.int64)
        n = ctypes.c_int64()
        self._check(lib().mdpf_get_trace_fallbacks(self._h, _ptr(fb), max_n, ctypes.byref(n)))
        return fb[:n.value]

    def frames(self, max_n: int | None = None):
        m = self.max_frames if max_n is None else max_n
        pos = np.zeros((max(m, 1), self.n, 3))
        en = np.zeros(max(m, 1))
        frc = np.zeros((max(m, 1), self.n, 3), dtype=np.float32)
        st = np.zeros(max(m, 1), dtype=np.int64)
        n = ctypes.c_int64()
        self._check(lib().mdpf_get_frames(self._h, m, _ptr(pos), _ptr(en), _ptr(frc), _ptr(st), ctypes.byref(n)))
        k = n.value
        return pos[:k], en[:k], frc[:k], st[:k]

    def exclusions(self):
        tot = ctypes.c_int64()
        self._check(lib().mdpf_get_exclusions(self._h, None, None, 0, ctypes.byref(tot)))
        off = np.zeros(self.n + 1, dtype=np.int32)
        idx = np.zeros(max(tot.value, 1), dtype=np.int32)
        self._check(lib().mdpf_get_exclusions(self._h, _ptr(off), _ptr(idx), idx.size, ctypes.byref(tot)))
        return off, idx[:tot.value]

    def angles(self):
        na = ctypes.c_int64()
        self._check(lib().mdpf_get_angles(self._h, None, 0, ctypes.byref(na)))
        out = np.zeros((max(na.value, 1), 3), dtype=np.int32)
        self._check(lib().mdpf_get_angles(self._h, _ptr(out), out.shape[0], ctypes.byref(na)))
        return out[:na.value]

    # -- learned-path stages (parity checks)
    def learned_neighbors(self, pos, max_per_atom: int = 128):
        """(count[N], rows) with rows[i] the ascending neighbour indices of atom i."""
        x = np.ascontiguousarray(pos, dtype=np.float64).reshape(self.n, 3)
        cnt = np.zeros(self.n, dtype=np.int32)
        idx = np.zeros((self.n, max_per_atom), dtype=np.int32)
        self._check(lib().mdpf_learned_neighbors(self._h, _ptr(x), int(max_per_atom), _ptr(cnt), _ptr(idx)))
        return cnt, [idx[i, :cnt[i]].copy() for i in range(self.n)]

    def learned_features(self, pos):
        x = np.ascontiguousarray(pos, dtype=np.float64).reshape(self.n, 3)
        G = np.zeros((self.n, 384), dtype=np.float32)
        self._check(lib().mdpf_learned_features(self._h, _ptr(x), _ptr(G)))
        return G

    def learned_mlp(self, G):
        """(E_atom[N] FP64, dE/dG[N,384] FP32) from features G[N,384]."""
        g = np.ascontiguousarray(G, dtype=np.float32).reshape(self.n, 384)
        E = np.zeros(self.n)
        d = np.zeros((self.n, 384), dtype=np.float32)
        self._check(lib().mdpf_learned_mlp(self._h, _ptr(g), _ptr(E), _ptr(d)))
        return E, d

    def learned_jvp(self, pos, v):
        """U[N,384] = sum_a dG/dx_a . v_a (FP32) at host positions pos along host vectors v."""
        x = np.ascontiguousarray(pos, dtype=np.float64).reshape(self.n, 3)
        vv = np.ascontiguousarray(v, dtype=np.float32).reshape(self.n, 3)
        U = np.zeros((self.n, 384), dtype=np.float32)
        self._check(lib().mdpf_learned_jvp(self._h, _ptr(x), _ptr(vv), _ptr(U)))
        return U

    def learned_counters(self) -> dict:
        rb = ctypes.c_int64()
        fb = ctypes.c_int64()
        mr = ctypes.c_int32()
        self._check(lib().mdpf_learned_counters(self._h, ctypes.byref(rb), ctypes.byref(fb), ctypes.byref(mr)))
        return {"rebuilds": rb.value, "fallback_steps": fb.value, "max_row": mr.value}

    def debug_set_status(self, bits: int):
        self._check(lib().mdpf_debug_set_status(self._h, bits))

    def debug_wait_timeout(self, limit_us: int):
        return lib().mdpf_debug_wait_timeout(self._h, int(limit_us))

    def set_profiling(self, enable: bool):
        self._check(lib().mdpf_set_profiling(self._h, 1 if enable else 0))

    def profile(self, slot: int):
        """(total_ms, launches) of a profiled kernel slot since profiling was enabled."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(lib().mdpf_get_profile(self._h, slot, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value


def pairs_noalloc(n_atoms: int, d_pos: int, d_element: int, d_charge: int, lj_sigma, lj_eps, coulomb_k: float,
                  d_energy: int, d_forces: int, stream: int = 0) -> None:
    """All-pairs LJ + Coulomb through the entry point that allocates no device memory
    (device addresses as ints; see mdpf_pairs_noalloc in include/mdpf.h)."""
    if len(lj_sigma) != 4 or len(lj_eps) != 4:
        raise ValueError("lj_sigma and lj_eps need one value per element (4 each)")
    sig = (_f64 * 4)(*[float(v) for v in lj_sigma])
    eps = (_f64 * 4)(*[float(v) for v in lj_eps])
    rc = lib().mdpf_pairs_noalloc(int(n_atoms), _vp(d_pos), _vp(d_element), _vp(d_charge), sig, eps,
                                  float(coulomb_k), _vp(d_energy), _vp(d_forces), _vp(stream))
    if rc != MDPF_OK:
        raise MdpfError(rc, lib().mdpf_last_error(None).decode())


def debug_tc_probe(d_a: int, d_b: int, d_d: int, n: int, a_off: int, b_off: int, d_status: int,
                   stream: int = 0) -> None:
    """D = A B^T through the MLP kernels' tensor-core operand path with the operands at chosen
    shared-memory offsets (device addresses as ints; see mdpf_debug_tc_probe in include/mdpf.h)."""
    rc = lib().mdpf_debug_tc_probe(_vp(d_a), _vp(d_b), _vp(d_d), int(n), int(a_off), int(b_off), _vp(d_status),
                                   _vp(stream))
    if rc != MDPF_OK:
        raise MdpfError(rc, lib().mdpf_last_error(None).decode())


class Trainer:
    """Device-side force-matching loss and gradient (mdpf_trainer_*); all tensors
    are caller-owned device memory passed by address (e.g. torch data_ptr())."""

    def __init__(self, max_frames: int, atoms_per_frame: int, e0, w_force: float = 10.0, core_a: float = 0.0,
                 core_rc: float = 0.0):
        """core_a, core_rc: the model's repulsive core (core_rc 0: none), part of the predicted E and F."""
        p = mdpf_train_params()
        p.max_frames = int(max_frames)
        p.atoms_per_frame = int(atoms_per_frame)
        p.w_force = float(w_force)
        for e in range(4):
            p.e0[e] = float(e0[e])
        p.core_a = float(core_a)
        p.core_rc = float(core_rc)
        h = _vp()
        rc = lib().mdpf_trainer_create(ctypes.byref(p), ctypes.byref(h))
        if rc != MDPF_OK:
            raise MdpfError(rc, lib().mdpf_trainer_last_error(None).decode())
        self._h = h
        self.max_frames = max_frames
        self.atoms_per_frame = atoms_per_frame

    def _check(self, rc):
        if rc != MDPF_OK:
            raise MdpfError(rc, lib().mdpf_trainer_last_error(self._h).decode())

    def loss_grad(self, d_params: int, d_grad: int, n_frames: int, d_pos: int, d_element: int, d_E_ref: int,
                  d_F_ref: int, d_loss3: int, stream: int = 0):
        self._check(lib().mdpf_trainer_loss_grad(self._h, _vp(d_params), _vp(d_grad), int(n_frames), _vp(d_pos),
                                                 _vp(d_element), _vp(d_E_ref), _vp(d_F_ref), _vp(d_loss3),
                                                 _vp(stream)))

    def status(self) -> int:
        st = ctypes.c_uint32()
        self._check(lib().mdpf_trainer_status(self._h, ctypes.byref(st)))
        return st.value

    def feature_range(self):
        lo = np.zeros((4, 384), dtype=np.float32)
        hi = np.zeros((4, 384), dtype=np.float32)
        self._check(lib().mdpf_trainer_feature_range(self._h, _ptr(lo), _ptr(hi)))
        return lo, hi

    def close(self):
        if getattr(self, "_h", None):
            lib().mdpf_trainer_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def adamw_step(d_params: int, d_grad: int, d_m: int, d_v: int, n: int, step: int, lr: float, beta1: float = 0.9,
               beta2: float = 0.999, eps: float = 1e-8, weight_decay: float = 0.01, stream: int = 0) -> None:
    rc = lib().mdpf_adamw_step(_vp(d_params), _vp(d_grad), _vp(d_m), _vp(d_v), int(n), int(step), float(lr),
                               float(beta1), float(beta2), float(eps), float(weight_decay), _vp(stream))
    if rc != MDPF_OK:
        raise MdpfError(rc, "mdpf_adamw_step failed")
