"""GPU parity of the learned path (cell-list neighbours, symmetry-function
features, per-element BF16 MLP, analytic force adjoint, range check with the
plain fallback, velocity Verlet) against the FP64 oracle, through the C ABI.

Tolerances:
  neighbour rows   identical (FP32 predicate evaluated the same way on both sides)
  features (FP32)  RMSE <= 1e-4 * RMS(G_oracle) per system; exact zeros stay zero
  MLP / forces     BF16 GEMM operands: force RMSE <= 1e-2 * RMS(F_oracle),
                   |E - E_oracle| / N <= 1e-3 kcal/mol/atom, against the oracle's
                   FP64 evaluation of the same (BF16-valued) weights
  MLP vs emulation a numpy model of the kernel's rounding points (BF16 inputs to
                   every GEMM, FP64 products, dE/dG rounded to BF16) agrees to FP32
                   accumulation error (plus the odd BF16 rounding flip of dE/dG)
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_18271_b300 import mdpf, model, synth
from tests import tiny

pytestmark = pytest.mark.gpu

G_RTOL = 1e-4
F_RTOL_BF16 = 1e-2
E_TOL_BF16 = 1e-3
LEARNED = mdpf.MDPF_MODE_LEARNED


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_18271_b300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()
    torch.cuda.init()


@pytest.fixture(scope="module")
def mdl():
    m = model.init_model(7)
    m.e0 = np.array([-0.5, -38.0, -54.6, -75.1])
    m.b3 = np.array([0.01, -0.02, 0.03, 0.0], dtype=np.float32)
    return m.rounded()


def _ctx(s, m, **kw):
    return mdpf.Context(s, mode=LEARNED, model=m.pack(), **kw)


def _rows_equal(rows, orows):
    assert len(rows) == len(orows)
    for i, (a, b) in enumerate(zip(rows, orows)):
        assert np.array_equal(a, b), (i, a, b)


# ------------------------------------------------------------ neighbours

@pytest.mark.parametrize("name", ["mol64", "mol256", "cluster2048"])
def test_neighbors_bit_exact(name, mdl):
    s = synth.workload(name)
    ctx = _ctx(s, mdl)
    cnt, rows = ctx.learned_neighbors(s.pos)
    _rows_equal(rows, O.neighbors(np.float32(s.pos), O.RC_LIST))
    assert ctx.learned_counters()["max_row"] == int(cnt.max())


def test_neighbors_with_far_outliers(mdl):
    # a cluster with a few atoms 1000 A away (a gas-phase cluster evaporates): the cell grid must not grow
    # with the bounding box until its cells overflow; rows (incl. the pairs among the far atoms) stay exact
    s = synth.workload("cluster2048")
    pos = np.array(s.pos, dtype=np.float64)
    far = {3: (1000.0, 0.0, 0.0), 700: (-1000.0, 0.0, 0.0), 1400: (0.0, 1000.0, 0.0), 1900: (0.0, -1000.0, 0.0),
           40: (0.0, 0.0, 1000.0), 1041: (0.0, 0.0, -1000.0), 77: (1000.0, 3.0, 0.0), 1777: (1000.0, 0.0, 4.0)}
    for a, p in far.items():
        pos[a] = p
    ctx = _ctx(s, mdl)
    cnt, rows = ctx.learned_neighbors(pos)
    orows = O.neighbors(np.float32(pos), O.RC_LIST)
    _rows_equal(rows, orows)
    assert sorted(rows[3]) == [77, 1777]
    assert ctx.counters()["status"] == 0


def test_neighbors_skin_sets_the_radius(mdl):
    s = synth.workload("mol256")
    ctx = _ctx(s, mdl, skin=0.25)
    _, rows = ctx.learned_neighbors(s.pos)
    _rows_equal(rows, O.neighbors(np.float32(s.pos), 5.2 + 0.25))


def test_neighbors_at_the_cutoff_boundary(mdl):
    # isolated pairs whose separations step through the list radius one FP32 ulp at a time
    k = np.arange(-40, 41)
    r = np.float32(6.2) + k.astype(np.float32) * np.spacing(np.float32(6.2))
    n = 2 * k.size
    pos = np.zeros((n, 3))
    pos[0::2, 0] = np.arange(k.size) * 50.0
    pos[1::2, 0] = pos[0::2, 0] + r.astype(np.float64)
    pos[1::2, 1] = 0.0
    s = tiny.isolated(n)
    ctx = _ctx(s, mdl)
    _, rows = ctx.learned_neighbors(pos)
    orows = O.neighbors(np.float32(pos), O.RC_LIST)
    _rows_equal(rows, orows)
    n_in = sum(len(rw) for rw in orows) // 2
    assert 0 < n_in < k.size


def test_neighbors_single_atom_and_empty_rows(mdl):
    s = tiny.isolated(1)
    ctx = _ctx(s, mdl)
    cnt, rows = ctx.learned_neighbors(np.zeros((1, 3)))
    assert cnt.tolist() == [0]
    s = tiny.isolated(3)
    ctx = _ctx(s, mdl)
    cnt, rows = ctx.learned_neighbors(np.array([[0.0, 0, 0], [30.0, 0, 0], [60.0, 0, 0]]))
    assert cnt.tolist() == [0, 0, 0]


def test_neighbor_overflow_is_reported(mdl):
    g = np.arange(6, dtype=np.float64) * 1.0
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    s = tiny.isolated(pos.shape[0])
    ctx = _ctx(s, mdl)
    with pytest.raises(mdpf.MdpfError) as ei:
        ctx.learned_neighbors(pos)
    assert ei.value.name == "NEIGHBOR_OVERFLOW"
    with pytest.raises(mdpf.MdpfError) as ei:
        ctx.compute(pos)
    assert ei.value.name == "NEIGHBOR_OVERFLOW"


# ------------------------------------------------------------ features

@pytest.mark.parametrize("name", ["mol64", "mol256", "cluster2048"])
def test_features_match_oracle(name, mdl):
    s = synth.workload(name)
    ctx = _ctx(s, mdl)
    G = ctx.learned_features(s.pos).astype(np.float64)
    Go = O.features(s.element, s.pos)
    rmse = np.sqrt(((G - Go) ** 2).mean())
    rms = np.sqrt((Go ** 2).mean())
    assert rmse <= G_RTOL * rms, (rmse, rms)
    # radial and angular blocks separately (angular values are orders of magnitude smaller)
    for sl in (slice(0, 64), slice(64, 384)):
        d = G[:, sl] - Go[:, sl]
        assert np.sqrt((d ** 2).mean()) <= G_RTOL * np.sqrt((Go[:, sl] ** 2).mean()), sl
    assert np.all(G[Go == 0.0] == 0.0)


def test_features_of_isolated_atoms_are_zero(mdl):
    s = tiny.isolated(2)
    ctx = _ctx(s, mdl)
    G = ctx.learned_features(np.array([[0.0, 0, 0], [7.0, 0, 0]]))
    assert np.all(G == 0.0)


# ------------------------------------------------------------ MLP

def _bf(x):
    return model.bf16_to_f32(model.bf16_bits(np.asarray(x, dtype=np.float32))).astype(np.float64)


def _mlp_emulated(m, element, G):
    """The kernel's rounding points: BF16 GEMM inputs (features, deltas; layer 1's
    CELU output as the pair hi + lo of BF16 values), everything else FP64."""
    def celu(x):
        return np.where(x > 0, x, 0.1 * np.expm1(x / 0.1))

    def dcelu(x):
        return np.where(x >= 0, 1.0, np.exp(x / 0.1))

    n = G.shape[0]
    E = np.zeros(n)
    g = np.zeros((n, 384))
    for e in range(4):
        idx = np.nonzero(element == e)[0]
        if idx.size == 0:
            continue
        W1, W2 = m.W1[e].astype(np.float64), m.W2[e].astype(np.float64)
        h1 = _bf(G[idx]) @ W1.T + m.b1[e]
        a1f = celu(h1).astype(np.float32).astype(np.float64)
        a1 = _bf(a1f) + _bf(a1f - _bf(a1f))
        h2 = a1 @ W2.T + m.b2[e]
        E[idx] = celu(h2) @ m.W3[e].astype(np.float64) + float(m.b3[e]) + m.e0[e]
        d2 = _bf(m.W3[e] * dcelu(h2))
        d1 = _bf((d2 @ W2) * dcelu(h1))
        g[idx] = _bf(d1 @ W1)   # dE/dG is stored in BF16 for the adjoint
    return E, g


MLP_KERNELS = [mdpf.MDPF_MLP_TENSOR, mdpf.MDPF_MLP_SIMT]


@pytest.mark.parametrize("kernel", MLP_KERNELS)
@pytest.mark.parametrize("name", ["mol64", "mol256"])
def test_mlp_matches_oracle_and_emulation(name, kernel, mdl):
    s = synth.workload(name)
    ctx = _ctx(s, mdl, mlp_kernel=kernel)
    Go = O.features(s.element, s.pos)
    G32 = Go.astype(np.float32)
    E, dG = ctx.learned_mlp(G32)
    _, Eo, dGo = O.Learned(mdl).mlp(s.element, Go)
    n = s.n_atoms
    assert abs(E.sum() - Eo.sum()) / n <= E_TOL_BF16
    assert np.sqrt(((dG - dGo) ** 2).mean()) <= F_RTOL_BF16 * np.sqrt((dGo ** 2).mean())
    # the kernel's own rounding points, reproduced in numpy: FP32 accumulation error only
    Ee, ge = _mlp_emulated(mdl, s.element, G32.astype(np.float64))
    assert np.max(np.abs(E - Ee)) <= 1e-4 * max(1.0, np.max(np.abs(Ee)))
    assert np.sqrt(((dG - ge) ** 2).mean()) <= 1e-3 * np.sqrt((ge ** 2).mean())


@pytest.mark.parametrize("kernel", MLP_KERNELS)
def test_mlp_rows_of_every_element_and_padding(kernel, mdl):
    # 1..3 atoms per element exercise the per-element row padding
    el = np.array([0, 1, 1, 2, 3, 3, 3, 0], dtype=np.int32)
    s = tiny.isolated(el.size, element=el)
    ctx = _ctx(s, mdl, mlp_kernel=kernel)
    rng = np.random.default_rng(5)
    G = rng.uniform(0.0, 2.0, size=(el.size, 384)).astype(np.float32)
    E, dG = ctx.learned_mlp(G)
    Ee, ge = _mlp_emulated(mdl, el, G.astype(np.float64))
    assert np.max(np.abs(E - Ee)) <= 1e-4 * max(1.0, np.max(np.abs(Ee)))
    assert np.sqrt(((dG - ge) ** 2).mean()) <= 1e-3 * np.sqrt((ge ** 2).mean())


def test_tensor_and_simt_mlp_agree_over_many_tiles(mdl):
    # 2048 atoms -> 17 row tiles of 128 over four elements; random features in the
    # range the workloads produce, so every GEMM sees dense nonzero operands
    s = synth.workload("cluster2048")
    rng = np.random.default_rng(9)
    G = (rng.gamma(0.5, 1.0, size=(s.n_atoms, 384)) * (rng.random((s.n_atoms, 384)) < 0.6)).astype(np.float32)
    out = []
    for kernel in MLP_KERNELS:
        ctx = _ctx(s, mdl, mlp_kernel=kernel)
        out.append(ctx.learned_mlp(G))
    (Et, gt), (Es, gs) = out
    Ee, ge = _mlp_emulated(mdl, s.element, G.astype(np.float64))
    assert np.max(np.abs(Et - Ee)) <= 1e-4 * max(1.0, np.max(np.abs(Ee)))
    assert np.max(np.abs(Et - Es)) <= 1e-4 * max(1.0, np.max(np.abs(Ee)))
    assert np.sqrt(((gt - gs) ** 2).mean()) <= 1e-3 * np.sqrt((gs ** 2).mean())
    assert np.sqrt(((gt - ge) ** 2).mean()) <= 1e-3 * np.sqrt((ge ** 2).mean())


@pytest.mark.parametrize("kernel", MLP_KERNELS)
def test_mlp_kernels_are_deterministic(kernel, mdl):
    s = synth.workload("mol256")
    ctx = _ctx(s, mdl, mlp_kernel=kernel)
    G = O.features(s.element, s.pos).astype(np.float32)
    E1, g1 = ctx.learned_mlp(G)
    E2, g2 = ctx.learned_mlp(G)
    assert np.array_equal(E1, E2) and np.array_equal(g1, g2)


# ------------------------------------------------------------ energy and forces

@pytest.mark.parametrize("kernel", MLP_KERNELS)
@pytest.mark.parametrize("name", ["mol64", "mol256", "cluster2048"])
def test_energy_forces_match_oracle(name, kernel, mdl):
    s = synth.workload(name)
    ctx = _ctx(s, mdl, mlp_kernel=kernel)
    e, f, terms = ctx.compute(s.pos)
    eo, fo, _ = O.Learned(mdl).energy_forces(s.element, s.pos)
    n = s.n_atoms
    assert abs(e - eo) / n <= E_TOL_BF16, (e, eo)
    rmse = np.sqrt(((f - fo) ** 2).mean())
    rms = np.sqrt((fo ** 2).mean())
    assert rmse <= F_RTOL_BF16 * rms, (rmse, rms)
    assert all(v == 0.0 for v in terms.values())
    # net force of an isolated system vanishes up to the fixed-point and FP32 rounding
    assert np.abs(f.sum(0)).max() <= 1e-3 * rms * np.sqrt(n)


def test_energy_forces_tiny_systems(mdl):
    for n in (1, 2, 3):
        s = tiny.isolated(n)
        pos = np.array([[0.0, 0, 0], [1.1, 0, 0], [1.5, 1.2, 0.3]])[:n]
        ctx = _ctx(s, mdl)
        e, f, _ = ctx.compute(pos)
        eo, fo, _ = O.Learned(mdl).energy_forces(s.element, pos)
        assert abs(e - eo) / n <= E_TOL_BF16
        rms = np.sqrt((fo ** 2).mean()) if n > 1 else 0.0
        assert np.sqrt(((f - fo) ** 2).mean()) <= F_RTOL_BF16 * rms + 1e-6


def _core_geometry(s, seps=(0.45, 0.6, 0.75)):
    """The molecule with a few bonded pairs pulled inside the core radius (one
    atom of each moved along its bond to the given separations)."""
    pos = s.pos.copy()
    for (a, b), r in zip(s.bonds[[3, 11, 20]], seps):
        d = pos[b] - pos[a]
        pos[b] = pos[a] + d / np.linalg.norm(d) * r
    return pos


@pytest.mark.parametrize("kernel", MLP_KERNELS + [mdpf.MDPF_MLP_SIMT_FP32, mdpf.MDPF_MLP_FUSED])
def test_core_pairs_match_oracle(kernel, mdl):
    s = synth.workload("mol64")
    pos = _core_geometry(s)
    ec, fc = O.core_energy_forces(pos, mdl.core_a, mdl.core_rc)
    assert ec > 30.0                      # the core carries real energy here
    ctx = _ctx(s, mdl, mlp_kernel=kernel)
    e, f, _ = ctx.compute(pos)
    eo, fo, _ = O.Learned(mdl).energy_forces(s.element, pos)
    assert abs(e - eo) / s.n_atoms <= E_TOL_BF16, (e, eo)
    assert np.sqrt(((f - fo) ** 2).mean()) <= F_RTOL_BF16 * np.sqrt((fo ** 2).mean())
    # the core part alone: the same model without its core, on the same kernels, differs by the
    # oracle's core energy and forces (FP32 pair arithmetic: relative 1e-5)
    off = model.Model(mdl.W1, mdl.b1, mdl.W2, mdl.b2, mdl.W3, mdl.b3, mdl.e0)
    e_off, f_off, _ = _ctx(s, off, mlp_kernel=kernel).compute(pos)
    assert abs((e - e_off) - ec) <= 1e-5 * ec
    assert np.abs((f - f_off) - fc).max() <= 1e-5 * np.abs(fc).max() + 1e-3


def test_learned_compute_is_deterministic(mdl):
    s = synth.workload("mol256")
    ctx = _ctx(s, mdl)
    e1, f1, _ = ctx.compute(s.pos)
    e2, f2, _ = ctx.compute(s.pos)
    assert e1 == e2 and np.array_equal(f1, f2)


# ------------------------------------------------------------ range check and fallback

def _ranged(m, s, widen=0.02):
    G = O.features(s.element, s.pos)
    lo = np.zeros((4, 384), dtype=np.float32)
    hi = np.zeros((4, 384), dtype=np.float32)
    for e in range(4):
        sel = G[s.element == e]
        if sel.size == 0:
            continue
        a, b = sel.min(0), sel.max(0)
        span = b - a
        lo[e] = a - widen * span - 1e-6
        hi[e] = b + widen * span + 1e-6
    r = model.Model(m.W1, m.b1, m.W2, m.b2, m.W3, m.b3, m.e0, lo, hi, m.alpha, m.core_a, m.core_rc)
    return r


def _expanded(s, factor=1.02):
    """The molecule stretched 2% about its centroid; some features then leave the
    range of the unstretched geometry (checked on the oracle's features)."""
    c = s.pos.mean(0)
    pos = c + (s.pos - c) * factor
    mr = _ranged(model.init_model(0), s)
    G = O.features(s.element, pos)
    assert np.any((G < mr.lo[s.element]) | (G > mr.hi[s.element]))
    return pos


def test_in_range_uses_the_model(mdl):
    s = synth.workload("mol256")
    mr = _ranged(mdl, s)
    ctx = _ctx(s, mr)
    e, f, terms = ctx.compute(s.pos)
    eo, _, _ = O.Learned(mdl).energy_forces(s.element, s.pos)
    assert abs(e - eo) / s.n_atoms <= E_TOL_BF16
    assert ctx.learned_counters()["fallback_steps"] == 0


def test_out_of_range_falls_back_to_the_plain_force_field(mdl):
    s = synth.workload("mol256")
    mr = _ranged(mdl, s)
    pos = _expanded(s)
    ctx = _ctx(s, mr)
    e, f, terms = ctx.compute(pos)
    ep, fp, tp = O.Plain(s).energy_forces(pos)
    assert abs(e - ep) / s.n_atoms <= 1e-5
    assert np.sqrt(((f - fp) ** 2).mean()) <= 1e-4 * np.sqrt((fp ** 2).mean())
    for k in ("bond", "angle", "lj", "coulomb"):
        assert abs(terms[k] - tp[k]) / s.n_atoms <= 1e-5
    assert ctx.learned_counters()["fallback_steps"] == 1
    # back in range: the model again
    e2, _, _ = ctx.compute(s.pos)
    eo, _, _ = O.Learned(mdl).energy_forces(s.element, s.pos)
    assert abs(e2 - eo) / s.n_atoms <= E_TOL_BF16
    assert ctx.learned_counters()["fallback_steps"] == 1


def test_out_of_range_without_fallback_is_an_error(mdl):
    s = synth.workload("mol256")
    mr = _ranged(mdl, s)
    pos = _expanded(s)
    ctx = _ctx(s, mr, fallback=False)
    with pytest.raises(mdpf.MdpfError) as ei:
        ctx.compute(pos)
    assert ei.value.name == "OUT_OF_RANGE"
    ctx2 = _ctx(s, mr, fallback=False)
    e, _, _ = ctx2.compute(s.pos)
    assert np.isfinite(e)


# ------------------------------------------------------------ learned MD

def _vv_oracle(mdl, s, pos, vel, dt, n_steps):
    """Velocity Verlet with the oracle's learned forces (FP64)."""
    acc = O.ACC / s.mass[:, None]
    x, v = pos.copy(), vel.copy()
    _, f, _ = O.Learned(mdl).energy_forces(s.element, x)
    for _ in range(n_steps):
        v = v + 0.5 * dt * acc * f
        x = x + dt * v
        _, f, _ = O.Learned(mdl).energy_forces(s.element, x)
        v = v + 0.5 * dt * acc * f
    return x, v


def test_learned_md_follows_the_oracle(mdl):
    s = synth.workload("mol64")
    vel = synth.velocities(s.mass, s.pos, 300.0, 11)
    ctx = _ctx(s, mdl, dt_fs=0.5)
    ctx.set_state(s.pos, vel)
    ctx.step(10)
    x, v = ctx.get_state()
    xo, vo = _vv_oracle(mdl, s, s.pos, vel, 0.5, 10)
    # BF16 force error (~4e-3 of RMS) over 10 steps of 0.5 fs moves atoms by ~1e-5 A
    assert np.abs(x - xo).max() <= 1e-4
    assert np.abs(v - vo).max() <= 1e-4


def test_rebuild_schedule_does_not_change_the_trajectory(mdl):
    s = synth.workload("mol256")
    vel = synth.velocities(s.mass, s.pos, 300.0, 12)
    out, rebuilds = [], []
    for every in (1, 7, 1000):
        ctx = _ctx(s, mdl, rebuild_every=every)
        ctx.set_state(s.pos, vel)
        ctx.step(60)
        out.append(ctx.get_state())
        rebuilds.append(ctx.learned_counters()["rebuilds"])
    # set_state builds once; every=1 rebuilds each step; every=1000 only on step 0 and on displacement
    assert rebuilds[0] == 61
    assert rebuilds[0] > rebuilds[1] >= rebuilds[2] >= 2
    for x, v in out[1:]:
        assert np.array_equal(x, out[0][0]) and np.array_equal(v, out[0][1])


def test_learned_split_steps_equal_one_run(mdl):
    s = synth.workload("mol256")
    vel = synth.velocities(s.mass, s.pos, 300.0, 13)
    a = _ctx(s, mdl)
    a.set_state(s.pos, vel)
    a.step(40)
    b = _ctx(s, mdl)
    b.set_state(s.pos, vel)
    b.step(15)
    b.step(25)
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    ua, ka = a.trace()
    ub, kb = b.trace()
    assert np.array_equal(ua, ub) and np.array_equal(ka, kb)


def test_graph_stepping_equals_direct_launches(mdl):
    # with profiling on, every step is launched kernel by kernel; off, each step is one graph launch
    s = synth.workload("mol256")
    vel = synth.velocities(s.mass, s.pos, 300.0, 14)
    out = []
    for prof in (False, True):
        ctx = _ctx(s, mdl, energy_every=5, trace_capacity=64)
        ctx.set_state(s.pos, vel)
        ctx.set_profiling(prof)
        ctx.step(23)
        ctx.step(17)
        out.append((ctx.get_state(), ctx.trace(), ctx.learned_counters()))
    (xa, va), (ua, ka), ca = out[0]
    (xb, vb), (ub, kb), cb = out[1]
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert np.array_equal(ua, ub) and np.array_equal(ka, kb)
    assert ca == cb


def test_fallback_every_step_reproduces_the_plain_trajectory(mdl):
    # ranges that every feature violates: each learned step is a plain force-field step
    s = synth.workload("mol256")
    r = model.Model(mdl.W1, mdl.b1, mdl.W2, mdl.b2, mdl.W3, mdl.b3, mdl.e0,
                    np.full((4, 384), -2.0, np.float32), np.full((4, 384), -1.0, np.float32))
    vel = synth.velocities(s.mass, s.pos, 300.0, 15)
    a = _ctx(s, r, energy_every=1)
    a.set_state(s.pos, vel)
    a.step(40)
    b = mdpf.Context(s, stepper=mdpf.MDPF_STEPPER_KERNELS, energy_every=1)
    b.set_state(s.pos, vel)
    b.step(40)
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert a.learned_counters()["fallback_steps"] == 41
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    ua, ka = a.trace()
    ub, kb = b.trace()
    assert np.allclose(ua, ub, rtol=1e-12, atol=1e-9) and np.array_equal(ka, kb)


def test_fp32_mlp_kernel_matches_the_oracle_tightly(mdl):
    # FP32 operands throughout: FP32 rounding only, against the FP64 oracle
    s = synth.workload("mol256")
    ctx = _ctx(s, mdl, mlp_kernel=mdpf.MDPF_MLP_SIMT_FP32)
    Go = O.features(s.element, s.pos)
    E, dG = ctx.learned_mlp(Go.astype(np.float32))
    _, Eo, dGo = O.Learned(mdl).mlp(s.element, Go)
    assert np.max(np.abs(E - Eo)) <= 1e-5 * max(1.0, np.max(np.abs(Eo)))
    assert np.sqrt(((dG - dGo) ** 2).mean()) <= 1e-4 * np.sqrt((dGo ** 2).mean())
    e, f, _ = ctx.compute(s.pos)
    eo, fo, _ = O.Learned(mdl).energy_forces(s.element, s.pos)
    assert abs(e - eo) / s.n_atoms <= 1e-5
    assert np.sqrt(((f - fo) ** 2).mean()) <= 1e-4 * np.sqrt((fo ** 2).mean())
