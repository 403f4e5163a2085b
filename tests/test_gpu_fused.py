"""GPU parity of the fused learned force kernel (features -> tensor-core MLP ->
adjoint in one CTA per tile, MDPF_MLP_FUSED).

It runs the per-stage kernels' own per-atom arithmetic, with the features and
dE/dG kept on chip, so against the stage-by-stage path (MDPF_MLP_TENSOR) the
bar is identity: the same energy and the same forces, bit for bit, and the
same MD trajectory.  Against the FP64 oracle the BF16 tolerances of the
learned path apply (force RMSE <= 1e-2 of RMS, |dE|/N <= 1e-3 kcal/mol/atom).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_18271_b300 import mdpf, model, synth
from tests import tiny
from tests.test_gpu_learned import _expanded, _ranged

pytestmark = pytest.mark.gpu

LEARNED = mdpf.MDPF_MODE_LEARNED
FUSED, STAGED = mdpf.MDPF_MLP_FUSED, mdpf.MDPF_MLP_TENSOR


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
    m.b1 = np.random.default_rng(1).normal(0, 0.2, m.b1.shape).astype(np.float32)
    return m.rounded()


def _ctx(s, m, kernel, **kw):
    return mdpf.Context(s, mode=LEARNED, model=m.pack(), mlp_kernel=kernel, **kw)


def _both(s, m, pos=None, **kw):
    pos = s.pos if pos is None else pos
    out = []
    for kernel in (FUSED, STAGED):
        ctx = _ctx(s, m, kernel, **kw)
        out.append(ctx.compute(pos))
        ctx.close()
    return out


def _replicas(s, n_side, spacing):
    """n_side^3 translated copies of s on a cubic grid (no interactions between copies
    when the spacing exceeds the molecule's extent plus the cutoff)."""
    k = n_side ** 3
    shifts = np.array([(a, b, c) for a in range(n_side) for b in range(n_side) for c in range(n_side)],
                      dtype=np.float64) * spacing
    n = s.n_atoms
    return synth.System(
        element=np.tile(s.element, k), mass=np.tile(s.mass, k), charge=np.tile(s.charge, k),
        bonds=np.concatenate([s.bonds + q * n for q in range(k)]).astype(np.int32),
        bond_r0=np.tile(s.bond_r0, k), bond_k=np.tile(s.bond_k, k), angle_k=s.angle_k,
        angle_theta0_deg=s.angle_theta0_deg, lj_sigma=s.lj_sigma, lj_eps=s.lj_eps,
        pos=np.concatenate([s.pos + d for d in shifts]), molecule=np.repeat(np.arange(k, dtype=np.int32), n))


@pytest.mark.parametrize("name", ["mol64", "mol256", "cluster2048"])
def test_fused_equals_stagewise(name, mdl):
    s = synth.workload(name)
    (ef, ff, tf), (es, fs, ts) = _both(s, mdl)
    assert ef == es
    assert np.array_equal(ff, fs)
    assert tf == ts


@pytest.mark.parametrize("name", ["mol64", "mol256"])
def test_fused_matches_oracle(name, mdl):
    s = synth.workload(name)
    ctx = _ctx(s, mdl, FUSED)
    e, f, terms = ctx.compute(s.pos)
    eo, fo, _ = O.Learned(mdl).energy_forces(s.element, s.pos)
    n = s.n_atoms
    assert abs(e - eo) / n <= 1e-3, (e, eo)
    assert np.sqrt(((f - fo) ** 2).mean()) <= 1e-2 * np.sqrt((fo ** 2).mean())
    assert all(v == 0.0 for v in terms.values())


def test_fused_tiny_systems_and_absent_elements(mdl):
    # single atoms, pairs, a triplet; one or two elements only; every tile of one atom
    cases = [
        (np.array([0]), np.zeros((1, 3))),
        (np.array([3, 3]), np.array([[0.0, 0, 0], [1.2, 0, 0]])),
        (np.array([1, 0, 2]), np.array([[0.0, 0, 0], [1.1, 0, 0], [-0.4, 1.3, 0.2]])),
    ]
    for el, pos in cases:
        s = tiny.isolated(el.size, element=el)
        (ef, ff, _), (es, fs, _) = _both(s, mdl, pos=pos)
        assert ef == es and np.array_equal(ff, fs), el
        eo, fo, _ = O.Learned(mdl).energy_forces(el, pos)
        assert abs(ef - eo) <= 1e-3 * max(1, el.size)
        assert np.abs(ff - fo).max() <= 1e-2 * max(1.0, np.abs(fo).max())


def test_fused_nine_atom_molecule(mdl):
    s = synth.molecule(9, seed=3)
    (ef, ff, _), (es, fs, _) = _both(s, mdl)
    assert ef == es and np.array_equal(ff, fs)


def test_fused_tiles_in_more_than_one_wave(mdl):
    # 125 copies of the 256-atom molecule, 30 A apart (32,000 atoms): more tiles of
    # 128 atoms than SMs, so the tiles are full 128-atom runs over two waves
    one = synth.workload("mol256")
    s = _replicas(one, 5, 30.0)
    (ef, ff, _), (es, fs, _) = _both(s, mdl)
    assert ef == es and np.array_equal(ff, fs)
    # the copies do not interact: each carries the single molecule's forces, up to the
    # FP32 rounding of the shifted coordinates
    _, f1, _ = _ctx(one, mdl, FUSED).compute(one.pos)
    n = one.n_atoms
    rms = np.sqrt((f1 ** 2).mean())
    for q in range(0, 125, 31):
        assert np.sqrt(((ff[q * n:(q + 1) * n] - f1) ** 2).mean()) <= 1e-3 * rms


def test_fused_is_deterministic(mdl):
    s = synth.workload("cluster2048")
    ctx = _ctx(s, mdl, FUSED)
    e1, f1, _ = ctx.compute(s.pos)
    e2, f2, _ = ctx.compute(s.pos)
    assert e1 == e2 and np.array_equal(f1, f2)


def test_fused_md_equals_stagewise(mdl):
    s = synth.workload("mol256")
    vel = synth.velocities(s.mass, s.pos, 300.0, 21)
    out = []
    for kernel, prof in ((FUSED, False), (FUSED, True), (STAGED, False)):
        ctx = _ctx(s, mdl, kernel, energy_every=5, trace_capacity=64)
        ctx.set_state(s.pos, vel)
        ctx.set_profiling(prof)
        ctx.step(30)
        out.append((ctx.get_state(), ctx.trace()))
        if prof:
            ms, n = ctx.profile(mdpf.MDPF_PROF_LEARN_FUSED)
            assert n == 30 and ms > 0.0
        ctx.close()
    (x0, v0), (u0, k0) = out[0]
    for (x, v), (u, k) in out[1:]:
        assert np.array_equal(x, x0) and np.array_equal(v, v0)
        assert np.array_equal(u, u0) and np.array_equal(k, k0)


def test_fused_out_of_range_falls_back_to_the_plain_force_field(mdl):
    s = synth.workload("mol256")
    mr = _ranged(mdl, s)
    pos = _expanded(s)
    ctx = _ctx(s, mr, FUSED)
    e, f, terms = ctx.compute(pos)
    ep, fp, tp = O.Plain(s).energy_forces(pos)
    assert abs(e - ep) / s.n_atoms <= 1e-5
    assert np.sqrt(((f - fp) ** 2).mean()) <= 1e-4 * np.sqrt((fp ** 2).mean())
    for k in ("bond", "angle", "lj", "coulomb"):
        assert abs(terms[k] - tp[k]) / s.n_atoms <= 1e-5
    assert ctx.learned_counters()["fallback_steps"] == 1
    # back in range: the model, the same bits as the stage-by-stage path
    e2, f2, _ = ctx.compute(s.pos)
    e3, f3, _ = _ctx(s, mr, STAGED).compute(s.pos)
    assert e2 == e3 and np.array_equal(f2, f3)
    assert ctx.learned_counters()["fallback_steps"] == 1


def test_fused_out_of_range_without_fallback_is_an_error(mdl):
    s = synth.workload("mol256")
    mr = _ranged(mdl, s)
    ctx = _ctx(s, mr, FUSED, fallback=False)
    with pytest.raises(mdpf.MdpfError) as ei:
        ctx.compute(_expanded(s))
    assert ei.value.name == "OUT_OF_RANGE"


def test_fused_fallback_every_step_reproduces_the_plain_trajectory(mdl):
    s = synth.workload("mol256")
    r = model.Model(mdl.W1, mdl.b1, mdl.W2, mdl.b2, mdl.W3, mdl.b3, mdl.e0,
                    np.full((4, 384), -2.0, np.float32), np.full((4, 384), -1.0, np.float32))
    vel = synth.velocities(s.mass, s.pos, 300.0, 22)
    a = _ctx(s, r, FUSED, energy_every=1)
    a.set_state(s.pos, vel)
    a.step(25)
    b = mdpf.Context(s, stepper=mdpf.MDPF_STEPPER_KERNELS, energy_every=1)
    b.set_state(s.pos, vel)
    b.step(25)
    assert a.learned_counters()["fallback_steps"] == 26
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
