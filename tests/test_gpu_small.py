"""GPU parity of the persistent learned stepper for molecules of up to 32 atoms
(one cooperative launch for all steps, network weights resident in shared
memory) against the FP64 oracle and against the stage kernels of the learned
path, through the C ABI.

Tolerances: the stepper uses the tensor-core MLP's rounding points (BF16
features, the BF16 pair of CELU(z1), BF16 deltas and dE/dG, FP32 sums), so its
forces differ from the oracle's FP64 ones by the BF16 tolerance of the other
learned tests (force RMSE <= 1e-2 RMS), and its trajectories over a few tens
of 0.5 fs steps stay within 1e-4 A of the oracle's velocity Verlet.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_18271_b300 import mdpf, model, synth

pytestmark = pytest.mark.gpu

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


@pytest.mark.parametrize("n", [2, 9, 17, 32])
def test_small_md_follows_the_oracle(mdl, n):
    s = synth.molecule(n, seed=9 if n == 9 else 100 + n)
    vel = synth.velocities(s.mass, s.pos, 300.0, 21)
    ctx = _ctx(s, mdl, dt_fs=0.5, energy_every=1, trace_capacity=64)
    ctx.set_state(s.pos, vel)
    ctx.step(12)
    assert ctx.counters()["status"] == 0
    x, v = ctx.get_state()
    xo, vo = _vv_oracle(mdl, s, s.pos, vel, 0.5, 12)
    assert np.abs(x - xo).max() <= 1e-4
    assert np.abs(v - vo).max() <= 1e-4
    # the trace: U of each step against the oracle's energy at the stepper's own positions, K from v
    U, K = ctx.trace()
    assert len(U) == 12
    eo, _, _ = O.Learned(mdl).energy_forces(s.element, x)
    assert abs(U[-1] - eo) / n <= 1e-3
    k_end = 0.5 * np.sum(s.mass[:, None] * v * v) / O.ACC
    assert abs(K[-1] - k_end) <= 1e-9 * max(1.0, k_end)


def test_small_forces_match_the_stage_kernels(mdl):
    # the state forces after a step come from the stepper; the same positions through mdpf_compute use the
    # stage kernels (tensor-core MLP): the same model at the same rounding points
    s = synth.molecule(9, seed=9)
    vel = synth.velocities(s.mass, s.pos, 300.0, 22)
    ctx = _ctx(s, mdl, dt_fs=0.5, record_every=5, max_frames=4)
    ctx.set_state(s.pos, vel)
    ctx.step(20)
    pos, en, frc, st = ctx.frames()
    assert st.tolist() == [5, 10, 15, 20]
    for k in range(4):
        e_c, f_c, _ = ctx.compute(pos[k])
        rms = np.sqrt((f_c ** 2).mean())
        assert np.sqrt(((frc[k] - f_c) ** 2).mean()) <= 1e-2 * rms
        assert abs(en[k] - e_c) / s.n_atoms <= 1e-3
        eo, fo, _ = O.Learned(mdl).energy_forces(s.element, pos[k])
        assert np.sqrt(((frc[k] - fo) ** 2).mean()) <= 1e-2 * np.sqrt((fo ** 2).mean())


def test_small_split_steps_equal_one_run_and_repeat(mdl):
    s = synth.molecule(9, seed=9)
    vel = synth.velocities(s.mass, s.pos, 300.0, 23)
    runs = []
    for split in ((40,), (15, 25), (40,)):
        ctx = _ctx(s, mdl, energy_every=5, trace_capacity=64)
        ctx.set_state(s.pos, vel)
        for k in split:
            ctx.step(k)
        runs.append((ctx.get_state(), ctx.trace()))
    for (x, v), (U, K) in runs[1:]:
        assert np.array_equal(x, runs[0][0][0]) and np.array_equal(v, runs[0][0][1])
        assert np.array_equal(U, runs[0][1][0]) and np.array_equal(K, runs[0][1][1])


def test_small_and_stage_stepper_trajectories_agree(mdl):
    s = synth.molecule(9, seed=9)
    vel = synth.velocities(s.mass, s.pos, 300.0, 24)
    a = _ctx(s, mdl, energy_every=10, trace_capacity=64)
    b = _ctx(s, mdl, energy_every=10, trace_capacity=64, stepper=mdpf.MDPF_STEPPER_KERNELS)
    for c in (a, b):
        c.set_state(s.pos, vel)
        c.step(100)
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert np.abs(xa - xb).max() <= 1e-4
    Ua, Ka = a.trace()
    Ub, Kb = b.trace()
    assert np.abs(Ua - Ub).max() / s.n_atoms <= 1e-3


def test_small_fallback_runs_the_plain_force_field(mdl):
    # ranges that every feature violates: each step is a plain force-field step, counted
    s = synth.molecule(9, seed=9)
    r = model.Model(mdl.W1, mdl.b1, mdl.W2, mdl.b2, mdl.W3, mdl.b3, mdl.e0,
                    np.full((4, 384), -2.0, np.float32), np.full((4, 384), -1.0, np.float32))
    vel = synth.velocities(s.mass, s.pos, 300.0, 25)
    a = _ctx(s, r, energy_every=1, trace_capacity=64)
    a.set_state(s.pos, vel)
    a.step(40)
    b = mdpf.Context(s, stepper=mdpf.MDPF_STEPPER_KERNELS, energy_every=1, trace_capacity=64)
    b.set_state(s.pos, vel)
    b.step(40)
    assert a.learned_counters()["fallback_steps"] == 41
    xa, va = a.get_state()
    xb, vb = b.get_state()
    # the same FP32 pair and bonded terms, summed in another order: agreement to FP32 rounding
    assert np.abs(xa - xb).max() <= 1e-7 and np.abs(va - vb).max() <= 1e-7
    Ua, Ka = a.trace()
    Ub, Kb = b.trace()
    assert np.abs(Ua - Ub).max() <= 1e-4 * max(1.0, np.abs(Ub).max())
    fb = a.trace_fallbacks()
    assert fb.tolist() == list(range(2, 42))


def test_small_fallback_off_reports_out_of_range(mdl):
    s = synth.molecule(9, seed=9)
    r = model.Model(mdl.W1, mdl.b1, mdl.W2, mdl.b2, mdl.W3, mdl.b3, mdl.e0,
                    np.full((4, 384), -2.0, np.float32), np.full((4, 384), -1.0, np.float32))
    ctx = _ctx(s, r, fallback=False, energy_every=1)
    # the start evaluation already leaves the range (the state is set all the same), then every step does
    with pytest.raises(mdpf.MdpfError):
        ctx.set_state(s.pos, synth.velocities(s.mass, s.pos, 300.0, 26))
    with pytest.raises(mdpf.MdpfError) as err:
        ctx.step(5)
    assert err.value.name == "OUT_OF_RANGE"
    # out-of-range evaluations are counted with the fallback off too (the start and the first step here)
    assert ctx.learned_counters()["fallback_steps"] >= 2
