"""NVE energy conservation of the learned BF16 path over 10,000 steps, and the
accounting of steps that fall back to the plain force field, through the C ABI.

Bound (a reading of the paper's NVE criterion, Results, "Example: Ethanol":
the total energy of the NVE runs is conserved to the precision of the force
arithmetic): drift = |least-squares slope of H(t)/N| x run length
<= 1e-2 kcal/mol/atom over 10,000 steps of 0.5 fs for the BF16 learned path,
with steps where the force field switches (fallback on/off) excluded and
counted separately."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_18271_b300 import mdpf, model, synth
from paper_2412_18271_b300.energy_drift import nve_drift

pytestmark = pytest.mark.gpu

LEARNED_DRIFT_BOUND = 1e-2


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_18271_b300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()
    torch.cuda.init()


@pytest.mark.parametrize("kernel", [mdpf.MDPF_MLP_TENSOR, mdpf.MDPF_MLP_FUSED])
def test_learned_bf16_nve_drift_10k_steps(kernel):
    s = synth.workload("mol256")
    m = model.init_model(7)                   # seeded Kaiming init with the repulsive core
    ctx = mdpf.Context(s, mode=mdpf.MDPF_MODE_LEARNED, model=m.pack(), dt_fs=0.5, energy_every=1,
                       trace_capacity=10000, mlp_kernel=kernel)
    ctx.set_state(s.pos, np.zeros_like(s.pos))
    ctx.init_velocities(300.0, synth.WORKLOAD_VELOCITY_SEED["mol256"])
    fb0 = ctx.counters()["fallbacks"]
    ctx.step(10000)
    U, K = ctx.trace()
    fb = ctx.trace_fallbacks()
    assert U.size == 10000 and fb.size == 10000
    r = nve_drift(U, K, s.n_atoms, fb, fb0)
    assert r["plain_steps"] == 0 and r["switch_steps"] == 0
    assert r["drift"] <= LEARNED_DRIFT_BOUND, r
    c = ctx.counters()
    assert c["status"] == 0 and c["steps"] == 10000
    # the initial energy right after set_state/init_velocities is the first point of the same line
    assert abs(c["h_initial"] / s.n_atoms - (U[0] + K[0]) / s.n_atoms) < LEARNED_DRIFT_BOUND
    ctx.close()


def test_trained_model_nve_drift_on_its_training_cluster():
    # the trained model on the 2048-atom cluster it was trained on (in distribution; no ranges): the
    # cluster heats to ~850 K as its start strain relaxes, where the fitted potential is stiffer than the
    # plain force field.  At dt = 0.5 fs velocity Verlet drifts 0.025 kcal/mol/atom over 10k steps with
    # either MLP precision (integration error); halving the step cuts that by 8x (BF16) and 27x (FP32).
    # So the energy conservation of the learned BF16 path is checked with the step resolved: 10,000
    # steps of 0.25 fs, A16's bound.
    import os
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(here, "paper_2412_18271_b300", "data", "learned_c3.mdpfmlp"), "rb") as fh:
        m = model.Model.unpack(fh.read())
    m.lo = m.hi = None
    s = synth.workload("cluster2048")
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=synth.WORKLOAD_VELOCITY_SEED["cluster2048"])
    ctx = mdpf.Context(s, mode=mdpf.MDPF_MODE_LEARNED, model=m.pack(), dt_fs=0.25, energy_every=1,
                       trace_capacity=10000)
    ctx.set_state(s.pos, v0)
    ctx.step(10000)
    U, K = ctx.trace()
    r = nve_drift(U, K, s.n_atoms)
    assert r["drift"] <= LEARNED_DRIFT_BOUND, r
    assert ctx.counters()["status"] == 0
    ctx.close()


def _ranged(m, s, widen):
    G = O.features(s.element, s.pos)
    lo = np.zeros((4, 384), dtype=np.float32)
    hi = np.zeros((4, 384), dtype=np.float32)
    for e in range(4):
        sel = G[s.element == e]
        if sel.size:
            a, b = sel.min(0), sel.max(0)
            lo[e] = a - widen * (b - a) - 1e-6
            hi[e] = b + widen * (b - a) + 1e-6
    return model.Model(m.W1, m.b1, m.W2, m.b2, m.W3, m.b3, m.e0, lo, hi, m.alpha, m.core_a, m.core_rc)


def test_fallback_steps_in_the_trace_match_the_counters():
    # a range fitted to the start geometry only: as the molecule moves, some steps leave it and run
    # on the plain force field; the trace's per-step record and the counters must agree
    s = synth.workload("mol256")
    mr = _ranged(model.init_model(7), s, widen=0.02)
    ctx = mdpf.Context(s, mode=mdpf.MDPF_MODE_LEARNED, model=mr.pack(), dt_fs=0.5, energy_every=1,
                       trace_capacity=300)
    ctx.set_state(s.pos, np.zeros_like(s.pos))
    ctx.init_velocities(300.0, 3)
    fb0 = ctx.counters()["fallbacks"]
    ctx.step(300)
    U, K = ctx.trace()
    fb = ctx.trace_fallbacks()
    c = ctx.counters()
    r = nve_drift(U, K, s.n_atoms, fb, fb0)
    assert fb[-1] == c["fallbacks"] == ctx.learned_counters()["fallback_steps"]
    assert r["plain_steps"] == c["fallbacks"] - fb0 > 0
    assert np.all(np.diff(np.concatenate([[fb0], fb])) <= 1)    # one evaluation per step
    ctx.close()


def test_plain_mode_trace_has_no_fallbacks():
    s = synth.workload("mol64")
    ctx = mdpf.Context(s, dt_fs=0.5, energy_every=1, trace_capacity=50)
    ctx.set_state(s.pos, np.zeros_like(s.pos))
    ctx.step(50)
    assert np.all(ctx.trace_fallbacks() == 0)
    ctx.close()
