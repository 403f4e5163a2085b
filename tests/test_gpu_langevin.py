"""GPU Langevin dynamics (BAOAB, Philox4x32-10 normals) against the FP64 oracle.

Both sides draw the same normals (counter = atom, step; key = seed), so the
trajectories agree to FP32-force accuracy (as velocity Verlet does), not just
in distribution."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_18271_b300 import mdpf, model, synth

pytestmark = pytest.mark.gpu
KB = 0.0019872041


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_18271_b300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()
    torch.cuda.init()


def test_langevin_trajectory_matches_the_oracle():
    s = synth.workload("mol64")
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=0)
    ctx = mdpf.Context(s, dt_fs=0.5, friction_per_ps=5.0, temperature_K=300.0, seed=123)
    ctx.set_state(s.pos, v0)
    ctx.step(50)
    x, v = ctx.get_state()
    xo, vo, Uo, Ko = O.Plain(s).langevin(s.pos, v0, 0.5, 50, gamma_ps=5.0, temp_K=300.0, seed=123)
    assert np.abs(x - xo).max() < 1e-4
    assert np.abs(v - vo).max() < 1e-4
    U, K = ctx.trace()
    assert np.abs(K - Ko).max() / s.n_atoms < 1e-4


def test_langevin_is_deterministic_and_seeded():
    s = synth.workload("mol64")
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=0)
    out = []
    for seed in (5, 5, 6):
        ctx = mdpf.Context(s, dt_fs=0.5, friction_per_ps=1.0, temperature_K=300.0, seed=seed)
        ctx.set_state(s.pos, v0)
        ctx.step(30)
        ctx.step(20)
        out.append(ctx.get_state()[0])
    assert np.array_equal(out[0], out[1])
    assert not np.array_equal(out[0], out[2])


def test_thermostat_holds_the_cluster_at_the_bath_temperature():
    s = synth.workload("cluster2048")
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=100)
    T = 300.0
    ctx = mdpf.Context(s, dt_fs=0.5, friction_per_ps=20.0, temperature_K=T, seed=9, trace_capacity=4000)
    ctx.set_state(s.pos, v0)
    ctx.step(4000)
    U, K = ctx.trace()
    assert abs(K[2000:].mean() / (1.5 * s.n_atoms * KB * T) - 1.0) < 0.03


def test_langevin_with_the_learned_potential():
    s = synth.workload("mol256")
    m = model.init_model(7)
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=2)
    a = mdpf.Context(s, mode=mdpf.MDPF_MODE_LEARNED, model=m.pack(), friction_per_ps=2.0, temperature_K=300.0,
                     seed=4)
    a.set_state(s.pos, v0)
    a.step(100)
    b = mdpf.Context(s, mode=mdpf.MDPF_MODE_LEARNED, model=m.pack(), friction_per_ps=2.0, temperature_K=300.0,
                     seed=4)
    b.set_state(s.pos, v0)
    b.set_profiling(True)   # kernel-by-kernel launches instead of the step graph
    b.step(100)
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert np.isfinite(a.counters()["kinetic"])
