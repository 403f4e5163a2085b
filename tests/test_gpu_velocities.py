"""Device Maxwell-Boltzmann initial velocities (mdpf_init_velocities) against
the FP64 oracle's draw from the same counter-based normals, and the extended
counters (h_now, rebuilds, fallbacks, max_disp), through the C ABI.

Tolerance: the same FP64 arithmetic on both sides, reductions in a different
order: max |v - v_oracle| <= 1e-12 max |v|."""
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


@pytest.mark.parametrize("name,T,seed", [("mol64", 300.0, 0), ("cluster2048", 300.0, 100), ("mol256", 50.0, 7)])
def test_velocities_match_oracle(name, T, seed):
    s = synth.workload(name)
    ctx = mdpf.Context(s, dt_fs=0.5)
    ctx.set_state(s.pos, np.zeros_like(s.pos))
    u0 = ctx.counters()["potential"]
    ctx.init_velocities(T, seed)
    x, v = ctx.get_state()
    vo = O.init_velocities(s.mass, s.pos, T, seed)
    assert np.array_equal(x, s.pos)
    assert np.abs(v - vo).max() <= 1e-12 * np.abs(vo).max()
    c = ctx.counters()
    k_target = 0.5 * (3 * s.n_atoms - 6) * KB * T
    assert c["kinetic"] == pytest.approx(k_target, rel=1e-9)
    assert c["h_initial"] == pytest.approx(u0 + k_target, rel=1e-9)
    assert c["h_now"] == pytest.approx(c["potential"] + c["kinetic"], rel=1e-15)
    assert c["rebuilds"] == 0 and c["fallbacks"] == 0 and c["max_disp"] == 0.0
    # stepping from the drawn state conserves what the plain path conserves (zero net momentum)
    ctx.step(20)
    _, v2 = ctx.get_state()
    assert np.abs((s.mass[:, None] * v2).sum(0)).max() <= 1e-9 * np.abs(s.mass[:, None] * v2).sum()
    ctx.close()


def test_init_velocities_needs_a_state_and_a_temperature():
    s = synth.workload("mol64")
    ctx = mdpf.Context(s, dt_fs=0.5)
    with pytest.raises(mdpf.MdpfError) as ei:
        ctx.init_velocities(300.0, 0)
    assert ei.value.name == "INVALID_ARG"
    ctx.set_state(s.pos, np.zeros_like(s.pos))
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(mdpf.MdpfError):
            ctx.init_velocities(bad, 0)
    ctx.init_velocities(0.0, 0)
    _, v = ctx.get_state()
    assert np.all(v == 0.0)
    ctx.close()


def test_learned_counters_in_the_extended_struct():
    s = synth.workload("mol256")
    m = model.init_model(7)
    ctx = mdpf.Context(s, mode=mdpf.MDPF_MODE_LEARNED, model=m.pack(), dt_fs=0.5, skin=1.0, rebuild_every=20)
    ctx.set_state(s.pos, np.zeros_like(s.pos))
    ctx.init_velocities(300.0, 200)
    ctx.step(50)
    c = ctx.counters()
    lc = ctx.learned_counters()
    assert c["rebuilds"] == lc["rebuilds"] >= 3        # set_state's build and every 20 steps at least
    assert c["fallbacks"] == lc["fallback_steps"] == 0
    # after a step the list is never more than skin/2 behind (a larger move triggers a rebuild)
    assert 0.0 <= c["max_disp"] <= 0.5 + 1e-6
    x, _ = ctx.get_state()
    assert c["h_now"] == pytest.approx(c["potential"] + c["kinetic"], rel=1e-15)
    ctx.close()
