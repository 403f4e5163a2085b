"""The oracle's threaded loops (used only to time the CPU baseline on all host
cores) give the serial results up to rounding: the same terms, summed per
thread and then in thread order."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_18271_b300 import model, synth


@pytest.fixture
def threads():
    yield
    O.set_threads(1)


def _close(a, b, rel=1e-12):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.abs(a - b).max() <= rel * max(np.abs(b).max(), 1e-300)


def test_plain_threaded_equals_serial(threads):
    s = synth.workload("mol256")
    O.set_threads(1)
    e1, f1, t1 = O.Plain(s).energy_forces(s.pos)
    assert O.set_threads(4) == 4
    e4, f4, t4 = O.Plain(s).energy_forces(s.pos)
    assert e4 == pytest.approx(e1, rel=1e-12)
    assert _close(f4, f1)
    for k in t1:
        assert t4[k] == pytest.approx(t1[k], rel=1e-11, abs=1e-9)


def test_learned_threaded_equals_serial(threads):
    s = synth.workload("mol64")
    m = model.init_model(7)
    O.set_threads(1)
    e1, f1, g1 = O.Learned(m).energy_forces(s.element, s.pos)
    O.set_threads(3)
    e3, f3, g3 = O.Learned(m).energy_forces(s.element, s.pos)
    assert np.array_equal(g1, g3)          # features are written row by row: identical
    assert e3 == e1                        # energies summed in atom order: identical
    assert _close(f3, f1)


def test_param_grad_threaded_equals_serial(threads):
    s = synth.workload("mol64")
    m = model.init_model(7)
    rng = np.random.default_rng(2)
    G = O.features(s.element, s.pos)
    U = rng.normal(size=G.shape)
    c = rng.normal(size=s.n_atoms)
    O.set_threads(1)
    g1 = O.mlp_param_grad(m, s.element, G, U, c)
    O.set_threads(4)
    g4 = O.mlp_param_grad(m, s.element, G, U, c)
    for k in g1:
        assert _close(g4[k], g1[k]), k
