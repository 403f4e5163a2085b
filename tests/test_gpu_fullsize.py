"""Parity at the benchmark's full sizes, on the launch configurations the
bench times: the 16,384-atom learned cluster (neighbour rows, features,
energies and forces against the FP64 oracle; at this size the cell-list row
phase gives each warp several atoms) and full-width 2,048-atom training frames
(loss and parameter gradient against the oracle).  The oracle runs its
threaded loops on all host cores here (same results up to rounding).

Tolerances as for the smaller cases: rows identical; features RMSE <=
1e-4 RMS per block; BF16 forces RMSE <= 1e-2 RMS and energy <= 1e-3
kcal/mol/atom; training loss within 1e-2 relative and each parameter
tensor's gradient within 2e-2 relative RMSE."""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2412_18271_b300 import autograd as AG
from paper_2412_18271_b300 import mdpf, model, synth

pytestmark = pytest.mark.gpu

TRAINED = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2412_18271_b300", "data",
                       "learned_c3.mdpfmlp")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_18271_b300 import build
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.init()
    O.set_threads(os.cpu_count() or 1)
    yield
    O.set_threads(1)


@pytest.fixture(scope="module")
def c4():
    return synth.workload("cluster16384")


@pytest.fixture(scope="module")
def trained():
    with open(TRAINED, "rb") as fh:
        m = model.Model.unpack(fh.read())
    m.lo = m.hi = None
    return m


def _rel(a, b):
    return float(np.sqrt(((a - b) ** 2).mean()) / np.sqrt((b ** 2).mean()))


def test_cluster16384_neighbor_rows_bit_exact(c4, trained):
    ctx = mdpf.Context(c4, mode=mdpf.MDPF_MODE_LEARNED, model=trained.pack())
    cnt, rows = ctx.learned_neighbors(c4.pos)
    orows = O.neighbors(np.float32(c4.pos), O.RC_LIST)
    assert len(rows) == len(orows) == 16384
    for i, (a, b) in enumerate(zip(rows, orows)):
        assert np.array_equal(a, b), i
    assert ctx.learned_counters()["max_row"] == int(cnt.max())
    # after some MD the rows are rebuilt from moved atoms: still identical to the brute force
    ctx.set_state(c4.pos, np.zeros_like(c4.pos))
    ctx.init_velocities(300.0, 400)
    ctx.step(60)
    x, _ = ctx.get_state()
    _, rows2 = ctx.learned_neighbors(x)
    orows2 = O.neighbors(np.float32(x), O.RC_LIST)
    assert all(np.array_equal(a, b) for a, b in zip(rows2, orows2))
    ctx.close()


def test_cluster16384_features_match_oracle(c4, trained):
    ctx = mdpf.Context(c4, mode=mdpf.MDPF_MODE_LEARNED, model=trained.pack())
    G = ctx.learned_features(c4.pos).astype(np.float64)
    Go = O.features(c4.element, c4.pos)
    for sl in (slice(0, 64), slice(64, 384)):
        assert _rel(G[:, sl], Go[:, sl]) <= 1e-4, sl
    assert np.all(G[Go == 0.0] == 0.0)
    ctx.close()


@pytest.mark.parametrize("kernel", [mdpf.MDPF_MLP_TENSOR, mdpf.MDPF_MLP_FUSED])
def test_cluster16384_energy_forces_match_oracle(c4, trained, kernel):
    for m in (model.init_model(7), trained):
        ctx = mdpf.Context(c4, mode=mdpf.MDPF_MODE_LEARNED, model=m.pack(), mlp_kernel=kernel)
        e, f, _ = ctx.compute(c4.pos)
        eo, fo, _ = O.Learned(m).energy_forces(c4.element, c4.pos)
        assert _rel(f, fo) <= 1e-2
        assert abs(e - eo) / c4.n_atoms <= 1e-3, (e, eo)
        ctx.close()


def test_full_width_training_frames_match_oracle(trained):
    # two 2048-atom frames recorded by the plain path (the training data's own kind)
    s = synth.workload("cluster2048")
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=100)
    ctx = mdpf.Context(s, dt_fs=0.5, record_every=50, max_frames=2, energy_every=10)
    ctx.set_state(s.pos, v0)
    ctx.step(100)
    P, En, Fr, _ = ctx.frames(2)
    ctx.close()
    frames = [(s.element, P[k], float(En[k]), Fr[k].astype(np.float64)) for k in range(2)]
    dev = torch.device("cuda")
    pos = torch.tensor(P.reshape(-1, 3), dtype=torch.float64, device=dev).contiguous()
    el = torch.tensor(np.concatenate([s.element, s.element]).astype(np.int32), device=dev)
    E = torch.tensor(En, dtype=torch.float64, device=dev)
    F = torch.tensor(Fr.reshape(-1, 3), dtype=torch.float32, device=dev).contiguous()
    tr = mdpf.Trainer(2, s.n_atoms, trained.e0, core_a=trained.core_a, core_rc=trained.core_rc)
    params = torch.tensor(model.to_flat(trained), device=dev, requires_grad=True)
    L, parts = AG.ForceMatchingLoss.apply(params, tr, pos, el, E, F)
    L.backward()
    assert tr.status() == 0
    Lo, go, _ = O.train_loss_grad(trained, frames)
    assert abs(float(L.detach()) - Lo) <= 1e-2 * abs(Lo)
    g = model.from_flat(params.grad.detach().cpu().numpy(), trained.e0)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        assert _rel(np.asarray(getattr(g, k), dtype=np.float64), go[k]) <= 2e-2, k
