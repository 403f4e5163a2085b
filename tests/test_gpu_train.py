"""GPU parity of the training path: feature JVP, the device force-matching
loss and its gradient, AdamW, the autograd wrappers and the feature range,
against the FP64 oracle.

Tolerances:
  JVP (FP32)         RMSE <= 1e-4 * RMS(U_oracle), radial and angular blocks separately
  loss / gradient    the forward runs the BF16 tensor-core MLP (energies ~6e-5
                     kcal/mol/atom, forces ~4e-3 of RMS from the FP64 values), the
                     gradient arithmetic is FP32: loss within 1e-2 relative, each
                     parameter tensor's gradient RMSE <= 2e-2 of its RMS
  AdamW (FP32)       within 1e-6 relative of the FP64 update
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2412_18271_b300 import autograd as AG
from paper_2412_18271_b300 import mdpf, model, synth

pytestmark = pytest.mark.gpu

E0 = np.array([-0.5, -38.0, -54.6, -75.1])


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_18271_b300 import build
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.init()


@pytest.fixture(scope="module")
def mdl():
    m = model.init_model(7)
    m.e0 = E0.copy()
    m.b1 = np.random.default_rng(1).normal(0, 0.2, m.b1.shape).astype(np.float32)
    return m.rounded()


def _batch(n_frames=3, name="mol64", seed=5, noise=0.05):
    s = synth.workload(name)
    rng = np.random.default_rng(seed)
    plain = O.Plain(s)
    frames = []
    for _ in range(n_frames):
        pos = s.pos + rng.normal(0, noise, s.pos.shape)
        e, f, _ = plain.energy_forces(pos)
        frames.append((s.element, pos, e, f.astype(np.float32).astype(np.float64)))
    return s, frames


def _device_batch(frames):
    dev = torch.device("cuda")
    pos = torch.tensor(np.concatenate([f[1] for f in frames]), dtype=torch.float64, device=dev).contiguous()
    el = torch.tensor(np.concatenate([f[0] for f in frames]), dtype=torch.int32, device=dev)
    E = torch.tensor([f[2] for f in frames], dtype=torch.float64, device=dev)
    F = torch.tensor(np.concatenate([f[3] for f in frames]), dtype=torch.float32, device=dev).contiguous()
    return pos, el, E, F


def _grad_via_autograd(m, frames, trainer):
    params = torch.tensor(model.to_flat(m), device="cuda", requires_grad=True)
    pos, el, E, F = _device_batch(frames)
    L, parts = AG.ForceMatchingLoss.apply(params, trainer, pos, el, E, F)
    L.backward()
    assert trainer.status() == 0
    return float(L.detach()), parts.cpu().numpy(), params.grad.cpu().numpy()


# ------------------------------------------------------------ feature JVP

@pytest.mark.parametrize("name", ["mol64", "mol256"])
def test_jvp_matches_oracle(name, mdl):
    s = synth.workload(name)
    ctx = mdpf.Context(s, mode=mdpf.MDPF_MODE_LEARNED, model=mdl.pack())
    v = np.random.default_rng(3).normal(0, 1.0, s.pos.shape).astype(np.float32)
    U = ctx.learned_jvp(s.pos, v).astype(np.float64)
    Uo = O.feature_jvp(s.element, s.pos, v.astype(np.float64))
    for sl in (slice(0, 64), slice(64, 384)):
        d = U[:, sl] - Uo[:, sl]
        assert np.sqrt((d ** 2).mean()) <= 1e-4 * np.sqrt((Uo[:, sl] ** 2).mean()), sl


# ------------------------------------------------------------ loss and gradient

def _rel_rmse(a, b):
    return np.sqrt(((a - b) ** 2).mean()) / max(np.sqrt((b ** 2).mean()), 1e-30)


def test_loss_includes_the_repulsive_core(mdl):
    # one frame with a bonded pair pulled inside the core radius: the loss and gradient follow the
    # oracle's, whose predicted energy and forces include the core
    s, frames = _batch()
    el, pos, e_ref, f_ref = frames[1]
    pos = pos.copy()
    a, b = s.bonds[5]
    d = pos[b] - pos[a]
    pos[b] = pos[a] + d / np.linalg.norm(d) * 0.5
    frames[1] = (el, pos, e_ref, f_ref)
    assert O.core_energy_forces(pos, mdl.core_a, mdl.core_rc)[0] > 30.0
    tr = mdpf.Trainer(len(frames), s.n_atoms, mdl.e0, core_a=mdl.core_a, core_rc=mdl.core_rc)
    L, parts, g = _grad_via_autograd(mdl, frames, tr)
    Lo, go, _ = O.train_loss_grad(mdl, frames)
    assert abs(L - Lo) <= 1e-2 * abs(Lo), (L, Lo)
    gm = model.from_flat(g, mdl.e0)
    present = np.unique(s.element)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        a_ = np.asarray(getattr(gm, k), dtype=np.float64)[present]
        assert _rel_rmse(a_, go[k][present]) <= 2e-2, k
    # without the core the device loss is a different number
    tr0 = mdpf.Trainer(len(frames), s.n_atoms, mdl.e0)
    L0, _, _ = _grad_via_autograd(mdl, frames, tr0)
    assert abs(L0 - L) > 1e-3 * abs(L)


def test_loss_and_gradient_match_oracle(mdl):
    s, frames = _batch()
    tr = mdpf.Trainer(len(frames), s.n_atoms, mdl.e0, core_a=mdl.core_a, core_rc=mdl.core_rc)
    L, parts, g = _grad_via_autograd(mdl, frames, tr)
    Lo, go, _ = O.train_loss_grad(mdl, frames)
    assert abs(L - Lo) <= 1e-2 * abs(Lo), (L, Lo)
    assert abs(parts[0] - parts[1] - parts[2]) <= 1e-12 * abs(parts[0])
    gm = model.from_flat(g, mdl.e0)
    present = np.unique(s.element)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        a = np.asarray(getattr(gm, k), dtype=np.float64)[present]
        b = go[k][present]
        assert _rel_rmse(a, b) <= 2e-2, (k, _rel_rmse(a, b))
    absent = [e for e in range(4) if e not in present]
    for e in absent:
        assert np.all(g.reshape(4, -1)[e] == 0.0)


def test_gradient_is_deterministic(mdl):
    s, frames = _batch(seed=6)
    tr = mdpf.Trainer(len(frames), s.n_atoms, mdl.e0, core_a=mdl.core_a, core_rc=mdl.core_rc)
    _, _, g1 = _grad_via_autograd(mdl, frames, tr)
    _, _, g2 = _grad_via_autograd(mdl, frames, tr)
    assert np.array_equal(g1, g2)


def test_zero_residual_gives_near_zero_gradient(mdl):
    s, frames = _batch(seed=7)
    ctx = mdpf.Context(s, mode=mdpf.MDPF_MODE_LEARNED, model=mdl.pack())
    own = []
    for el, pos, _, _ in frames:
        e, f, _ = ctx.compute(pos)
        own.append((el, pos, e, f.astype(np.float32).astype(np.float64)))
    tr = mdpf.Trainer(len(frames), s.n_atoms, mdl.e0, core_a=mdl.core_a, core_rc=mdl.core_rc)
    L0, _, g0 = _grad_via_autograd(mdl, own, tr)
    L1, _, g1 = _grad_via_autograd(mdl, frames, tr)
    assert L0 <= 1e-9 * L1
    assert np.linalg.norm(g0) <= 1e-5 * np.linalg.norm(g1)


def test_multi_frame_batch_with_different_molecules(mdl):
    # frames of different molecules (different element sequences), same atom count
    frames = []
    rng = np.random.default_rng(8)
    for seed in (11, 12, 13, 14):
        s = synth.molecule(48, seed=seed)
        e, f, _ = O.Plain(s).energy_forces(s.pos)
        frames.append((s.element, s.pos + rng.normal(0, 0.02, s.pos.shape), e, f))
    tr = mdpf.Trainer(4, 48, mdl.e0, core_a=mdl.core_a, core_rc=mdl.core_rc)
    L, _, g = _grad_via_autograd(mdl, frames, tr)
    Lo, go, _ = O.train_loss_grad(mdl, frames)
    assert abs(L - Lo) <= 1e-2 * abs(Lo)
    gm = model.from_flat(g, mdl.e0)
    for k in ("W1", "W2", "W3"):
        assert _rel_rmse(np.asarray(getattr(gm, k), np.float64), go[k]) <= 2e-2, k


# ------------------------------------------------------------ AdamW, training

def test_adamw_matches_oracle():
    rng = np.random.default_rng(9)
    n = 100_003
    th = rng.normal(size=n).astype(np.float32)
    p = torch.tensor(th, device="cuda")
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    tho, mo, vo = th.astype(np.float64), np.zeros(n), np.zeros(n)
    for t in range(1, 6):
        g = rng.normal(size=n).astype(np.float32)
        gd = torch.tensor(g, device="cuda")
        lr = O.cosine_lr(t - 1, 1e-3, 10)
        mdpf.adamw_step(p.data_ptr(), gd.data_ptr(), m.data_ptr(), v.data_ptr(), n, t, lr)
        O.adamw_step(tho, g.astype(np.float64), mo, vo, t, lr)
    torch.cuda.synchronize()
    assert np.allclose(p.cpu().numpy(), tho, rtol=1e-6, atol=1e-7)


def test_training_reduces_the_loss(mdl):
    s, frames = _batch(n_frames=4, seed=10)
    tr = mdpf.Trainer(4, s.n_atoms, mdl.e0, core_a=mdl.core_a, core_rc=mdl.core_rc)
    params = torch.tensor(model.to_flat(mdl), device="cuda", requires_grad=True)
    opt = AG.CosineAdamW([params], lr=1e-3, total_steps=60)
    pos, el, E, F = _device_batch(frames)
    losses = []
    for _ in range(60):
        opt.zero_grad()
        L, _ = AG.ForceMatchingLoss.apply(params, tr, pos, el, E, F)
        L.backward()
        opt.step()
        losses.append(float(L.detach()))
    assert tr.status() == 0
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])


def test_feature_range_matches_oracle(mdl):
    s, frames = _batch(seed=12)
    tr = mdpf.Trainer(len(frames), s.n_atoms, mdl.e0, core_a=mdl.core_a, core_rc=mdl.core_rc)
    _grad_via_autograd(mdl, frames, tr)
    lo, hi = tr.feature_range()
    G = np.concatenate([O.features(f[0], f[1]) for f in frames])
    el = np.concatenate([f[0] for f in frames])
    for e in np.unique(el):
        sel = G[el == e]
        assert np.allclose(lo[e], sel.min(0), rtol=1e-4, atol=1e-5)
        assert np.allclose(hi[e], sel.max(0), rtol=1e-4, atol=1e-5)


def test_learned_energy_autograd_gives_minus_forces(mdl):
    s = synth.workload("mol64")
    ctx = mdpf.Context(s, mode=mdpf.MDPF_MODE_LEARNED, model=mdl.pack())
    e, f, _ = ctx.compute(s.pos)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda", requires_grad=True)
    E = AG.LearnedEnergy.apply(pos, ctx)
    E.backward()
    torch.cuda.synchronize()
    assert abs(float(E.detach()) - e) <= 1e-9 * max(1.0, abs(e))
    assert np.allclose(pos.grad.cpu().numpy(), -f, rtol=1e-6, atol=1e-6)
