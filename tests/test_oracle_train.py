"""Pins of the oracle's force-matching loss gradient (FP64, CPU).

The training gradient has two parts: the energy term (ordinary reverse mode)
and the force term, which reaches the parameters through the MLP's input
gradient (reverse mode over the tangent pass along U = J v).  Pins:
  - central finite differences of the whole loss (features, MLP, forces) in
    every parameter tensor of every element present;
  - an independent torch FP64 double-backward of the per-row objective;
  - the zero-residual case (targets equal to the model's own outputs);
  - linearity of the MLP gradient in the weights c and the tangents U.
"""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2412_18271_b300 import model, synth


def _model64(seed):
    m = model.init_model(seed)
    rng = np.random.default_rng(seed + 100)
    f = {k: np.asarray(getattr(m, k), dtype=np.float64).copy() for k in ("W1", "b1", "W2", "b2", "W3", "b3")}
    f["b1"] += rng.normal(0, 0.3, f["b1"].shape)
    f["b2"] += rng.normal(0, 0.3, f["b2"].shape)
    f["b3"] += rng.normal(0, 0.1, f["b3"].shape)
    return model.Model(f["W1"], f["b1"], f["W2"], f["b2"], f["W3"], f["b3"], np.array([-0.5, -38.0, -54.6, -75.1]))


def _frames(n_atoms=14, n_frames=2, seed=3):
    s = synth.molecule(n_atoms, seed=seed)
    rng = np.random.default_rng(seed)
    frames = []
    for k in range(n_frames):
        pos = s.pos + rng.normal(0, 0.05, s.pos.shape)
        frames.append((s.element, pos, float(rng.normal(-30, 5)), rng.normal(0, 2.0, s.pos.shape)))
    return s, frames


@pytest.fixture(scope="module")
def setup():
    m = _model64(11)
    s, frames = _frames()
    L, g, _ = O.train_loss_grad(m, frames)
    return m, s, frames, L, g


def test_zero_residual_gives_zero_loss_and_gradient():
    m = _model64(12)
    s, frames = _frames(seed=4)
    lrn = O.Learned(m)
    own = []
    for el, pos, _, _ in frames:
        E, F, _ = lrn.energy_forces(el, pos)
        own.append((el, pos, E, F))
    L, g, _ = O.train_loss_grad(m, own)
    assert L == 0.0
    for k, v in g.items():
        assert np.all(v == 0.0), k


@pytest.mark.parametrize("name", ["W1", "b1", "W2", "b2", "W3", "b3"])
def test_loss_gradient_matches_finite_differences(setup, name):
    m, s, frames, L0, g = setup
    rng = np.random.default_rng(7)
    present = np.unique(s.element)
    h = 1e-6
    arr = getattr(m, name)
    scale = np.abs(g[name]).max()
    for e in present:
        for _ in range(4):
            idx = (e,) + tuple(int(rng.integers(0, d)) for d in arr.shape[1:])
            plus = dataclasses.replace(m, **{name: arr.copy()})
            minus = dataclasses.replace(m, **{name: arr.copy()})
            getattr(plus, name)[idx] += h
            getattr(minus, name)[idx] -= h
            Lp, _, _ = O.train_loss_grad(plus, frames)
            Lm, _, _ = O.train_loss_grad(minus, frames)
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - g[name][idx]) <= 1e-6 * scale + 1e-5 * abs(fd), (name, idx, fd, g[name][idx])


def test_elements_absent_from_the_batch_get_no_gradient(setup):
    m, s, frames, L0, g = setup
    for e in range(4):
        if e not in s.element:
            for k in g:
                assert np.all(g[k][e] == 0.0)


def _torch_objective_grads(m, element, G, U, c):
    """Independent FP64 torch evaluation: grad over parameters of
    sum_i [c_i E_i - U_i . dE_i/dG_i] via autograd double-backward."""
    params = {k: torch.tensor(np.asarray(getattr(m, k), dtype=np.float64), requires_grad=True)
              for k in ("W1", "b1", "W2", "b2", "W3", "b3")}
    Gt = torch.tensor(G, requires_grad=True)
    el = torch.tensor(element, dtype=torch.long)
    W1, b1, W2, b2, W3, b3 = (params[k][el] for k in ("W1", "b1", "W2", "b2", "W3", "b3"))
    a1 = torch.nn.functional.celu(torch.einsum("naf,nf->na", W1, Gt) + b1, alpha=0.1)
    a2 = torch.nn.functional.celu(torch.einsum("nba,na->nb", W2, a1) + b2, alpha=0.1)
    E = (W3 * a2).sum(1) + b3
    (dEdG,) = torch.autograd.grad(E.sum(), Gt, create_graph=True)
    J = (torch.tensor(c) * E).sum() - (torch.tensor(U) * dEdG).sum()
    gr = torch.autograd.grad(J, list(params.values()))
    return {k: v.detach().numpy() for k, v in zip(params, gr)}


def test_mlp_gradient_matches_torch_double_backward():
    m = _model64(13)
    rng = np.random.default_rng(21)
    n = 40
    el = rng.integers(0, 4, n).astype(np.int32)
    G = rng.gamma(0.5, 1.0, (n, 384)) * (rng.random((n, 384)) < 0.6)
    U = rng.normal(0, 0.3, (n, 384))
    c = rng.normal(0, 1.0, n)
    g = O.mlp_param_grad(m, el, G, U, c)
    gt = _torch_objective_grads(m, el, G, U, c)
    for k in g:
        # torch forms celu'(z) as (celu(z) + alpha) / alpha, which loses ~1e-8 absolute
        assert np.allclose(g[k], gt[k], rtol=1e-6, atol=1e-7 * np.abs(gt[k]).max()), k


def test_mlp_gradient_is_linear_in_weights_and_tangents():
    m = _model64(14)
    rng = np.random.default_rng(22)
    n = 12
    el = rng.integers(0, 4, n).astype(np.int32)
    G = rng.gamma(0.5, 1.0, (n, 384))
    U1, U2 = rng.normal(0, 0.3, (n, 384)), rng.normal(0, 0.3, (n, 384))
    c1, c2 = rng.normal(0, 1, n), rng.normal(0, 1, n)
    ga = O.mlp_param_grad(m, el, G, U1 + 2 * U2, c1 - 3 * c2)
    g1 = O.mlp_param_grad(m, el, G, U1, c1)
    g2 = O.mlp_param_grad(m, el, G, U2, c2)
    g0 = O.mlp_param_grad(m, el, G, np.zeros_like(U1), np.zeros(n))
    for k in ga:
        assert np.all(g0[k] == 0.0)
        comb = g1[k] + 2 * (g2[k] - O.mlp_param_grad(m, el, G, np.zeros_like(U1), c2)[k]) \
            - 3 * O.mlp_param_grad(m, el, G, np.zeros_like(U1), c2)[k]
        assert np.allclose(ga[k], comb, rtol=1e-9, atol=1e-12 * max(1.0, np.abs(ga[k]).max())), k


# ---------------------------------------------------------------- AdamW + cosine

def test_cosine_schedule_endpoints_and_midpoint():
    assert O.cosine_lr(0, 1e-3, 100) == 1e-3
    assert abs(O.cosine_lr(50, 1e-3, 100) - 0.5e-3) < 1e-18
    assert O.cosine_lr(100, 1e-3, 100) == 0.0
    lrs = [O.cosine_lr(t, 1e-3, 100) for t in range(101)]
    assert all(a >= b for a, b in zip(lrs, lrs[1:]))


def test_adamw_first_step_closed_form():
    rng = np.random.default_rng(5)
    th = rng.normal(size=50)
    g = rng.normal(size=50)
    m, v = np.zeros(50), np.zeros(50)
    out = O.adamw_step(th.copy(), g, m, v, 1, 1e-3)
    # first step: mh = g, vh = g^2
    expect = th - 1e-3 * (g / (np.abs(g) + 1e-8) + 0.01 * th)
    assert np.allclose(out, expect, rtol=1e-14, atol=1e-16)


def test_adamw_matches_torch_over_steps():
    rng = np.random.default_rng(6)
    th0 = rng.normal(size=(7, 5))
    grads = [rng.normal(size=(7, 5)) for _ in range(12)]
    p = torch.nn.Parameter(torch.tensor(th0.copy()))
    opt = torch.optim.AdamW([p], lr=1e-3, betas=(0.9, 0.999), eps=1e-8, weight_decay=0.01)
    th = th0.copy()
    m, v = np.zeros_like(th), np.zeros_like(th)
    for t, g in enumerate(grads, start=1):
        lr = O.cosine_lr(t - 1, 1e-3, 20)
        for gr in opt.param_groups:
            gr["lr"] = lr
        p.grad = torch.tensor(g)
        opt.step()
        O.adamw_step(th, g, m, v, t, lr)
    assert np.allclose(th, p.detach().numpy(), rtol=1e-12, atol=1e-15)
