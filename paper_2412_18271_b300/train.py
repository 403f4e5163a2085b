"""Train the learned potential on plain-force-field MD data, on the device.

    python -m paper_2412_18271_b300.train [--trajectories 50] [--md-steps 10000] [--iters 20000] [--out FILE]

Steps:
  1. data: per trajectory t, the 2,048-atom cluster (64 seeded 32-atom
     molecules, seed 100 + t), Maxwell-Boltzmann velocities at 300 K, NVE
     velocity Verlet at 0.5 fs on the plain force field through libmdpf;
     a frame (positions, energy, forces) every 10 steps;
  2. per-element self energies e0 by least squares of the frame energies on
     the element counts (not trained);
  3. force-matching training: batches of 64 frames drawn from the training
     trajectories, L = energy MSE per atom + 10 x force MSE, gradient by the
     device trainer (autograd.ForceMatchingLoss), AdamW with cosine decay
     (autograd.CosineAdamW, lr 1e-3, weight decay 0.01);
  4. test force RMSE of the trained model against the plain force field on
     the held-out trajectories (learned forces through mdpf_compute);
  5. the model blob (BF16 weights) with the per-element feature ranges of the
     training data widened by 2% of their span.
Prints one JSON summary line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def generate(n_traj: int, md_steps: int, record_every: int, dev):
    import torch

    from . import mdpf, synth
    pos, ener, forc, els = [], [], [], []
    for t in range(n_traj):
        s = synth.workload("cluster2048", trajectory=t)
        v0 = synth.velocities(s.mass, s.pos, 300.0, seed=100 + t)
        nf = md_steps // record_every
        ctx = mdpf.Context(s, dt_fs=0.5, record_every=record_every, max_frames=nf, energy_every=record_every)
        ctx.set_state(s.pos, v0)
        ctx.step(md_steps)
        p, e, f, _ = ctx.frames(nf)
        ctx.close()
        pos.append(torch.tensor(p, dtype=torch.float64, device=dev))
        ener.append(torch.tensor(e, dtype=torch.float64, device=dev))
        forc.append(torch.tensor(f, dtype=torch.float32, device=dev))
        els.append(s.element.astype(np.int32))
    return pos, ener, forc, els


def fit_e0(ener, els, train):
    counts = np.array([[np.sum(els[t] == e) for e in range(4)] for t in train], dtype=np.float64)
    mean_e = np.array([float(ener[t].mean()) for t in train])
    rows = np.repeat(counts, [ener[t].numel() for t in train], axis=0)
    ys = np.concatenate([ener[t].cpu().numpy() for t in train])
    e0, *_ = np.linalg.lstsq(rows, ys, rcond=None)
    return e0, counts, mean_e


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--trajectories", type=int, default=50)
    ap.add_argument("--test-trajectories", type=int, default=5)
    ap.add_argument("--md-steps", type=int, default=10000)
    ap.add_argument("--record-every", type=int, default=10)
    ap.add_argument("--iters", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--init-seed", type=int, default=7)
    ap.add_argument("--log-every", type=int, default=500)
    ap.add_argument("--test-frames", type=int, default=20, help="frames per test trajectory")
    ap.add_argument("--out", default="")
    a = ap.parse_args(argv)

    import torch

    from . import autograd as AG
    from . import build, mdpf, model

    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    t0 = time.perf_counter()
    pos, ener, forc, els = generate(a.trajectories, a.md_steps, a.record_every, dev)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    n_test = min(a.test_trajectories, a.trajectories - 1)
    train = list(range(a.trajectories - n_test))
    test = list(range(a.trajectories - n_test, a.trajectories))
    e0, _, _ = fit_e0(ener, els, train)
    N = els[0].shape[0]
    nf = pos[0].shape[0]

    # training set on the device: frame index -> (trajectory, frame)
    pos_all = torch.stack([pos[t] for t in train])            # [T, nf, N, 3]
    f_all = torch.stack([forc[t] for t in train])
    e_all = torch.stack([ener[t] for t in train])
    el_all = torch.tensor(np.stack([els[t] for t in train]), dtype=torch.int32, device=dev)
    n_frames = len(train) * nf

    m0 = model.init_model(a.init_seed)
    m0.e0 = e0
    params = torch.tensor(model.to_flat(m0), device=dev, requires_grad=True)
    trainer = mdpf.Trainer(a.batch, N, e0, core_a=m0.core_a, core_rc=m0.core_rc)
    opt = AG.CosineAdamW([params], lr=a.lr, total_steps=a.iters)
    gen = torch.Generator(device="cpu").manual_seed(a.seed)
    log = []
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for it in range(a.iters):
        idx = torch.randint(0, n_frames, (a.batch,), generator=gen).to(dev)
        ti, fi = idx // nf, idx % nf
        bpos = pos_all[ti, fi].reshape(-1, 3).contiguous()
        bF = f_all[ti, fi].reshape(-1, 3).contiguous()
        bE = e_all[ti, fi].contiguous()
        bel = el_all[ti].reshape(-1).contiguous()
        opt.zero_grad(set_to_none=True)
        L, parts = AG.ForceMatchingLoss.apply(params, trainer, bpos, bel, bE, bF)
        L.backward()
        opt.step()
        if it % a.log_every == 0 or it == a.iters - 1:
            p = parts.cpu().numpy()
            log.append({"iter": it, "loss": float(p[0]), "energy": float(p[1]), "force": float(p[2])})
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    if trainer.status() != 0:
        raise RuntimeError("trainer reported a device status")

    lo, hi = trainer.feature_range()
    span = hi - lo
    trained = model.from_flat(params.detach().cpu().numpy(), e0, lo - 0.02 * span, hi + 0.02 * span,
                              m0.core_a, m0.core_rc)
    blob = trained.pack()
    if a.out:
        with open(a.out, "wb") as fh:
            fh.write(blob)

    # test force RMSE against the plain force field (held-out trajectories): the
    # model's own forces (a range-free copy), and how many test frames leave the range
    from . import synth
    plain_blob = model.from_flat(params.detach().cpu().numpy(), e0, core_a=m0.core_a, core_rc=m0.core_rc).pack()
    se, ss, cnt, n_eval, n_out = 0.0, 0.0, 0, 0, 0
    for t in test:
        s = synth.workload("cluster2048", trajectory=t)
        ctx = mdpf.Context(s, mode=mdpf.MDPF_MODE_LEARNED, model=plain_blob)
        rctx = mdpf.Context(s, mode=mdpf.MDPF_MODE_LEARNED, model=blob)
        sel = np.linspace(0, nf - 1, min(a.test_frames, nf)).astype(int)
        P = pos[t].cpu().numpy()
        Fp = forc[t].cpu().numpy()
        for k in sel:
            _, f, _ = ctx.compute(P[k])
            rctx.compute(P[k])
            se += float(((f - Fp[k]) ** 2).sum())
            ss += float((Fp[k].astype(np.float64) ** 2).sum())
            cnt += f.size
            n_eval += 1
        n_out += rctx.learned_counters()["fallback_steps"]
        ctx.close()
        rctx.close()
    out = {"trajectories": a.trajectories, "train_frames": n_frames, "atoms_per_frame": N, "iters": a.iters,
           "batch_frames": a.batch, "data_s": t_data, "train_s": t_train, "ms_per_iter": 1e3 * t_train / a.iters,
           "e0": [float(x) for x in e0], "log": log,
           "test_force_rmse": float(np.sqrt(se / max(cnt, 1))), "test_force_rms_plain": float(np.sqrt(ss / max(cnt, 1))),
           "test_components": cnt, "test_frames": n_eval, "test_frames_out_of_range": int(n_out)}
    print(json.dumps(out), flush=True)
    return out


if __name__ == "__main__":
    main()
