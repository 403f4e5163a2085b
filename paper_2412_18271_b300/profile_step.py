"""Run a few MD steps of a named workload with every kernel launched on its own
(no CUDA graph), for a profiler's launch list and per-kernel captures.

    python -m paper_2412_18271_b300.profile_step cluster16384 --mode learned --steps 8
    python -m paper_2412_18271_b300.profile_step cluster2048 --mode plain --steps 20
    python -m paper_2412_18271_b300.profile_step molecule9 --steps 20
    python -m paper_2412_18271_b300.profile_step mol256 --model seeded --evals 5

A workload is a named one of synth.workload, or moleculeN: one seeded N-atom
molecule (seed 9 for N = 9, else N), as the bench's small-molecule legs use.

Learned mode runs the shipped trained model without its feature ranges (every
step runs the model: no step is diverted to the plain force field), so each
step launches the neighbour check, features, MLP and adjoint once.  The first
``--setup-steps`` steps (default 2) run before profiling is switched on, so a
capture that skips them sees steady-state launches.  Prints the per-kernel
totals the library's own profiling counters recorded.

``--evals N`` makes N single evaluations through mdpf_compute_device on device
buffers (back to back on one stream, a fresh neighbour build each) instead of
the MD steps, and prints their CUDA-event time.  ``--model seeded`` uses the
seeded model (``model.init_model(7)``, as the bench's 256-atom leg) instead of
the shipped trained one.
"""
from __future__ import annotations

import argparse
import os

from . import build, mdpf, model, synth

MODEL_BLOB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "learned_c3.mdpfmlp")
MLP_KERNELS = {"tensor": mdpf.MDPF_MLP_TENSOR, "fused": mdpf.MDPF_MLP_FUSED, "simt": mdpf.MDPF_MLP_SIMT}
SLOTS = {"step": mdpf.MDPF_PROF_STEP, "stepper": mdpf.MDPF_PROF_STEPPER, "force_eval": mdpf.MDPF_PROF_NONBONDED,
         "neighbors": mdpf.MDPF_PROF_LEARN_NEIGHBORS, "features": mdpf.MDPF_PROF_LEARN_FEATURES,
         "mlp": mdpf.MDPF_PROF_LEARN_MLP, "adjoint": mdpf.MDPF_PROF_LEARN_ADJOINT,
         "fused": mdpf.MDPF_PROF_LEARN_FUSED}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("workload", nargs="?", default="cluster16384")
    ap.add_argument("--mode", choices=["learned", "plain"], default="learned")
    ap.add_argument("--mlp", choices=sorted(MLP_KERNELS), default="tensor")
    ap.add_argument("--stepper", choices=["persistent", "kernels"], default="persistent")
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--setup-steps", type=int, default=2)
    ap.add_argument("--dt-fs", type=float, default=0.5)
    ap.add_argument("--seed", type=int, default=None, help="velocity seed (default: the workload's own)")
    ap.add_argument("--evals", type=int, default=0, help="single evaluations instead of MD steps")
    ap.add_argument("--model", choices=["trained", "seeded"], default="trained")
    a = ap.parse_args(argv)

    import torch
    build.build()
    stepper = mdpf.MDPF_STEPPER_PERSISTENT if a.stepper == "persistent" else mdpf.MDPF_STEPPER_KERNELS
    torch.cuda.set_device(0)
    if a.workload.startswith("molecule"):
        na = int(a.workload[len("molecule"):])
        s = synth.molecule(na, seed=9 if na == 9 else na)
    else:
        s = synth.workload(a.workload)
    seed = a.seed if a.seed is not None else synth.WORKLOAD_VELOCITY_SEED.get(a.workload, 0)
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=seed)
    if a.mode == "learned":
        if a.model == "seeded":
            m = model.init_model(7)
        else:
            with open(MODEL_BLOB, "rb") as fh:
                m = model.Model.unpack(fh.read())
            m.lo = m.hi = None
        ctx = mdpf.Context(s, mode=mdpf.MDPF_MODE_LEARNED, model=m.pack(), dt_fs=a.dt_fs,
                           mlp_kernel=MLP_KERNELS[a.mlp], stepper=stepper)
    else:
        ctx = mdpf.Context(s, mode=mdpf.MDPF_MODE_PLAIN, dt_fs=a.dt_fs, stepper=stepper)
    ctx.set_state(s.pos, v0)
    if a.evals > 0:
        dev = torch.device("cuda")
        pos = torch.tensor(s.pos, dtype=torch.float64, device=dev).contiguous()
        E = torch.empty(1, dtype=torch.float64, device=dev)
        F = torch.empty((s.n_atoms, 3), dtype=torch.float32, device=dev)
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            ctx.compute_device(pos.data_ptr(), E.data_ptr(), F.data_ptr(), st.cuda_stream)
            st.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(a.evals):
                ctx.compute_device(pos.data_ptr(), E.data_ptr(), F.data_ptr(), st.cuda_stream)
            e1.record(st)
            st.synchronize()
        c = ctx.counters()
        print(f"{a.workload} {a.mode}: {a.evals} evaluations, {1e3 * e0.elapsed_time(e1) / a.evals:.1f} us each, "
              f"status {c['status']}")
        return 0 if c["status"] == 0 else 1
    if a.setup_steps > 0:
        ctx.step(a.setup_steps)
    ctx.set_profiling(True)
    ctx.step(a.steps)
    torch.cuda.synchronize()
    c = ctx.counters()
    print(f"{a.workload} {a.mode}: {a.steps} steps, status {c['status']}, rebuilds {c['rebuilds']}, "
          f"fallbacks {c['fallbacks']}")
    for name, slot in SLOTS.items():
        ms, n = ctx.profile(slot)
        if n:
            print(f"  {name:12s} {n:6d} launches {1e3 * ms / n:9.1f} us each")
    ctx.set_profiling(False)
    return 0 if c["status"] == 0 else 1


if __name__ == "__main__":
    raise SystemExit(main())
