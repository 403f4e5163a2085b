"""The external force-provider path (MDPF_MODE_CALLBACK): the library calls a
Python callable for energy and forces each step, as the paper's plugin calls
its Python force module.  Checked against the FP64 oracle's trajectory, the
in-library force field (the provider wraps it) and torch autograd (a provider
that returns the energy only)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2412_18271_b300 import mdpf, synth
from tests import tiny

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_18271_b300 import build
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.init()


def _library_provider(plain):
    n = plain.n

    def prov(pos):
        E = torch.empty(1, dtype=torch.float64, device=pos.device)
        F = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
        plain.compute_device(pos.data_ptr(), E.data_ptr(), F.data_ptr(), torch.cuda.current_stream().cuda_stream)
        return E[0], F
    return prov


def test_provider_returning_forces_matches_the_library():
    s = synth.workload("mol64")
    plain = mdpf.Context(s, stepper=mdpf.MDPF_STEPPER_KERNELS)
    cb = mdpf.Context(s, mode=mdpf.MDPF_MODE_CALLBACK, provider=_library_provider(plain))
    e, f, _ = cb.compute(s.pos)
    ep, fp, _ = plain.compute(s.pos)
    assert abs(e - ep) <= 1e-6 * max(1.0, abs(ep))
    # the provider hands over FP32 forces
    assert np.abs(f - fp).max() <= 1e-6 * np.abs(fp).max()
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=0)
    cb.set_state(s.pos, v0)
    cb.step(100)
    ref = mdpf.Context(s, stepper=mdpf.MDPF_STEPPER_KERNELS)
    ref.set_state(s.pos, v0)
    ref.step(100)
    (xa, va), (xb, vb) = cb.get_state(), ref.get_state()
    assert np.abs(xa - xb).max() < 1e-5
    ua, ka = cb.trace()
    ub, kb = ref.trace()
    assert np.abs(ua - ub).max() / s.n_atoms < 1e-5 and np.abs(ka - kb).max() / s.n_atoms < 1e-5


def test_callback_trajectory_matches_the_oracle():
    # the engine side (FP64 velocity Verlet in the library) driven by a provider's FP32 forces follows
    # the FP64 oracle's trajectory within the paper's coordinate criterion (1e-3 A after 100 steps,
    # Results, "Example: Ethanol"); energies within the FP32 force field's tolerance
    s = synth.workload("mol64")
    plain = mdpf.Context(s, stepper=mdpf.MDPF_STEPPER_KERNELS)
    cb = mdpf.Context(s, mode=mdpf.MDPF_MODE_CALLBACK, provider=_library_provider(plain), dt_fs=0.5)
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=0)
    cb.set_state(s.pos, v0)
    cb.step(100)
    x, v = cb.get_state()
    xo, vo, Uo, Ko, _ = O.Plain(s).vv(s.pos, v0, 0.5, 100)
    assert np.abs(x - xo).max() < 1e-3
    assert np.abs(v - vo).max() < 1e-3 * np.abs(vo).max()
    U, K = cb.trace()
    assert np.abs(U - Uo).max() / s.n_atoms < 1e-4 and np.abs(K - Ko).max() / s.n_atoms < 1e-4


def _lj_energy(pos, sigma=3.0, eps=0.2):
    d = pos[:, None, :] - pos[None, :, :]
    n = pos.shape[0]
    iu = torch.triu_indices(n, n, 1, device=pos.device)
    r2 = (d ** 2).sum(-1)[iu[0], iu[1]]
    s6 = (sigma * sigma / r2) ** 3
    return (4.0 * eps * (s6 * s6 - s6)).sum()


def test_provider_returning_energy_gets_autograd_forces():
    rng = np.random.default_rng(4)
    g = np.arange(3) * 3.6
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + rng.normal(0, 0.1, (27, 3))
    s = tiny.isolated(27)
    cb = mdpf.Context(s, mode=mdpf.MDPF_MODE_CALLBACK, provider=_lj_energy, provider_kind="energy")
    e, f, _ = cb.compute(pos)
    x = torch.tensor(pos, dtype=torch.float64, requires_grad=True)
    et = _lj_energy(x)
    (gt,) = torch.autograd.grad(et, x)
    assert abs(e - float(et.detach())) <= 1e-9 * max(1.0, abs(float(et.detach())))
    assert np.abs(f + gt.numpy()).max() <= 1e-6 * np.abs(gt.numpy()).max()
    # NVE with the provider's forces conserves the provider's energy
    v0 = synth.velocities(s.mass, pos, 100.0, seed=1)
    cb2 = mdpf.Context(s, mode=mdpf.MDPF_MODE_CALLBACK, provider=_lj_energy, provider_kind="energy",
                       dt_fs=0.5, trace_capacity=400)
    cb2.set_state(pos, v0)
    cb2.step(400)
    U, K = cb2.trace()
    H = U + K
    assert np.abs(H - H[0]).max() < 2e-3 * np.abs(K).mean()


def test_provider_error_is_reported_and_the_context_recovers():
    s = synth.workload("mol64")
    plain = mdpf.Context(s)
    inner = _library_provider(plain)
    state = {"fail": True}

    def prov(pos):
        if state["fail"]:
            raise ValueError("provider failure")
        return inner(pos)

    cb = mdpf.Context(s, mode=mdpf.MDPF_MODE_CALLBACK, provider=prov)
    with pytest.raises(mdpf.MdpfError) as ei:
        cb.compute(s.pos)
    assert ei.value.name == "CALLBACK" and isinstance(ei.value.__cause__, ValueError)
    state["fail"] = False
    e, _, _ = cb.compute(s.pos)
    assert np.isfinite(e)
