"""GPU parity of the plain path (exclusions, bonded, all-pairs LJ + Coulomb,
velocity Verlet) against the FP64 oracle, through the C ABI.

Tolerances (FP32 forces, FP64 state):
  forces   RMSE(F_gpu - F_oracle) <= 1e-4 * RMS(F_oracle)
  energy   |E_gpu - E_oracle| / N <= 1e-5 kcal/mol/atom
  indices  exclusion and angle sets identical
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_18271_b300 import mdpf, synth
from tests import tiny

pytestmark = pytest.mark.gpu

F_RTOL = 1e-4
E_TOL_PER_ATOM = 1e-5
# Absolute floor for systems whose exact forces cancel to ~0 (e.g. a relaxed
# 3-atom molecule with every pair excluded): FP32 evaluation of a single bond
# term of size k*r ~ 4e2 kcal/mol/A carries ~1e-5 of rounding.
F_ABS_FLOOR = 1e-4
STEPPERS = [mdpf.MDPF_STEPPER_PERSISTENT, mdpf.MDPF_STEPPER_KERNELS]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_18271_b300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()
    torch.cuda.init()


def _check_forces(sys_, pos, ctx=None, f_rtol=F_RTOL, e_tol=E_TOL_PER_ATOM):
    ctx = ctx or mdpf.Context(sys_)
    e, f, terms = ctx.compute(pos)
    eo, fo, to = O.Plain(sys_).energy_forces(pos)
    n = sys_.n_atoms
    rms = np.sqrt((fo ** 2).mean()) if n > 1 else 1.0
    rmse = np.sqrt(((f - fo) ** 2).mean())
    assert rmse <= f_rtol * rms or rmse <= F_ABS_FLOOR, (rmse, rms)
    assert abs(e - eo) / n <= e_tol, (e, eo)
    for k in ("bond", "angle", "lj", "coulomb"):
        assert abs(terms[k] - to[k]) / n <= e_tol, (k, terms[k], to[k])
    return e, f, eo, fo


# ------------------------------------------------------------ exclusions / angles

@pytest.mark.parametrize("name", ["mol64", "cluster2048", "mol256"])
def test_exclusions_and_angles_bit_exact(name):
    s = synth.workload(name)
    ctx = mdpf.Context(s)
    off, idx = ctx.exclusions()
    ooff, oidx = O.exclusions(s.n_atoms, s.bonds)
    assert np.array_equal(off, ooff)
    assert np.array_equal(idx, oidx)
    assert np.array_equal(ctx.angles(), O.angles(s.n_atoms, s.bonds))


def test_exclusions_hand_tree():
    s = tiny.system(np.random.default_rng(0).normal(size=(5, 3)) * 3, [0] * 5, bonds=[(0, 1), (1, 2), (1, 3), (3, 4)])
    off, idx = mdpf.Context(s).exclusions()
    rows = [idx[off[i]:off[i + 1]].tolist() for i in range(5)]
    assert rows == [[1, 2, 3], [0, 2, 3, 4], [0, 1, 3], [0, 1, 2, 4], [1, 3]]


# ------------------------------------------------------------ force evaluation

@pytest.mark.parametrize("name", ["mol64", "cluster2048", "mol256"])
def test_compute_matches_oracle(name):
    s = synth.workload(name)
    _check_forces(s, s.pos)


@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 63, 64, 65, 95, 100, 161])
def test_compute_ragged_sizes(n):
    # molecules of n atoms: ragged last tile, diagonal-only, single atom
    s = synth.molecule(n, seed=1000 + n) if n > 1 else tiny.system([[0, 0, 0]], [2], charge=[0.3])
    e, f, eo, fo = _check_forces(s, s.pos)
    if n == 1:
        assert e == 0.0 and np.all(f == 0.0)


def test_compute_molecules_spanning_tiles():
    # 3 molecules of 23 atoms: exclusions straddle tile boundaries
    s = synth.cluster(3, 23, 12.0, seed=5)
    _check_forces(s, s.pos)


def test_compute_closed_form_pair():
    # LJ minimum: E = -eps_ij, F = 0
    sigma = (2.6, 3.1, 2.9, 3.4)
    eps = (0.07, 0.18, 0.11, 0.15)
    rmin = 2 ** (1 / 6) * 0.5 * (sigma[1] + sigma[3])
    s = tiny.system([[0, 0, 0], [0, 0, rmin]], [1, 3], sigma=sigma, eps=eps)
    e, f, _ = mdpf.Context(s).compute(s.pos)
    assert e == pytest.approx(-np.sqrt(0.18 * 0.15), rel=1e-5)
    assert np.abs(f).max() < 1e-4


def test_compute_device_matches_host():
    import torch
    s = synth.workload("mol64")
    ctx = mdpf.Context(s)
    e_h, f_h, _ = ctx.compute(s.pos)
    dpos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
    de = torch.zeros(1, dtype=torch.float64, device="cuda")
    df = torch.zeros((s.n_atoms, 3), dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    ctx.compute_device(dpos.data_ptr(), de.data_ptr(), df.data_ptr(), st.cuda_stream)
    st.synchronize()
    assert de.item() == e_h
    np.testing.assert_array_equal(df.cpu().numpy(), f_h.astype(np.float32))


def test_compute_device_single_outputs():
    # one output pointer NULL at a time: the other output is the same as with both (plain and learned mode)
    import torch
    from paper_2412_18271_b300 import model
    s = synth.workload("mol64")
    for kw in ({}, {"mode": mdpf.MDPF_MODE_LEARNED, "model": model.init_model(7).pack()}):
        ctx = mdpf.Context(s, **kw)
        dpos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
        st = torch.cuda.current_stream()
        de = torch.zeros(1, dtype=torch.float64, device="cuda")
        df = torch.zeros((s.n_atoms, 3), dtype=torch.float32, device="cuda")
        ctx.compute_device(dpos.data_ptr(), de.data_ptr(), df.data_ptr(), st.cuda_stream)
        de1 = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
        ctx.compute_device(dpos.data_ptr(), de1.data_ptr(), 0, st.cuda_stream)
        df1 = torch.full((s.n_atoms, 3), 7.0, dtype=torch.float32, device="cuda")
        ctx.compute_device(dpos.data_ptr(), 0, df1.data_ptr(), st.cuda_stream)
        st.synchronize()
        assert de1.item() == de.item()
        assert torch.equal(df1, df)
        assert ctx.counters()["status"] == 0


def test_compute_is_deterministic_and_stateless():
    s = synth.workload("cluster2048")
    ctx = mdpf.Context(s)
    a = ctx.compute(s.pos)
    b = ctx.compute(s.pos)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


# ------------------------------------------------------------ integrator

@pytest.mark.parametrize("stepper", STEPPERS)
def test_trajectory_matches_oracle_100_steps(stepper):
    # same start, 100 steps, coordinates within 1e-3 A (the paper's trajectory criterion)
    s = synth.workload("mol64")
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=0)
    ctx = mdpf.Context(s, dt_fs=0.5, stepper=stepper)
    ctx.set_state(s.pos, v0)
    ctx.step(100)
    x, v = ctx.get_state()
    U, K = ctx.trace()
    xo, vo, Uo, Ko, _ = O.Plain(s).vv(s.pos, v0, 0.5, 100)
    assert np.abs(x - xo).max() < 1e-3
    assert U.shape == (100,)
    assert np.abs(U - Uo).max() / s.n_atoms < 1e-4
    assert np.abs(K - Ko).max() / s.n_atoms < 1e-4


@pytest.mark.parametrize("stepper", STEPPERS)
def test_harmonic_diatomic_exact_discrete_solution(stepper):
    import math
    m1, m2, k, r0, dt, d0 = 1.008, 15.999, 300.0, 1.0, 0.5, 0.05
    s = tiny.system([[0, 0, 0], [r0 + d0, 0, 0]], [0, 3], bonds=[(0, 1)], r0=[r0], k=k, mass=[m1, m2])
    ctx = mdpf.Context(s, dt_fs=dt, stepper=stepper)
    mu = m1 * m2 / (m1 + m2)
    wt = math.acos(1 - 0.5 * k * O.ACC / mu * dt * dt)
    for nstep in (1, 10, 57):
        ctx.set_state(s.pos, np.zeros((2, 3)))
        ctx.step(nstep)
        x, _ = ctx.get_state()
        # FP32 bond force: relative error ~1e-6 of the displacement
        assert x[1, 0] - x[0, 0] - r0 == pytest.approx(d0 * math.cos(nstep * wt), abs=2e-6)


@pytest.mark.parametrize("stepper", STEPPERS)
def test_nve_drift_cluster2048_10k_steps(stepper):
    s = synth.workload("cluster2048")
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=synth.WORKLOAD_VELOCITY_SEED["cluster2048"])
    ctx = mdpf.Context(s, dt_fs=0.5, trace_capacity=10000, stepper=stepper)
    ctx.set_state(s.pos, v0)
    ctx.step(10000)
    U, K = ctx.trace()
    H = U + K
    assert H.shape == (10000,)
    assert np.all(np.isfinite(H))
    slope = np.polyfit(np.arange(H.size), H, 1)[0]
    drift = abs(slope) * H.size / s.n_atoms
    assert drift < DRIFT_BOUND, drift


# Bound on |least-squares slope of H| x 10k steps / N for the 2048-atom cluster
# at dt = 0.5 fs: 2e-3 kcal/mol/atom.  The FP64 oracle itself drifts by
# 3.6e-4 kcal/mol/atom over the same 10k steps from the same start (the cluster
# heats from 300 to ~970 K as the start strain relaxes).
DRIFT_BOUND = 2e-3


@pytest.mark.parametrize("stepper", STEPPERS)
def test_frames_recorded_every_k_steps(stepper):
    s = synth.workload("mol64")
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=0)
    ctx = mdpf.Context(s, record_every=10, max_frames=5, stepper=stepper)
    ctx.set_state(s.pos, v0)
    ctx.step(70)
    pos, en, frc, st = ctx.frames()
    assert st.tolist() == [30, 40, 50, 60, 70]
    x, _ = ctx.get_state()
    assert np.array_equal(pos[-1], x)
    e, f, _ = ctx.compute(x)
    assert en[-1] == pytest.approx(e, abs=1e-5)
    np.testing.assert_allclose(frc[-1], f.astype(np.float32), rtol=0, atol=1e-4)
    c = ctx.counters()
    assert c["steps"] == 70 and c["frames"] == 7


@pytest.mark.parametrize("stepper", STEPPERS)
def test_checkpoint_resume_is_bit_identical(stepper):
    s = synth.workload("mol64")
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=0)
    a = mdpf.Context(s, stepper=stepper)
    a.set_state(s.pos, v0)
    a.step(200)
    xa, va = a.get_state()
    b = mdpf.Context(s, stepper=stepper)
    b.set_state(s.pos, v0)
    b.step(120)
    xm, vm = b.get_state()
    c = mdpf.Context(s, stepper=stepper)
    c.set_state(xm, vm)
    c.step(80)
    xc, vc = c.get_state()
    assert np.array_equal(xa, xc) and np.array_equal(va, vc)


def test_steppers_agree_and_split_calls_agree():
    # one persistent launch of 150 steps == 3 launches of 50 == the kernel-sequence stepper
    s = synth.workload("cluster2048")
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=100)
    a = mdpf.Context(s, stepper=mdpf.MDPF_STEPPER_PERSISTENT)
    a.set_state(s.pos, v0)
    a.step(150)
    b = mdpf.Context(s, stepper=mdpf.MDPF_STEPPER_PERSISTENT)
    b.set_state(s.pos, v0)
    for _ in range(3):
        b.step(50)
    c = mdpf.Context(s, stepper=mdpf.MDPF_STEPPER_KERNELS)
    c.set_state(s.pos, v0)
    c.step(150)
    xa, va = a.get_state()
    xb, vb = b.get_state()
    xc, vc = c.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    # both steppers add the same FP32 terms as integers and update the state with the same
    # FP64 operations; any difference would come from instruction contraction only
    assert np.abs(xa - xc).max() < 1e-9 and np.abs(va - vc).max() < 1e-9
    Ua, Ka = a.trace()
    Uc, Kc = c.trace()
    assert np.abs(Ua - Uc).max() / s.n_atoms < 1e-7


def _hub_system():
    # two hub atoms with 30 bonded neighbours each: the tile of a hub owns 30 bonds and 435 angles, so
    # the persistent stepper evaluates most of them with the tile pair's 32x32 item, and they touch
    # four tiles
    rng = np.random.default_rng(11)
    n = 128
    pos = np.zeros((n, 3))
    far = np.array([[x, y, z] for x in range(8) for y in range(8) for z in range(4)], dtype=np.float64) * 6.0
    pos[:] = far[:n] + 40.0
    bonds = []
    for hub, nbrs, centre in ((0, list(range(1, 16)) + list(range(64, 79)), (0.0, 0.0, 0.0)),
                              (40, list(range(41, 56)) + list(range(96, 111)), (20.0, 0.0, 0.0))):
        k = np.arange(len(nbrs)) + 0.5
        phi = np.arccos(1 - 2 * k / len(nbrs))
        th = np.pi * (1 + 5 ** 0.5) * k
        dirs = np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)
        pos[hub] = centre
        pos[nbrs] = np.asarray(centre) + 1.2 * dirs + 0.02 * rng.standard_normal((len(nbrs), 3))
        bonds += [(hub, j) for j in nbrs]
    el = rng.integers(0, 4, n).astype(np.int32)
    q = rng.uniform(-0.3, 0.3, n)
    return tiny.system(pos, el, bonds=bonds, charge=q - q.mean(), angle_k=2.0, theta0_deg=90.0)


@pytest.mark.parametrize("which", ["hub", "cluster8192"])
def test_persistent_bonded_split_and_many_items(which):
    # hub: tiles whose bonded terms are shared between the self item and the diagonal 32x32 item;
    # cluster8192: more work items than warps, so every warp takes several items per step
    if which == "hub":
        s = _hub_system()
        _check_forces(s, s.pos)
        steps = 60
    else:
        s = synth.cluster(256, 32, 110.0, seed=8)
        steps = 20
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=5)
    a = mdpf.Context(s, stepper=mdpf.MDPF_STEPPER_PERSISTENT)
    a.set_state(s.pos, v0)
    a.step(steps)
    c = mdpf.Context(s, stepper=mdpf.MDPF_STEPPER_KERNELS)
    c.set_state(s.pos, v0)
    c.step(steps)
    xa, va = a.get_state()
    xc, vc = c.get_state()
    assert np.abs(xa - xc).max() < 1e-9 and np.abs(va - vc).max() < 1e-9
    Ua, _ = a.trace()
    Uc, _ = c.trace()
    # the persistent stepper sums each warp's pair energies over its items in FP32 before the FP64
    # block sums, the kernel sequence per item: the totals agree to FP32 accumulation error
    assert np.abs(Ua - Uc).max() <= 1e-7 * np.abs(Uc).max()
    if which == "hub":
        xo, vo, Uo, Ko, _ = O.Plain(s).vv(s.pos, v0, 0.5, steps)
        assert np.abs(xa - xo).max() < 1e-4
        assert abs(Ua[-1] - Uo[-1]) / s.n_atoms < 1e-5


@pytest.mark.parametrize("n_mol", [3, 37, 90, 161])
def test_persistent_matches_kernel_sequence_across_sizes(n_mol):
    # 96 to 5,152 atoms: one item per warp with blocks that straddle runs of i-tiles, a partly filled grid,
    # and several items per warp; the persistent stepper must follow the kernel sequence's trajectory
    s = synth.cluster(n_mol, 32, max(20.0, 60.0 * (n_mol / 64.0) ** (1.0 / 3.0)), seed=50 + n_mol)  # c1's density
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=9)
    a = mdpf.Context(s, stepper=mdpf.MDPF_STEPPER_PERSISTENT, energy_every=5)
    a.set_state(s.pos, v0)
    a.step(30)
    c = mdpf.Context(s, stepper=mdpf.MDPF_STEPPER_KERNELS, energy_every=5)
    c.set_state(s.pos, v0)
    c.step(30)
    xa, va = a.get_state()
    xc, vc = c.get_state()
    assert np.abs(xa - xc).max() < 1e-9 and np.abs(va - vc).max() < 1e-9
    Ua, Ka = a.trace()
    Uc, Kc = c.trace()
    assert np.abs(Ua - Uc).max() <= 1e-7 * np.abs(Uc).max()
    assert np.abs(Ka - Kc).max() <= 1e-9 * np.abs(Kc).max()


def test_persistent_is_reproducible():
    s = synth.workload("cluster2048")
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=7)
    out = []
    for _ in range(2):
        ctx = mdpf.Context(s)
        ctx.set_state(s.pos, v0)
        ctx.step(300)
        out.append(ctx.get_state() + ctx.trace())
    for u, w in zip(out[0], out[1]):
        assert np.array_equal(u, w)


@pytest.mark.parametrize("stepper", STEPPERS)
def test_energy_every_keeps_trajectory_and_thins_trace(stepper):
    s = synth.workload("mol64")
    v0 = synth.velocities(s.mass, s.pos, 300.0, seed=0)
    a = mdpf.Context(s, stepper=stepper)
    a.set_state(s.pos, v0)
    a.step(100)
    b = mdpf.Context(s, stepper=stepper, energy_every=10, record_every=20, max_frames=10)
    b.set_state(s.pos, v0)
    b.step(100)
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    Ua, Ka, sa = a.trace(with_steps=True)
    Ub, Kb, sb = b.trace(with_steps=True)
    assert sb.tolist() == list(range(10, 101, 10))
    assert np.array_equal(sa[9::10], sb)
    np.testing.assert_allclose(Ub, Ua[9::10], rtol=0, atol=1e-5)
    np.testing.assert_array_equal(Kb, Ka[9::10])
    pos, en, frc, st = b.frames()
    assert st.tolist() == [20, 40, 60, 80, 100]


def test_persistent_small_and_large_grids():
    # 1-block (64 atoms) and many-block (2048 atoms) launches both match the oracle after 30 steps
    for name in ("mol64", "cluster2048"):
        s = synth.workload(name)
        v0 = synth.velocities(s.mass, s.pos, 300.0, seed=3)
        ctx = mdpf.Context(s)
        ctx.set_state(s.pos, v0)
        ctx.step(30)
        x, v = ctx.get_state()
        xo, vo, Uo, Ko, _ = O.Plain(s).vv(s.pos, v0, 0.5, 30)
        assert np.abs(x - xo).max() < 1e-4
        U, K = ctx.trace()
        assert abs(U[-1] - Uo[-1]) / s.n_atoms < 1e-5


# ------------------------------------------------------------ failure paths (no GPU fault)

@pytest.mark.parametrize("stepper", STEPPERS)
def test_injected_status_is_reported_and_cleared(stepper):
    s = synth.workload("mol64")
    ctx = mdpf.Context(s, stepper=stepper)
    ctx.set_state(s.pos, np.zeros_like(s.pos))
    ctx.debug_set_status(mdpf.MDPF_STATUS_NONFINITE)
    with pytest.raises(mdpf.MdpfError) as ei:
        ctx.step(1)
    assert ei.value.name == "NONFINITE"
    ctx.set_state(s.pos, np.zeros_like(s.pos))
    ctx.step(5)


def test_bounded_wait_times_out_and_context_survives():
    s = synth.workload("mol64")
    ctx = mdpf.Context(s)
    ctx.set_state(s.pos, np.zeros_like(s.pos))
    rc = ctx.debug_wait_timeout(20000)
    assert rc == -6
    assert ctx.counters()["status"] & mdpf.MDPF_STATUS_TIMEOUT
    ctx.set_state(s.pos, np.zeros_like(s.pos))
    ctx.step(3)
    e, f, _ = ctx.compute(s.pos)
    assert np.isfinite(e)


def test_nonfinite_positions_are_reported():
    s = synth.workload("mol64")
    ctx = mdpf.Context(s)
    x = s.pos.copy()
    x[3] = np.nan
    with pytest.raises(mdpf.MdpfError) as ei:
        ctx.compute(x)
    assert ei.value.name == "NONFINITE"
    e, f, _ = ctx.compute(s.pos)
    assert np.isfinite(e)
