"""The entry point that allocates no device memory, checked against the
regular evaluation.

It exists for callers that cannot call cudaMalloc at the moment they need
forces (an engine calling its force provider inside its step loop and memory
pool, or code that must avoid the synchronisation of cudaMalloc/cudaFree);
they pass their own device buffers and the library works in a fixed array of
its own.  This file is collected last so that a run stopping at the first
failure has run every other test first; it creates everything it needs, so it
also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2412_18271_b300 import mdpf, synth

pytestmark = pytest.mark.gpu

F_RTOL = 1e-4          # the FP32 force tolerance of the other GPU tests (relative to RMS force)
E_TOL_PER_ATOM = 1e-5  # kcal/mol/atom
# The two paths add the FP32 pair energies in different groupings (Newton-pair tiles here, per-row tasks in the
# context's kernels), so the difference also scales with the size of the sum: one FP32 ulp of the total on top.
E_RTOL = 1e-7


def _e_ok(e, e_ref, n):
    return abs(e - e_ref) <= E_TOL_PER_ATOM * n + E_RTOL * abs(e_ref)


def _unbonded(n_mol, per_mol, radius, seed):
    # atoms of a seeded cluster with the bonds removed: every pair interacts
    s = synth.cluster(n_mol, per_mol, radius, seed=seed)
    s.bonds = np.zeros((0, 2), dtype=np.int32)
    s.bond_r0 = np.zeros(0)
    s.bond_k = np.zeros(0)
    return s


def _reference(ctx, dpos, n, torch):
    de = torch.zeros(1, dtype=torch.float64, device="cuda")
    df = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    ctx.compute_device(dpos.data_ptr(), de.data_ptr(), df.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return de.item(), df.cpu().numpy()


def test_noalloc_matches_compute_on_two_calls_in_a_row():
    import torch
    from paper_2412_18271_b300 import build
    build.build()
    s = _unbonded(8, 32, 25.0, seed=31)          # 256 atoms
    n = s.n_atoms
    ctx = mdpf.Context(s)
    del_ = torch.tensor(s.element, dtype=torch.int32, device="cuda")
    dq = torch.tensor(s.charge, dtype=torch.float64, device="cuda")
    de = torch.zeros(1, dtype=torch.float64, device="cuda")
    df = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(0)
    for call in range(2):
        pos = s.pos + (0.0 if call == 0 else rng.normal(scale=0.05, size=s.pos.shape))
        dpos = torch.tensor(pos, dtype=torch.float64, device="cuda")
        e_ref, f_ref = _reference(ctx, dpos, n, torch)
        df.fill_(123.0)
        de.fill_(123.0)
        mdpf.pairs_noalloc(n, dpos.data_ptr(), del_.data_ptr(), dq.data_ptr(), s.lj_sigma, s.lj_eps, 0.0,
                           de.data_ptr(), df.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        e, f = de.item(), df.cpu().numpy()
        rms = np.sqrt((f_ref.astype(np.float64) ** 2).mean())
        assert np.sqrt(((f - f_ref) ** 2).mean()) <= F_RTOL * rms, call
        assert _e_ok(e, e_ref, n), (call, e, e_ref)


def test_noalloc_largest_size_and_rejects_larger():
    import torch
    s = _unbonded(64, 32, 60.0, seed=100)        # 2048 atoms: the largest accepted size
    n = s.n_atoms
    ctx = mdpf.Context(s)
    dpos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
    del_ = torch.tensor(s.element, dtype=torch.int32, device="cuda")
    dq = torch.tensor(s.charge, dtype=torch.float64, device="cuda")
    de = torch.zeros(1, dtype=torch.float64, device="cuda")
    df = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    e_ref, f_ref = _reference(ctx, dpos, n, torch)
    mdpf.pairs_noalloc(n, dpos.data_ptr(), del_.data_ptr(), dq.data_ptr(), s.lj_sigma, s.lj_eps, 0.0,
                       de.data_ptr(), df.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    f = df.cpu().numpy()
    rms = np.sqrt((f_ref.astype(np.float64) ** 2).mean())
    assert np.sqrt(((f - f_ref) ** 2).mean()) <= F_RTOL * rms
    assert _e_ok(de.item(), e_ref, n)
    with pytest.raises(mdpf.MdpfError) as ei:
        mdpf.pairs_noalloc(n + 1, dpos.data_ptr(), del_.data_ptr(), dq.data_ptr(), s.lj_sigma, s.lj_eps, 0.0,
                           de.data_ptr(), df.data_ptr(), 0)
    assert ei.value.name == "INVALID_ARG" and "2048" in str(ei.value)


@pytest.mark.parametrize("n", [1, 33, 100, 2047])
def test_noalloc_ragged_sizes_match_the_oracle(n):
    # sizes that are not multiples of the 64-atom padding, so the padding atoms the kernel adds take part;
    # an explicit Coulomb constant; against the FP64 oracle of the same unbonded system
    import torch
    from oracle import oracle as O
    from tests import tiny
    src = _unbonded(64, 32, 60.0, seed=100)
    # n atoms on a jittered 3.5 A grid (a dense gas: every pair interacts, no two atoms overlap)
    rng = np.random.default_rng(n)
    g = np.arange(13) * 3.5
    grid = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)[:n]
    pos = grid + rng.normal(scale=0.2, size=grid.shape)
    s = tiny.system(pos, src.element[:n], charge=src.charge[:n], sigma=src.lj_sigma, eps=src.lj_eps)
    ke = 300.0
    eo, fo, _ = O.Plain(s, coulomb_k=ke).energy_forces(s.pos)
    dpos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
    del_ = torch.tensor(s.element, dtype=torch.int32, device="cuda")
    dq = torch.tensor(s.charge, dtype=torch.float64, device="cuda")
    de = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    df = torch.full((n, 3), 7.0, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    mdpf.pairs_noalloc(n, dpos.data_ptr(), del_.data_ptr(), dq.data_ptr(), s.lj_sigma, s.lj_eps, ke,
                       de.data_ptr(), df.data_ptr(), stream)
    torch.cuda.synchronize()
    f = df.cpu().numpy().astype(np.float64)
    rms = np.sqrt((fo ** 2).mean())
    assert np.sqrt(((f - fo) ** 2).mean()) <= F_RTOL * rms + (1e-12 if n == 1 else 0.0)
    assert abs(de.item() - eo) / n <= E_TOL_PER_ATOM
    # either output may be omitted: each alone equals the full call's
    df2 = torch.full((n, 3), 7.0, dtype=torch.float32, device="cuda")
    mdpf.pairs_noalloc(n, dpos.data_ptr(), del_.data_ptr(), dq.data_ptr(), s.lj_sigma, s.lj_eps, ke,
                       0, df2.data_ptr(), stream)
    de2 = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    mdpf.pairs_noalloc(n, dpos.data_ptr(), del_.data_ptr(), dq.data_ptr(), s.lj_sigma, s.lj_eps, ke,
                       de2.data_ptr(), 0, stream)
    torch.cuda.synchronize()
    assert np.array_equal(df2.cpu().numpy(), df.cpu().numpy())
    assert de2.item() == de.item()
