"""Pins of the oracle's learned path (neighbour list, symmetry-function features
and their derivatives, per-element MLP and its input gradient) against facts
that do not come from the oracle: an independent FP32 brute force, closed-form
values at special geometries, the layout of feature blocks, finite
differences, conservation laws, symmetry, and PyTorch's own dense layers and
autograd in FP64."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2412_18271_b300 import model, synth

RC_R, RC_A = 5.2, 3.5


def fc(r, rc):
    return 0.5 * math.cos(math.pi * r / rc) + 0.5 if r < rc else 0.0


# ------------------------------------------------------------ neighbour list

def _numpy_neighbors(x32, rc):
    # independent FP32 evaluation of the same predicate (numpy rounds each op to float32)
    rc2 = np.float32(rc * rc)
    d = x32[None, :, :] - x32[:, None, :]
    d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    np.fill_diagonal(d2, np.float32(np.inf))
    return [np.nonzero(d2[i] < rc2)[0] for i in range(x32.shape[0])]


@pytest.mark.parametrize("name", ["mol64", "mol256"])
def test_neighbors_match_fp32_brute_force(name):
    x = synth.workload(name).pos.astype(np.float32)
    a = O.neighbors(x, 6.2)
    b = _numpy_neighbors(x, 6.2)
    assert all(np.array_equal(u, v) for u, v in zip(a, b))


def test_neighbors_strict_inequality_at_the_cutoff():
    rc2 = np.float32(6.2 * 6.2)
    # find an FP32 separation whose FP32 square equals rc2 exactly, if one exists; otherwise the
    # largest one below it: the pair at that separation must be excluded / included accordingly
    dx = np.float32(math.sqrt(float(rc2)))
    for _ in range(8):
        if dx * dx >= rc2:
            dx = np.nextafter(dx, np.float32(0))
        else:
            break
    inside = dx
    outside = np.nextafter(dx, np.float32(10))
    assert inside * inside < rc2 <= outside * outside
    x = np.array([[0, 0, 0], [inside, 0, 0], [0, outside, 0]], dtype=np.float32)
    nb = O.neighbors(x, 6.2)
    assert nb[0].tolist() == [1]
    assert nb[1].tolist() == [0, 2] or 2 not in nb[0]


# ------------------------------------------------------------ features

@pytest.mark.parametrize("ej", [0, 1, 2, 3])
def test_radial_one_pair_closed_form_and_block(ej):
    r = 2.37
    G = O.features(np.array([1, ej]), np.array([[0, 0, 0], [r, 0, 0.0]]))
    for k in range(16):
        rk = 0.9 + k * (RC_R - 0.9) / 16
        expect = math.exp(-16.0 * (r - rk) ** 2) * fc(r, RC_R)
        assert G[0, 16 * ej + k] == pytest.approx(expect, rel=1e-12, abs=1e-300)
    other = [f for f in range(64) if f // 16 != ej]
    assert np.all(G[0, other] == 0) and np.all(G[0, 64:] == 0)


def test_radial_at_shell_centre_and_cutoff():
    # at r = R_k the k-th Gaussian is 1, so the feature equals fc(R_k); at and beyond rc it is 0
    k = 5
    rk = 0.9 + k * (RC_R - 0.9) / 16
    G = O.features(np.array([0, 0]), np.array([[0, 0, 0], [0, 0, rk]]))
    assert G[0, k] == pytest.approx(fc(rk, RC_R), rel=1e-14)
    assert fc(RC_R / 2, RC_R) == pytest.approx(0.5)
    for r in (RC_R, RC_R + 1e-9, 7.0):
        G = O.features(np.array([0, 0]), np.array([[0, 0, 0], [r, 0, 0]]))
        assert np.all(G == 0)
    # continuity: just inside the cutoff the features are ~0
    G = O.features(np.array([0, 0]), np.array([[0, 0, 0], [RC_R - 1e-6, 0, 0]]))
    assert np.abs(G).max() < 1e-10


PAIRS = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (0, 3): 3, (1, 1): 4, (1, 2): 5, (1, 3): 6, (2, 2): 7, (2, 3): 8,
         (3, 3): 9}


@pytest.mark.parametrize("zj,zk", sorted(PAIRS))
def test_angular_peak_value_block_and_index(zj, zk):
    # i at the origin, j and k at r = R_m with 0.95 cos(theta_ijk) = cos(theta_p): the angular
    # factor 2^(1-zeta) (1 + cos 0)^zeta = 2 and the radial factor is 1, so G = 2 fc(R_m)^2
    m, p = 2, 3
    rm = 0.9 + m * (RC_A - 0.9) / 4
    thp = (2 * p + 1) * math.pi / 16
    th = math.acos(math.cos(thp) / 0.95)
    x = np.array([[0, 0, 0], [rm, 0, 0], [rm * math.cos(th), rm * math.sin(th), 0]])
    G = O.features(np.array([1, zj, zk]), x)
    P = PAIRS[(min(zj, zk), max(zj, zk))]
    f = 64 + 32 * P + 8 * m + p
    assert G[0, f] == pytest.approx(2 * fc(rm, RC_A) ** 2, rel=1e-12)
    # nothing of atom 0's angular features lives outside block P
    blk = np.zeros(320, dtype=bool)
    blk[32 * P:32 * P + 32] = True
    assert np.all(G[0, 64:][~blk] == 0)
    # the peak is the maximum over the 8 angular sections of shell m
    row = G[0, 64 + 32 * P + 8 * m: 64 + 32 * P + 8 * m + 8]
    assert int(np.argmax(row)) == p


def test_angular_symmetric_in_j_k_and_zero_beyond_cutoff():
    x = np.array([[0, 0, 0], [1.3, 0.2, 0.1], [-0.4, 1.5, 0.3]])
    a = O.features(np.array([0, 1, 3]), x)
    b = O.features(np.array([0, 3, 1]), x[[0, 2, 1]])
    np.testing.assert_allclose(a[0], b[0], rtol=1e-13, atol=1e-15)
    x2 = x.copy()
    x2[2] *= 3.6 / np.linalg.norm(x2[2])   # k beyond the angular cutoff
    g = O.features(np.array([0, 1, 3]), x2)
    assert np.all(g[0, 64:] == 0) and np.any(g[0, :64] != 0)


@pytest.fixture(scope="module")
def mol():
    s = synth.molecule(40, seed=11)
    return s


def test_feature_jvp_matches_finite_differences(mol):
    rng = np.random.default_rng(1)
    u = rng.normal(size=mol.pos.shape)
    h = 1e-5
    fd = (O.features(mol.element, mol.pos + h * u) - O.features(mol.element, mol.pos - h * u)) / (2 * h)
    jv = O.feature_jvp(mol.element, mol.pos, u)
    assert np.abs(fd - jv).max() < 1e-6 * max(1.0, np.abs(jv).max())


def test_feature_forces_are_transpose_of_jvp(mol):
    # <F(w), u> = -<w, J u> for any w, u (adjoint identity between the two analytic derivatives)
    rng = np.random.default_rng(2)
    w = rng.normal(size=(mol.n_atoms, 384))
    u = rng.normal(size=mol.pos.shape)
    F = O.feature_forces(mol.element, mol.pos, w)
    Jv = O.feature_jvp(mol.element, mol.pos, u)
    assert (F * u).sum() == pytest.approx(-(w * Jv).sum(), rel=1e-10)


def _rotation(seed):
    q = np.random.default_rng(seed).normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a*a+b*b-c*c-d*d, 2*(b*c-a*d), 2*(b*d+a*c)],
                     [2*(b*c+a*d), a*a-b*b+c*c-d*d, 2*(c*d-a*b)],
                     [2*(b*d-a*c), 2*(c*d+a*b), a*a-b*b-c*c+d*d]])


def test_features_invariant(mol):
    G = O.features(mol.element, mol.pos)
    R = _rotation(4)
    G2 = O.features(mol.element, mol.pos @ R.T + np.array([3.0, -1.0, 7.0]))
    np.testing.assert_allclose(G2, G, rtol=1e-10, atol=1e-12)
    perm = np.random.default_rng(5).permutation(mol.n_atoms)
    G3 = O.features(mol.element[perm], mol.pos[perm])
    np.testing.assert_allclose(G3, G[perm], rtol=1e-10, atol=1e-12)


# ------------------------------------------------------------ MLP

@pytest.fixture(scope="module")
def mdl():
    m = model.init_model(3)
    rng = np.random.default_rng(9)
    m.b1[:] = rng.normal(scale=0.1, size=m.b1.shape)
    m.b2[:] = rng.normal(scale=0.1, size=m.b2.shape)
    m.b3[:] = rng.normal(size=4)
    m.e0[:] = rng.normal(size=4)
    return m


def test_mlp_matches_torch_dense_layers(mdl, mol):
    G = O.features(mol.element, mol.pos)
    E, Ei, dG = O.Learned(mdl).mlp(mol.element, G)
    Gt = torch.tensor(G, dtype=torch.float64, requires_grad=True)
    Et = torch.zeros(mol.n_atoms, dtype=torch.float64)
    for e in range(4):
        idx = np.nonzero(mol.element == e)[0]
        if idx.size == 0:
            continue
        x = Gt[idx]
        h = torch.nn.functional.celu(torch.nn.functional.linear(
            x, torch.tensor(mdl.W1[e], dtype=torch.float64), torch.tensor(mdl.b1[e], dtype=torch.float64)), 0.1)
        h = torch.nn.functional.celu(torch.nn.functional.linear(
            h, torch.tensor(mdl.W2[e], dtype=torch.float64), torch.tensor(mdl.b2[e], dtype=torch.float64)), 0.1)
        out = torch.nn.functional.linear(h, torch.tensor(mdl.W3[e][None, :], dtype=torch.float64),
                                         torch.tensor([float(mdl.b3[e])], dtype=torch.float64))[:, 0]
        Et = Et.index_put((torch.tensor(idx),), out + float(mdl.e0[e]))
    np.testing.assert_allclose(Ei, Et.detach().numpy(), rtol=1e-12, atol=1e-12)
    (g,) = torch.autograd.grad(Et.sum(), Gt)
    # torch's CELU backward rebuilds exp(x/alpha) from the layer output, which costs relative
    # precision for very negative x; 1e-7 of the gradient scale is far below any structural error
    np.testing.assert_allclose(dG, g.numpy(), rtol=1e-6, atol=1e-7 * np.abs(g.numpy()).max())
    assert E == pytest.approx(Et.sum().item(), rel=1e-12)


def test_learned_forces_match_finite_differences(mdl, mol):
    L = O.Learned(mdl)
    E, F, _ = L.energy_forces(mol.element, mol.pos)
    # the steep features (zeta = 32, eta = 16) give a large third derivative: the O(h^2) central
    # difference error is ~4e-5 at h = 1e-4 A and ~1e-7 at h = 1e-5 A
    h = 1e-5
    rng = np.random.default_rng(0)
    for a in rng.choice(mol.n_atoms, 8, replace=False):
        for c in range(3):
            xp = mol.pos.copy(); xp[a, c] += h
            xm = mol.pos.copy(); xm[a, c] -= h
            fd = -(L.energy_forces(mol.element, xp)[0] - L.energy_forces(mol.element, xm)[0]) / (2 * h)
            assert fd == pytest.approx(F[a, c], rel=1e-5, abs=1e-7)


def test_learned_net_force_torque_and_invariance(mdl, mol):
    L = O.Learned(mdl)
    E, F, _ = L.energy_forces(mol.element, mol.pos)
    scale = np.abs(F).sum()
    assert np.abs(F.sum(axis=0)).max() < 1e-10 * scale
    c = mol.pos.mean(axis=0)
    assert np.abs(np.cross(mol.pos - c, F).sum(axis=0)).max() < 1e-9 * scale * np.abs(mol.pos - c).max()
    R = _rotation(8)
    E2, F2, _ = L.energy_forces(mol.element, mol.pos @ R.T - 2.0)
    assert E2 == pytest.approx(E, rel=1e-11)
    np.testing.assert_allclose(F2, F @ R.T, atol=1e-9 * np.abs(F).max())


def test_model_blob_roundtrip(mdl):
    blob = mdl.pack()
    back = model.Model.unpack(blob)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3", "e0"):
        np.testing.assert_array_equal(getattr(back, name), getattr(mdl, name))
    # bf16 rounding is round-to-nearest-even on the bit pattern
    x = np.array([1.0, 1.00390625, 1.005859375, -3.0e-3, 65504.0], dtype=np.float32)
    r = model.bf16_to_f32(model.bf16_bits(x))
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == np.float32(1.0078125)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8)


def test_flat_parameter_layout_roundtrip(mdl):
    flat = model.to_flat(mdl)
    assert flat.shape == (4 * model.PARAMS_PER_ELEMENT,) and flat.dtype == np.float32
    assert 4 * model.PARAMS_PER_ELEMENT == 526340
    back = model.from_flat(flat, mdl.e0)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        assert np.array_equal(np.asarray(getattr(back, k), np.float32), np.asarray(getattr(mdl, k), np.float32)), k
    # element 2's W2[5][7] sits at 2 * P + 256*384 + 256 + 5*256 + 7
    P = model.PARAMS_PER_ELEMENT
    assert flat[2 * P + 256 * 384 + 256 + 5 * 256 + 7] == np.float32(mdl.W2[2][5][7])


# ------------------------------------------------------------ repulsive core

CORE_A, CORE_RC = 400.0, 0.8


def _dimer(r):
    return np.array([[0.0, 0.0, 0.0], [0.3 * r, -0.4 * r, math.sqrt(1 - 0.25) * r]])


@pytest.mark.parametrize("r,e_hand", [(0.4, 100.0), (0.2, 675.0), (0.6, 25.0 / 3.0), (0.8, 0.0), (1.3, 0.0)])
def test_core_dimer_values_by_hand(r, e_hand):
    # A (1 - x)^3 / x at x = 1/2: 400 / 8 * 2 = 100;  x = 1/4: 400 * 27/64 * 4 = 675;
    # x = 3/4: 400 / 64 * 4/3 = 25/3;  zero from rc on
    e, f = O.core_energy_forces(_dimer(r), CORE_A, CORE_RC)
    assert e == pytest.approx(e_hand, rel=1e-12, abs=1e-12)
    assert np.abs(f.sum(axis=0)).max() < 1e-10


def test_core_vanishes_smoothly_at_rc():
    # a cubic contact: E(rc - d) ~ A (d / rc)^3 (a quadratic or linear one would be 10^2 / 10^4 x larger)
    d = 1e-3
    e, f = O.core_energy_forces(_dimer(CORE_RC - d), CORE_A, CORE_RC)
    assert e == pytest.approx(CORE_A * (d / CORE_RC) ** 3, rel=5e-3)
    # and its force ~ 3 A d^2 / rc^3, so it vanishes quadratically
    assert np.linalg.norm(f[0]) == pytest.approx(3 * CORE_A * d * d / CORE_RC ** 3, rel=1e-2)


def test_core_repels_and_matches_finite_differences():
    rng = np.random.default_rng(3)
    x = np.array([[0, 0, 0], [0.5, 0.1, 0], [0.2, 0.55, 0.1], [1.5, 0.2, 0.3], [0.1, 0.1, 0.7]], dtype=np.float64)
    x += rng.normal(scale=0.01, size=x.shape)
    e, f = O.core_energy_forces(x, CORE_A, CORE_RC)
    h = 1e-6
    fd = np.zeros_like(x)
    for a in range(x.shape[0]):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[a, c] += h
            xm[a, c] -= h
            fd[a, c] = -(O.core_energy_forces(xp, CORE_A, CORE_RC)[0] - O.core_energy_forces(xm, CORE_A, CORE_RC)[0]) / (2 * h)
    assert np.abs(f - fd).max() < 1e-5 * np.abs(fd).max()
    assert np.abs(f.sum(axis=0)).max() < 1e-9 * np.abs(f).max()
    assert np.abs(np.cross(x, f).sum(axis=0)).max() < 1e-9 * np.abs(f).max()
    # repulsive: the force on atom 1 of a close dimer points away from atom 0
    _, fd2 = O.core_energy_forces(_dimer(0.5), CORE_A, CORE_RC)
    assert float(np.dot(fd2[1], _dimer(0.5)[1])) > 0


def test_learned_energy_includes_the_core():
    s = synth.molecule(5, seed=3)
    x = s.pos.copy()
    x[1] = x[0] + np.array([0.45, 0.0, 0.0])   # one pair inside the core radius
    m_on = model.init_model(7)
    m_off = model.init_model(7, core=False)
    e_on, f_on, _ = O.Learned(m_on).energy_forces(s.element, x)
    e_off, f_off, _ = O.Learned(m_off).energy_forces(s.element, x)
    ec, fc_ = O.core_energy_forces(x, model.CORE_A, model.CORE_RC)
    assert ec > 10.0
    assert e_on - e_off == pytest.approx(ec, rel=1e-12)
    assert np.abs((f_on - f_off) - fc_).max() < 1e-9 * np.abs(fc_).max()
    assert model.Model.unpack(m_on.pack()).core_rc == model.CORE_RC
