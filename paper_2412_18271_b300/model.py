"""Learned-potential model: per-element MLP weights, packed for the C ABI.

Architecture (per element Z in H, C, N, O): 384 symmetry-function features
-> 256 -> 128 -> 1 with CELU(alpha = 0.1) between layers; atomic energy
E_i = W3 . celu(W2 celu(W1 G_i + b1) + b2) + b3 + e0_Z.  The weights that
define the model are the BF16 values of W1 and W2 (the GEMM operands run in
BF16 with FP32 accumulation); biases, W3, b3 are FP32 and e0 FP64.

Repulsive core: E_core = sum over pairs i < j with r < rc of A (1 - r/rc)^3 (rc/r).
The symmetry functions vanish as r -> 0 (the first radial shell sits at
0.9 A with eta = 16 A^-2), so a network on them sees two merging atoms as no
neighbour at all and cannot hold them apart; without this term, bonded H-H
pairs of the synthetic molecules fuse in hot NVE runs.  Its value, slope and
curvature vanish at rc, so it changes nothing above rc.  The default
(CORE_A = 400 kcal/mol, CORE_RC = 0.8 A) lies below every bond length the
workloads draw (1.0 to 1.5 A).

Blob layout (little endian):
  header   64 bytes: magic "MDPFMLP1", int32 version=1, n_elem=4, n_feat=384,
           h1=256, h2=128, flags (bit 0: feature ranges present, bit 1: core
           present), float64 celu_alpha, float64 core_A, float64 core_rc,
           8 bytes reserved
  per element e = 0..3:
           uint16 W1[h1][n_feat] (bf16 bits), float32 b1[h1],
           uint16 W2[h2][h1] (bf16 bits),     float32 b2[h2],
           float32 W3[h2], float32 b3, float32 pad, float64 e0
  ranges   float32 lo[4][n_feat], hi[4][n_feat]   (when flags & 1)
"""
from __future__ import annotations

import dataclasses
import struct

import numpy as np

N_ELEM, N_FEAT, H1, H2 = 4, 384, 256, 128
CELU_ALPHA = 0.1
MAGIC = b"MDPFMLP1"
HEADER = struct.Struct("<8s6iddd8x")
CORE_A = 400.0     # kcal/mol
CORE_RC = 0.8      # A


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to BF16 (round to nearest even) and return the bit patterns."""
    xf = np.ascontiguousarray(x, dtype=np.float32)
    u = xf.view(np.uint32).astype(np.uint64)
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    rounded = np.where(np.isnan(xf), 0x7FC0, rounded)
    return rounded.astype(np.uint16)


def bf16_to_f32(bits: np.ndarray) -> np.ndarray:
    return (np.asarray(bits, dtype=np.uint32) << 16).view(np.float32)


@dataclasses.dataclass
class Model:
    W1: np.ndarray    # f32 [4, 256, 384]  (BF16-representable values)
    b1: np.ndarray    # f32 [4, 256]
    W2: np.ndarray    # f32 [4, 128, 256]  (BF16-representable values)
    b2: np.ndarray    # f32 [4, 128]
    W3: np.ndarray    # f32 [4, 128]
    b3: np.ndarray    # f32 [4]
    e0: np.ndarray    # f64 [4]
    lo: np.ndarray | None = None   # f32 [4, 384] feature range of the training data
    hi: np.ndarray | None = None
    alpha: float = CELU_ALPHA
    core_a: float = 0.0            # repulsive core A (kcal/mol) and rc (A); core_rc == 0: no core
    core_rc: float = 0.0

    def pack(self) -> bytes:
        flags = (1 if self.lo is not None else 0) | (2 if self.core_rc > 0 else 0)
        core = (float(self.core_a), float(self.core_rc)) if self.core_rc > 0 else (0.0, 0.0)
        out = [HEADER.pack(MAGIC, 1, N_ELEM, N_FEAT, H1, H2, flags, float(self.alpha), *core)]
        for e in range(N_ELEM):
            out.append(bf16_bits(self.W1[e]).tobytes())
            out.append(np.asarray(self.b1[e], dtype="<f4").tobytes())
            out.append(bf16_bits(self.W2[e]).tobytes())
            out.append(np.asarray(self.b2[e], dtype="<f4").tobytes())
            out.append(np.asarray(self.W3[e], dtype="<f4").tobytes())
            out.append(struct.pack("<ffd", float(self.b3[e]), 0.0, float(self.e0[e])))
        if flags & 1:
            out.append(np.asarray(self.lo, dtype="<f4").tobytes())
            out.append(np.asarray(self.hi, dtype="<f4").tobytes())
        return b"".join(out)

    @staticmethod
    def unpack(blob: bytes) -> "Model":
        magic, ver, ne, nf, h1, h2, flags, alpha, core_a, core_rc = HEADER.unpack_from(blob, 0)
        if not flags & 2:
            core_a = core_rc = 0.0
        if magic != MAGIC or ver != 1 or (ne, nf, h1, h2) != (N_ELEM, N_FEAT, H1, H2):
            raise ValueError("not an MDPFMLP1 blob of the expected shape")
        off = HEADER.size
        W1, b1, W2, b2, W3, b3, e0 = [], [], [], [], [], [], []

        def take(dtype, count):
            nonlocal off
            a = np.frombuffer(blob, dtype=dtype, count=count, offset=off)
            off += a.nbytes
            return a

        for _ in range(N_ELEM):
            W1.append(bf16_to_f32(take("<u2", H1 * N_FEAT)).reshape(H1, N_FEAT))
            b1.append(take("<f4", H1).copy())
            W2.append(bf16_to_f32(take("<u2", H2 * H1)).reshape(H2, H1))
            b2.append(take("<f4", H2).copy())
            W3.append(take("<f4", H2).copy())
            b3v, _, e0v = struct.unpack_from("<ffd", blob, off)
            off += 16
            b3.append(b3v)
            e0.append(e0v)
        lo = hi = None
        if flags & 1:
            lo = take("<f4", N_ELEM * N_FEAT).reshape(N_ELEM, N_FEAT).copy()
            hi = take("<f4", N_ELEM * N_FEAT).reshape(N_ELEM, N_FEAT).copy()
        return Model(np.stack(W1), np.stack(b1), np.stack(W2), np.stack(b2), np.stack(W3),
                     np.array(b3, dtype=np.float32), np.array(e0), lo, hi, alpha, core_a, core_rc)

    def rounded(self) -> "Model":
        """Copy whose W1, W2 hold the BF16-rounded values (the values the blob stores)."""
        return Model.unpack(self.pack())


PARAMS_PER_ELEMENT = H1 * N_FEAT + H1 + H2 * H1 + H2 + H2 + 1   # 131,585


def to_flat(m: Model) -> np.ndarray:
    """FP32 parameter vector in the trainer's layout: per element W1, b1, W2, b2, W3, b3."""
    parts = []
    for e in range(N_ELEM):
        parts += [np.asarray(m.W1[e], np.float32).ravel(), np.asarray(m.b1[e], np.float32),
                  np.asarray(m.W2[e], np.float32).ravel(), np.asarray(m.b2[e], np.float32),
                  np.asarray(m.W3[e], np.float32), np.asarray([m.b3[e]], np.float32)]
    return np.concatenate(parts)


def from_flat(flat, e0, lo=None, hi=None, core_a: float = 0.0, core_rc: float = 0.0) -> Model:
    """Model from an FP32 parameter vector (W1, W2 keep their FP32 values; pack() rounds them to BF16)."""
    flat = np.asarray(flat, dtype=np.float32).reshape(N_ELEM, PARAMS_PER_ELEMENT)
    o1 = H1 * N_FEAT
    o2 = o1 + H1
    o3 = o2 + H2 * H1
    o4 = o3 + H2
    o5 = o4 + H2
    return Model(flat[:, :o1].reshape(N_ELEM, H1, N_FEAT).copy(), flat[:, o1:o2].copy(),
                 flat[:, o2:o3].reshape(N_ELEM, H2, H1).copy(), flat[:, o3:o4].copy(), flat[:, o4:o5].copy(),
                 flat[:, o5].copy(), np.asarray(e0, dtype=np.float64), lo, hi, CELU_ALPHA, core_a, core_rc)


def init_model(seed: int, core: bool = True) -> Model:
    """Kaiming-uniform weights U(+-sqrt(6/fan_in)), zero biases, zero e0 (seeded), with the default
    repulsive core unless core is False."""
    rng = np.random.default_rng(seed)

    def ku(shape, fan_in):
        b = np.sqrt(6.0 / fan_in)
        return rng.uniform(-b, b, size=shape).astype(np.float32)

    W1 = ku((N_ELEM, H1, N_FEAT), N_FEAT)
    W2 = ku((N_ELEM, H2, H1), H1)
    W3 = ku((N_ELEM, H2), H2)
    m = Model(W1, np.zeros((N_ELEM, H1), np.float32), W2, np.zeros((N_ELEM, H2), np.float32), W3,
              np.zeros(N_ELEM, np.float32), np.zeros(N_ELEM))
    if core:
        m.core_a, m.core_rc = CORE_A, CORE_RC
    return m.rounded()
