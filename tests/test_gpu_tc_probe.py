"""The tensor-core operand path shared by the MLP kernels (st_operand32, sdesc,
idesc_bf16, mma_bf16, tmem_ld32 in csrc/tc_util.cuh), checked on its own:
operands stored by threads into the swizzled K-major layout at every 1 KB-aligned
placement class of a CTA's shared memory, one 64-wide K chunk of tcgen05 MMAs,
D read back from tensor memory, against the exact product of the same BF16
values.  The products of BF16 values are exact in FP32; only the order of the
FP32 additions differs, hence the tolerance."""
import numpy as np
import pytest

from paper_2412_18271_b300 import mdpf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KB = 1024
# (a_off, b_off): A (16 KB) and B (n x 128 bytes) below, across and above 128 KB, adjacent and far apart,
# A above B and B above A, up to the last 1 KB-aligned placement inside 225 KB
PLACEMENTS = [(0, 16 * KB), (16 * KB, 0), (48 * KB, 96 * KB), (112 * KB, 128 * KB), (127 * KB, 160 * KB),
              (128 * KB, 0), (144 * KB, 64 * KB), (192 * KB, 144 * KB), (209 * KB, 1 * KB), (3 * KB, 193 * KB)]


def _case(n, seed):
    g = torch.Generator().manual_seed(seed)
    a = torch.randn(128, 64, generator=g).to(torch.bfloat16)
    b = torch.randn(n, 64, generator=g).to(torch.bfloat16)
    ref = a.double() @ b.double().T   # exact: BF16 products and their sums fit FP64
    return a, b, ref.numpy()


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_18271_b300 import build
    build.build()
    mdpf.load()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("n", [128, 256])
@pytest.mark.parametrize("place", PLACEMENTS)
def test_tc_operand_path_at_every_placement(n, place):
    a_off, b_off = place
    if b_off + n * 128 > 225 * KB or (a_off < b_off + n * 128 and b_off < a_off + 16 * KB):
        pytest.skip("placement does not hold this n")
    a, b, ref = _case(n, 17 * n + a_off // KB)
    da, db = a.cuda().contiguous(), b.cuda().contiguous()
    dd = torch.full((128, n), float("nan"), device="cuda", dtype=torch.float32)
    st = torch.zeros(1, device="cuda", dtype=torch.int32)
    mdpf.debug_tc_probe(da.data_ptr(), db.data_ptr(), dd.data_ptr(), n, a_off, b_off, st.data_ptr())
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    d = dd.cpu().double().numpy()
    assert np.isfinite(d).all()
    # FP32 accumulation of 64 exact products: error below 64 ulp of the largest partial sum
    scale = np.abs(a.double().numpy()) @ np.abs(b.double().numpy()).T
    assert np.all(np.abs(d - ref) <= 64 * 2.0 ** -23 * scale + 1e-30)


def test_tc_probe_repeats_bit_for_bit():
    a, b, _ = _case(256, 5)
    da, db = a.cuda(), b.cuda()
    st = torch.zeros(1, device="cuda", dtype=torch.int32)
    outs = []
    for a_off, b_off in [(0, 16 * KB), (160 * KB, 16 * KB)]:
        dd = torch.empty((128, 256), device="cuda", dtype=torch.float32)
        mdpf.debug_tc_probe(da.data_ptr(), db.data_ptr(), dd.data_ptr(), 256, a_off, b_off, st.data_ptr())
        outs.append(dd.cpu())
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert torch.equal(outs[0], outs[1])
