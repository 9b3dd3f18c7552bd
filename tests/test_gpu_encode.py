"""GPU parity for the device encoder: byte-exact against the oracle's encoder
(Sec. 1, Table 1; differential coding with x_{-1} = prev), through the C ABI.
Expected bytes come only from the oracle; nothing expected comes from the
CUDA path.  Also checks the byte count, the bytes past it (untouched), the
unaligned-input path, and the round trip through the GPU decoder."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1503_07387_gb300 import inputs, vbyte

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

TILE = 6144   # values per encoder tile


def all_lengths(n, seed):
    """Values of every code length 1..5, equally often."""
    rng = np.random.default_rng(seed)
    bits = rng.integers(1, 33, n)
    return (rng.integers(0, 1 << 64, n, dtype=np.uint64) >> (64 - bits).astype(np.uint64)).astype(np.uint32)


def run_encode(vals, delta=False, prev=0, elem_off=0):
    """Encode on the GPU with the input `elem_off` uint32 into a buffer; the
    output buffer is pre-filled so bytes past the count can be checked."""
    vals = np.ascontiguousarray(vals, dtype=np.uint32)
    n = vals.size
    buf = torch.zeros(elem_off + n + 4, dtype=torch.int32, device="cuda")
    if n:
        buf[elem_off:elem_off + n] = torch.from_numpy(vals.view(np.int32)).cuda()
    d_in = buf[elem_off:elem_off + n]
    out = torch.full((5 * n + 64,), 0xEE, dtype=torch.uint8, device="cuda")
    nb = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    assert vbyte.get_status() == 0
    vbyte.encode_device(d_in, delta=delta, prev=prev, out=out, nbytes=nb)
    st = vbyte.get_status()
    k = int(nb.item())
    o = out.cpu().numpy()
    assert np.all(o[k:] == 0xEE), "bytes past the count were written"
    return o[:k], st


def expect(vals, delta=False, prev=0):
    return oracle.encode_delta(vals, prev) if delta else oracle.encode(vals)


@pytest.mark.parametrize("n", [0, 1, 7, 8, 9, TILE - 1, TILE, TILE + 1, 3 * TILE + 5, 100_003])
@pytest.mark.parametrize("delta", [False, True])
def test_parity_sizes(n, delta):
    vals = all_lengths(n, seed=n + 11)
    if delta:
        vals = np.sort(vals)
    got, st = run_encode(vals, delta=delta, prev=3)
    assert st == 0
    assert np.array_equal(got, expect(vals, delta, 3))


@pytest.mark.parametrize("elem_off", [1, 2, 3])
def test_unaligned_input(elem_off):
    vals = all_lengths(5 * TILE + 17, seed=elem_off)
    got, st = run_encode(vals, elem_off=elem_off)
    assert st == 0
    assert np.array_equal(got, expect(vals))


def test_length_boundaries():
    edges = []
    for k in range(1, 5):
        edges += [(1 << (7 * k)) - 1, 1 << (7 * k)]
    vals = np.array(edges * 300 + [0, 1, 0xFFFFFFFF, 0x0FFFFFFF, 0x10000000], dtype=np.uint32)
    got, st = run_encode(vals)
    assert st == 0
    assert np.array_equal(got, expect(vals))
    # Table 1's worked values, independently of the oracle's encoder
    for v, want in [(0, [0x00]), (127, [0x7F]), (128, [0x80, 0x01]), (16383, [0xFF, 0x7F]),
                    (16384, [0x80, 0x80, 0x01]), (0xFFFFFFFF, [0xFF, 0xFF, 0xFF, 0xFF, 0x0F])]:
        g, _ = run_encode(np.array([v], dtype=np.uint32))
        assert list(g) == want, v


def test_delta_wraps_and_prev():
    rng = np.random.default_rng(5)
    vals = rng.integers(0, 1 << 32, 4 * TILE + 3, dtype=np.uint64).astype(np.uint32)   # gaps wrap mod 2^32
    for prev in (0, 0xFFFFFFFF, 12345):
        got, st = run_encode(vals, delta=True, prev=prev)
        assert st == 0
        assert np.array_equal(got, expect(vals, True, prev))


@pytest.mark.parametrize("delta", [False, True])
def test_full_size_round_trip(delta):
    """The 2^26-value geometric stream: bytes equal to the oracle's, and the
    GPU decoder gives the values back."""
    gaps = inputs.geometric_gaps(1 << 26, seed=0)
    vals = np.cumsum(gaps.astype(np.uint64)).astype(np.uint32) if delta else gaps
    got, st = run_encode(vals, delta=delta, prev=0)
    assert st == 0
    want = expect(vals, delta, 0)
    assert got.size == want.size and np.array_equal(got, want)
    d = torch.from_numpy(got).cuda()
    back = vbyte.decode_delta(d, vals.size) if delta else vbyte.decode(d, vals.size)
    assert vbyte.get_status() == 0
    assert np.array_equal(back.cpu().numpy().view(np.uint32), vals)


def test_rejects_bad_arguments():
    lib = vbyte.load()
    x = torch.zeros(16, dtype=torch.int32, device="cuda")
    out = torch.empty(80, dtype=torch.uint8, device="cuda")
    nb = torch.empty(1, dtype=torch.int64, device="cuda")
    # a misaligned input pointer is refused before any launch
    rc = lib.vbyte_encode_device(ctypes.c_void_p(x.data_ptr() + 2), 4, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(nb.data_ptr()), None)
    assert rc == 1
    rc = lib.vbyte_encode_device(ctypes.c_void_p(x.data_ptr()), 4, ctypes.c_void_p(out.data_ptr()), None, None)
    assert rc == 1
