"""GPU parity for the gaps-minus-one differential variant (Sec. 1: x_1 - x_0,
x_2 - x_1 - 1, ...): the decoder and the device encoder against the oracle,
bit for bit, through the C ABI.  Expected values and bytes come only from
the oracle (or from the ids the streams were built from)."""
import numpy as np
import pytest

import oracle
from paper_1503_07387_gb300 import inputs, vbyte

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, params=[1, 2, 3, 4], ids=["onepass", "twopass", "split", "split_table"])
def kernel(request):
    """Every test runs on each single-stream kernel: the single pass with a
    decoupled look-back, count-then-decode in one launch, and the split
    count / scan / decode launches (4: the table-driven setting, which this
    variant must ignore)."""
    vbyte.debug_force_passes(request.param)
    yield request.param
    vbyte.debug_force_passes(0)

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

MASK32 = (1 << 32) - 1


def ids_from_gaps(G, prev):
    """x_0 = prev + G_0, x_i = x_{i-1} + 1 + G_i (mod 2^32)."""
    G = np.asarray(G, dtype=np.uint64)
    return ((prev + np.cumsum(G) + np.arange(G.size, dtype=np.uint64)) & MASK32).astype(np.uint32)


def decode_gpu(data, n, prev):
    d = torch.from_numpy(np.ascontiguousarray(data, dtype=np.uint8)).cuda()
    guard = torch.full((n + 64,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    out = guard[32:32 + n]
    assert vbyte.get_status() == 0
    vbyte.decode_delta_m1(d, n, prev=prev, out=out)
    st = vbyte.get_status()
    g = guard.cpu().numpy().view(np.uint32)
    assert np.all(g[:32] == 0x5A5A5A5A) and np.all(g[32 + n:] == 0x5A5A5A5A), "writes outside the output"
    return g[32:32 + n].copy(), st


GAPS = {
    "one_byte": lambda n, s: inputs.geometric_gaps(n, seed=s) - 1,          # almost all one-byte codes
    "one_two": lambda n, s: inputs.uniform_gaps(n, lo=0, hi=300, seed=s),   # one and two bytes
    "long": lambda n, s: inputs.full_range(n, seed=s),                       # mostly five bytes, wrapping
}


@pytest.mark.parametrize("kind", sorted(GAPS))
@pytest.mark.parametrize("n", [1, 511, 512, 513, 4095, 70_001, 1_000_003])
def test_decode_parity(kind, n):
    G = GAPS[kind](n, n % 97).astype(np.uint32)
    prev = 1000 + n
    x = ids_from_gaps(G, prev)
    data = oracle.encode_delta_m1(x, prev=prev)
    assert np.array_equal(oracle.decode(data), G)   # the stored integers are the chosen gaps
    got, st = decode_gpu(data, n, prev)
    assert st == 0
    assert np.array_equal(got, oracle.decode_delta_m1(data, n, prev=prev))
    assert np.array_equal(got, x)


def test_decode_empty_and_count_mismatch():
    got, st = decode_gpu(np.zeros(0, np.uint8), 0, 7)
    assert got.size == 0 and st == 0
    data = oracle.encode_delta_m1(np.arange(10, dtype=np.uint32))
    got, st = decode_gpu(data, 9, 0)    # one value fewer than the stream holds
    assert st == oracle.validate(data, 9)
    assert np.array_equal(got, oracle.decode_delta_m1(data, prev=0)[:9])


def test_decode_full_size_sampled():
    """2^26 values (a mix of all code lengths) checked at sampled ranks plus
    the end, against the ids the stream was built from."""
    n = 1 << 26
    rng = np.random.default_rng(3)
    G = (rng.integers(0, 1 << 63, n, dtype=np.uint64) >> rng.integers(32, 64, n).astype(np.uint64)).astype(np.uint32)
    x = ids_from_gaps(G, 5)
    data = vbyte.encode_delta_m1(x, prev=5)          # the library's host encoder; checked below
    idx = np.unique(np.concatenate([rng.integers(0, n, 4096), np.arange(n - 600, n)]))
    assert np.array_equal(oracle.decode(data[:200_000])[:1000], G[:1000])
    got, st = decode_gpu(data, n, 5)
    assert st == 0
    assert np.array_equal(got[idx], x[idx])


@pytest.mark.parametrize("n", [0, 1, 6143, 6144, 6145, 50_021])
@pytest.mark.parametrize("elem_off", [0, 1])
def test_encode_parity(n, elem_off):
    G = GAPS["one_two"](n, 11).astype(np.uint32)
    x = ids_from_gaps(G, 77)
    buf = torch.zeros(n + 8, dtype=torch.int32, device="cuda")
    if n:
        buf[elem_off:elem_off + n] = torch.from_numpy(x.view(np.int32)).cuda()
    out, nb = vbyte.encode_device(buf[elem_off:elem_off + n], prev=77, minus_one=True)
    k = int(nb.item())
    assert vbyte.get_status() == 0
    want = oracle.encode_delta_m1(x, prev=77)
    assert k == want.size and np.array_equal(out[:k].cpu().numpy(), want)
    assert np.array_equal(vbyte.encode_delta_m1(x, prev=77), want)   # the host encoder too


def test_encode_decode_round_trip_wrapping():
    x = inputs.full_range(3 * 6144 + 5, seed=8)   # unsorted: every gap wraps mod 2^32
    d = torch.from_numpy(x.view(np.int32)).cuda()
    out, nb = vbyte.encode_device(d, prev=9, minus_one=True)
    k = int(nb.item())
    back, st = decode_gpu(out[:k].cpu().numpy(), x.size, 9)
    assert st == 0 and np.array_equal(back, x)
