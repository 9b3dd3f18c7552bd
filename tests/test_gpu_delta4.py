"""GPU parity of blocked differences (Sec. 1, "Differential coding": x_1, x_2,
x_3, x_4, x_5 - x_1, x_6 - x_2, ...): vbyte_decode_delta4 against the
oracle's Algorithm 1 followed by x_i = g_i + x_{i-4}, bit for bit, on bytes
from the oracle's encoder.  Every class of ranks modulo 4 is its own running
sum; the four values before the list seed the classes."""
import numpy as np
import pytest

import oracle
from paper_1503_07387_gb300 import inputs, vbyte

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SENTINEL = 0xA5A5A5A5


def interleaved_ids(n, seed):
    """Four sorted id lists interleaved: x_{4j+k} is list k's j-th id, so
    blocked differences are each list's own gaps."""
    g = inputs.geometric_gaps(n, seed=seed).astype(np.uint64) + 1
    x = np.zeros(n, dtype=np.uint64)
    for k in range(4):
        x[k::4] = np.cumsum(g[k::4])
    return x.astype(np.uint32)


GENS = {
    "interleaved": lambda n, s: interleaved_ids(n, s),
    "mixed": lambda n, s: inputs.uniform_bits(n, seed=s),
    "full_range": lambda n, s: inputs.full_range(n, seed=s),
}


def run(data, n, prev4=None, in_off=0, out_off=0, guard=8):
    data = np.ascontiguousarray(data, dtype=np.uint8)
    dbuf = torch.zeros(in_off + data.size + 16, dtype=torch.uint8, device="cuda")
    if data.size:
        dbuf[in_off:in_off + data.size] = torch.from_numpy(data.copy()).cuda()
    obuf = torch.from_numpy(np.full(out_off + n + 2 * guard, SENTINEL, np.uint32)).cuda()
    d_out = obuf[guard + out_off:guard + out_off + n]
    assert vbyte.get_status() == 0
    vbyte.decode_delta4(dbuf[in_off:in_off + data.size], n, prev4=prev4, out=d_out)
    st = vbyte.get_status()
    h = obuf.cpu().numpy()
    assert (h[:guard + out_off] == SENTINEL).all() and (h[guard + out_off + n:] == SENTINEL).all(), \
        "write outside the output"
    return h[guard + out_off:guard + out_off + n].copy(), st


def check(x, prev4=None, **kw):
    data = oracle.encode_delta4(x, prev4=prev4)
    want = oracle.decode_delta4(data, x.size, prev4=prev4)
    assert np.array_equal(want, x.astype(np.uint32))   # the round trip the oracle pins
    got, st = run(data, x.size, prev4=prev4, **kw)
    assert st == 0
    if not np.array_equal(got, want):
        bad = np.flatnonzero(got != want)
        raise AssertionError(f"{bad.size} mismatches, first at {bad[0]}: got {got[bad[0]]} want {want[bad[0]]}")


@pytest.mark.parametrize("kind", sorted(GENS))
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 100, 513, 2049, 8191, 100_003, 1_000_003])
def test_ragged_sizes(kind, n):
    check(GENS[kind](n, 5), prev4=None)


@pytest.mark.parametrize("prev4", [None, [1, 2, 3, 4], [0xFFFFFFFF, 0xFFFFFFF0, 7, 0x80000000]])
@pytest.mark.parametrize("n", [3, 6, 77_777, 3_000_001])
def test_seeds_and_wraparound(prev4, n):
    check(GENS["mixed"](n, 6), prev4=prev4)
    check(GENS["interleaved"](n, 7), prev4=prev4)


@pytest.mark.parametrize("in_off", [0, 1, 5, 15])
@pytest.mark.parametrize("out_off", [0, 1, 2, 3])
def test_unaligned(in_off, out_off):
    check(GENS["interleaved"](50_001, 8), prev4=[9, 8, 7, 6], in_off=in_off, out_off=out_off)


def test_paper_list_form():
    # stored integers x_1, x_2, x_3, x_4, x_5 - x_1, ... (zero seeds)
    x = np.array([3, 10, 11, 20, 23, 31, 40, 44, 60], np.uint32)
    stored = np.concatenate([x[:4], x[4:] - x[:-4]])
    data = oracle.encode(stored)
    got, st = run(data, x.size)
    assert st == 0 and np.array_equal(got, x)


def test_count_mismatch_and_clamp():
    x = GENS["mixed"](1000, 9)
    data = oracle.encode_delta4(x)
    got, st = run(data, 900)
    assert st == vbyte.ERR_COUNT_MISMATCH == oracle.validate(data, 900)
    assert np.array_equal(got, oracle.decode_delta4(data)[:900])   # the first 900 of its 1000
    got, st = run(data, 1100)
    assert st & vbyte.ERR_COUNT_MISMATCH
    assert np.array_equal(got[:1000], x)


def test_empty():
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    vbyte.decode_delta4(torch.zeros(0, dtype=torch.uint8, device="cuda"), 0, out=out)
    assert vbyte.get_status() == 0


@pytest.mark.slow
def test_full_size_2_26():
    n = 1 << 26
    x = interleaved_ids(n, 10)
    data = vbyte.encode_delta4(x)
    assert np.array_equal(data, oracle.encode_delta4(x))
    out = vbyte.decode_delta4(torch.from_numpy(data.copy()).cuda(), n)
    assert vbyte.get_status() == 0
    assert torch.equal(out.view(torch.int32), torch.from_numpy(x.view(np.int32)).cuda())
