"""GPU parity for 64-bit VByte decoding (Sec. 1 notes the format covers 64-bit
integers; Algorithm 1 read for uint64): vbyte_decode64 and
vbyte_decode_delta64 against the oracle, bit for bit, through the C ABI.
Expected values come only from the oracle or from the values the streams were
built from."""
import numpy as np
import pytest

import oracle
from paper_1503_07387_gb300 import inputs, vbyte

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

GUARD = 0x5A5A5A5A5A5A5A5A
MASK64 = (1 << 64) - 1


def all_widths(n, seed):
    """uint64 values of every bit width 0..64, equally often (code lengths 1..10)."""
    return inputs.uniform_bits64(n, seed=seed)


VALUES = {
    "one_byte": lambda n, s: (inputs.geometric_gaps(n, seed=s) & 127).astype(np.uint64),
    "all_widths": all_widths,
    "ten_bytes": lambda n, s: all_widths(n, s) | np.uint64(1 << 63),
}


def decode_gpu(data, n, delta=False, prev=0, byte_off=0):
    """Decode with the stream `byte_off` bytes into a device buffer; the output
    sits between guard words that must stay untouched."""
    data = np.array(data, dtype=np.uint8)   # a writable copy
    buf = torch.zeros(byte_off + data.size + 16, dtype=torch.uint8, device="cuda")
    if data.size:
        buf[byte_off:byte_off + data.size] = torch.from_numpy(data).cuda()
    d = buf[byte_off:byte_off + data.size]
    g = np.full(n + 64, GUARD, dtype=np.uint64)
    guard = torch.from_numpy(g.view(np.int64)).cuda()
    out = guard[32:32 + n]
    assert vbyte.get_status() == 0
    if delta:
        vbyte.decode_delta64(d, n, prev=prev, out=out)
    else:
        vbyte.decode64(d, n, out=out)
    st = vbyte.get_status()
    h = guard.cpu().numpy().view(np.uint64)
    assert np.all(h[:32] == GUARD) and np.all(h[32 + n:] == GUARD), "writes outside the output"
    return h[32:32 + n].copy(), st


@pytest.mark.parametrize("kind", sorted(VALUES))
@pytest.mark.parametrize("n", [1, 7, 409, 410, 4095, 4097, 70_001, 1_000_003])
@pytest.mark.parametrize("byte_off", [0, 9])
def test_plain_parity(kind, n, byte_off):
    v = VALUES[kind](n, n % 89)
    data = oracle.encode64(v)
    got, st = decode_gpu(data, n, byte_off=byte_off)
    assert st == 0
    assert np.array_equal(got, oracle.decode64(data, n))
    assert np.array_equal(got, v)


@pytest.mark.parametrize("byte_off", range(16))
def test_every_input_alignment(byte_off):
    v = all_widths(3 * 4096 + 11, byte_off)
    data = oracle.encode64(v)
    got, st = decode_gpu(data, v.size, byte_off=byte_off)
    assert st == 0 and np.array_equal(got, v)


@pytest.mark.parametrize("kind", sorted(VALUES))
@pytest.mark.parametrize("n", [1, 4097, 300_007])
def test_delta_parity_wraps(kind, n):
    """Gaps of every width: the running sums wrap modulo 2^64."""
    x = VALUES[kind](n, n % 31 + 1)
    for prev in (0, MASK64, 1 << 40):
        data = oracle.encode_delta64(x, prev=prev)
        got, st = decode_gpu(data, n, delta=True, prev=prev, byte_off=3)
        assert st == 0
        assert np.array_equal(got, oracle.decode_delta64(data, n, prev=prev))
        assert np.array_equal(got, x)


def test_sorted_ids_delta():
    ids = np.cumsum(inputs.geometric_gaps(1 << 20, seed=4).astype(np.uint64)) + np.uint64(1 << 50)
    data = oracle.encode_delta64(ids)
    got, st = decode_gpu(data, ids.size, delta=True)
    assert st == 0 and np.array_equal(got, ids)


def test_length_boundaries():
    edges = [0, 1, MASK64] + [(1 << (7 * k)) + d for k in range(1, 10) for d in (-1, 0)]
    v = np.array(edges * 700, dtype=np.uint64)
    data = oracle.encode64(v)
    got, st = decode_gpu(data, v.size)
    assert st == 0 and np.array_equal(got, v)


def test_empty_and_count_mismatch():
    got, st = decode_gpu(np.zeros(0, np.uint8), 0)
    assert got.size == 0 and st == 0
    got, st = decode_gpu(np.zeros(0, np.uint8), 3)
    assert st == oracle.ERR_COUNT_MISMATCH
    v = all_widths(5000, 1)
    data = oracle.encode64(v)
    for n in (4999, 5001):
        got, st = decode_gpu(data, n)
        assert st == oracle.validate64(data, n) == oracle.ERR_COUNT_MISMATCH
        k = min(n, v.size)
        assert np.array_equal(got[:k], v[:k])


def test_malformed_status_parity():
    """Random streams with many high-bit bytes: the status bits equal the
    oracle's validation (runs of ten or more, a truncated end, the count);
    where the stream is well formed the values equal the oracle's."""
    rng = np.random.default_rng(12)
    for trial in range(60):
        L = int(rng.integers(1, 20_000))
        p = float(rng.random()) * 0.97
        data = (rng.integers(0, 128, L) | ((rng.random(L) < p) * 128)).astype(np.uint8)
        n = int((data < 128).sum()) + int(rng.integers(-1, 2))
        n = max(n, 0)
        got, st = decode_gpu(data, n, byte_off=trial % 16)
        assert st == oracle.validate64(data, n), trial
        if st == 0:
            assert np.array_equal(got, oracle.decode64(data, n))


def test_ten_byte_runs_and_truncation():
    good = b"\x80" * 9 + b"\x01"
    data = np.frombuffer(good * 1000, dtype=np.uint8)
    got, st = decode_gpu(data, 1000)
    assert st == 0 and np.all(got == np.uint64(1 << 63))
    bad = np.frombuffer(b"\x05" + b"\x80" * 10 + b"\x01", dtype=np.uint8)
    _, st = decode_gpu(bad, 2)
    assert st & oracle.ERR_MALFORMED_LONG and st == oracle.validate64(bad, 2)
    trunc = np.frombuffer(b"\x05\x06\x80", dtype=np.uint8)
    got, st = decode_gpu(trunc, 2)
    assert st == oracle.ERR_TRUNCATED and got.tolist() == [5, 6]


def test_full_size_sampled():
    """2^26 values of every width (about 340 MB of input), with the library's
    host encoder (pinned byte for byte to the oracle's on CPU); every value
    is checked against the values the stream was built from."""
    n = 1 << 26
    v = all_widths(n, 7)
    data = vbyte.encode64(v)
    assert np.array_equal(data[:100_000], oracle.encode64(v[:100_000])[:100_000])
    got, st = decode_gpu(data, n)
    assert st == 0 and np.array_equal(got, v)
