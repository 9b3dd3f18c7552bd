"""GPU parity: the CUDA decoder against the CPU oracle, element by element.

Integer work, so the bar is bit-exact equality.  Every input is seeded and
synthetic; the bytes come from the oracle's encoder and the expected values
from the oracle's Algorithm 1 (Sec. 2), so nothing expected comes from the
CUDA path.  Calls go through the C ABI via the ctypes binding.
"""
import numpy as np
import pytest

import oracle
from paper_1503_07387_gb300 import inputs, vbyte

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, params=[1, 2, 3, 4], ids=["onepass", "twopass", "split", "table"])
def kernel(request):
    """Every test runs on each single-stream kernel: the single pass with a
    decoupled look-back, count-then-decode in one launch, the split count /
    scan / decode launches, and the split launches decoding by the
    table-driven steps of Sec. 4."""
    vbyte.debug_force_passes(request.param)
    yield request.param
    vbyte.debug_force_passes(0)

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

TILE = 4096


def run_gpu(data: np.ndarray, n: int, delta=False, prev=0, in_off=0, out_off=0, guard=16):
    """Decode on the GPU with the input placed `in_off` bytes into a buffer and
    the output `out_off` words into a buffer padded by `guard` sentinel words on
    both sides.  Returns (values, status) and checks the sentinels."""
    data = np.ascontiguousarray(data, dtype=np.uint8)
    dbuf = torch.zeros(in_off + data.size + 16, dtype=torch.uint8, device="cuda")
    if data.size:
        dbuf[in_off:in_off + data.size] = torch.from_numpy(data).cuda()
    d_in = dbuf[in_off:in_off + data.size]
    sentinel = 0xA5A5A5A5
    obuf = torch.from_numpy(np.full(out_off + n + 2 * guard, sentinel, np.uint32)).cuda()
    d_out = obuf[guard + out_off:guard + out_off + n]
    assert vbyte.get_status() == 0
    if delta:
        vbyte.decode_delta(d_in, n, prev=prev, out=d_out)
    else:
        vbyte.decode(d_in, n, out=d_out)
    st = vbyte.get_status()
    host = obuf.cpu().numpy()
    assert (host[:guard + out_off] == sentinel).all(), "write before the output"
    assert (host[guard + out_off + n:] == sentinel).all(), "write past the output"
    return host[guard + out_off:guard + out_off + n].copy(), st


def check(values_or_bytes, delta=False, prev=0, encoded=False, **kw):
    data = values_or_bytes if encoded else oracle.encode(values_or_bytes)
    ref = oracle.decode_delta(data, prev=prev) if delta else oracle.decode(data)
    got, st = run_gpu(data, ref.size, delta=delta, prev=prev, **kw)
    assert st == oracle.validate(data, ref.size)
    if not np.array_equal(got, ref):
        bad = np.flatnonzero(got != ref)
        raise AssertionError(f"{bad.size} mismatches, first at {bad[0]}: got {got[bad[0]]} want {ref[bad[0]]}")
    return got


# ------------------------------------------------------------ paper vectors --

def test_fig1_on_gpu():
    data = np.array([0x80, 0x01, 0x82, 0x03, 0x10, 0x20], np.uint8)
    got, st = run_gpu(data, 4)
    assert st == 0 and got.tolist() == [128, 386, 16, 32]
    got, st = run_gpu(data, 4, delta=True)
    assert st == 0 and got.tolist() == [128, 514, 530, 562]


def test_table1_on_gpu():
    vals = [1, 2, 4, 128, 256, 512, 16384, 32768]
    check(np.array(vals, np.uint32))


# ------------------------------------------------------------- small / ragged --

GENS = {
    "mixed": lambda n, s: inputs.uniform_bits(n, seed=s),
    "one_byte": lambda n, s: (inputs.uniform_bits(n, seed=s) & 0x7F).astype(np.uint32),
    "one_two": lambda n, s: inputs.one_two_byte_mix(n, seed=s),
    "five_byte": lambda n, s: inputs.full_range(n, seed=s) | np.uint32(1 << 28),
    "geometric": lambda n, s: inputs.geometric_gaps(n, seed=s),
    "uniform300": lambda n, s: inputs.uniform_gaps(n, seed=s),
}


@pytest.mark.parametrize("kind", sorted(GENS))
@pytest.mark.parametrize("n", [1, 2, 3, 7, 100, 819, 4095, 4096, 4097, 12289, 100_003])
@pytest.mark.parametrize("delta", [False, True])
def test_ragged_sizes(kind, n, delta):
    v = GENS[kind](n, n + 17)
    check(v, delta=delta, prev=(12345 if delta else 0))


@pytest.mark.parametrize("in_off", list(range(16)))
@pytest.mark.parametrize("delta", [False, True])
def test_unaligned_input(in_off, delta):
    v = inputs.uniform_bits(20_000, seed=in_off)
    check(v, delta=delta, in_off=in_off)


@pytest.mark.parametrize("out_off", [1, 2, 3, 5])
@pytest.mark.parametrize("kind", ["mixed", "one_byte", "one_two"])
@pytest.mark.parametrize("delta", [False, True])
def test_unaligned_output(out_off, kind, delta):
    v = GENS[kind](30_001, out_off)
    check(v, delta=delta, out_off=out_off, in_off=3)


@pytest.mark.parametrize("nbytes", list(range(0, 65)))
def test_tiny_streams_around_alignment(nbytes):
    rng = np.random.default_rng(nbytes)
    # random well-formed stream of exactly nbytes bytes: lengths 1..5
    lens = []
    left = nbytes
    while left:
        L = int(rng.integers(1, min(5, left) + 1))
        lens.append(L)
        left -= L
    data = bytearray()
    for L in lens:
        body = rng.integers(0, 128, size=L).astype(np.uint8)
        body[:-1] |= 0x80
        data += bytes(body)
    data = np.frombuffer(bytes(data), np.uint8)
    for off in (0, 7, 13):
        check(data, encoded=True, in_off=off)
        check(data, encoded=True, delta=True, in_off=off, prev=9)


def test_empty_is_noop():
    got, st = run_gpu(np.zeros(0, np.uint8), 0)
    assert got.size == 0 and st == 0


def test_straddles_every_tile_boundary():
    """Place a 1..5-byte code so that its terminator falls k = 0..L-1 bytes after
    the first tile boundary (tiles start at 16-byte aligned addresses, so with
    the input at offset in_off the boundary is stream byte TILE - in_off)."""
    for in_off in (0, 5):
        boundary = TILE - in_off
        for L in range(1, 6):
            code = 5 if L == 1 else (1 << (7 * (L - 1))) + 12345
            assert len(oracle.encode_one(code)) == L
            for k in range(L):
                start = boundary + k - (L - 1)
                v = np.concatenate([np.full(start, 3, np.uint32), np.array([code], np.uint32),
                                    np.full(TILE + 50, 9, np.uint32),
                                    np.array([2**32 - 1], np.uint32),
                                    np.arange(3000, dtype=np.uint32)])
                check(v, in_off=in_off)
                check(v, delta=True, in_off=in_off)


def test_five_byte_edge_values():
    v = np.array([0xF0000000, 0xFFFFFFFF, 1 << 28, (1 << 28) - 1, 0, 127, 128] * 3000, np.uint32)
    check(v)
    check(v, delta=True)


def test_noncanonical_and_high_fifth_byte():
    # overlong zero and a fifth byte >= 16: Algorithm 1 keeps b * 2^28 mod 2^32
    data = np.frombuffer(b"\x80\x00" + b"\x80\x80\x80\x80\x7f" + b"\x81\x82\x83\x84\x10" * 2000 +
                         b"\x05", np.uint8)
    check(data, encoded=True)
    check(data, encoded=True, delta=True)


# ---------------------------------------------------------- malformed input --

def _status_only(data, n, delta=False):
    _, st = run_gpu(np.frombuffer(bytes(data), np.uint8), n, delta=delta)
    return st


def test_status_truncated():
    assert _status_only(b"\x05\x06\x80", 2) == oracle.validate(b"\x05\x06\x80", 2)
    body = bytes(oracle.encode(inputs.uniform_bits(9000, seed=1))) + b"\x81"
    assert _status_only(body, 9000) == oracle.ERR_TRUNCATED


def test_status_malformed_long():
    body = bytes(oracle.encode(np.arange(5000, dtype=np.uint32))) + b"\x80" * 6 + b"\x01" + \
        bytes(oracle.encode(np.arange(7000, dtype=np.uint32)))
    n = 5000 + 1 + 7000
    assert _status_only(body, n) == oracle.validate(body, n)
    assert _status_only(body, n) & oracle.ERR_MALFORMED_LONG


def test_status_count_mismatch_and_clamp():
    v = inputs.uniform_bits(10_000, seed=2)
    data = oracle.encode(v)
    ref = oracle.decode(data)
    # ask for fewer values: the first n are exact, nothing past n is written
    got, st = run_gpu(data, 6000)
    assert st == oracle.ERR_COUNT_MISMATCH
    assert np.array_equal(got, ref[:6000])
    # ask for more values: the ones the stream defines are exact
    got, st = run_gpu(data, 12_000)
    assert st == oracle.ERR_COUNT_MISMATCH
    assert np.array_equal(got[:10_000], ref)
    # empty stream but values expected
    _, st = run_gpu(np.zeros(0, np.uint8), 5)
    assert st == oracle.ERR_COUNT_MISMATCH


def test_status_is_per_stream_and_cleared():
    data = np.frombuffer(b"\x01\x80", np.uint8)
    _, st = run_gpu(data, 1)
    assert st == oracle.ERR_TRUNCATED
    assert vbyte.get_status() == 0


# ---------------------------------------------------------- host-buffer API --

def test_decode_host_round_trip():
    v = inputs.uniform_bits(300_000, seed=8)
    data = oracle.encode(v)
    assert np.array_equal(vbyte.decode_host(data, v.size), oracle.decode(data))
    assert np.array_equal(vbyte.decode_host(data, v.size, delta=True, prev=4),
                          oracle.decode_delta(data, prev=4))
    assert vbyte.get_status() == 0


@pytest.mark.parametrize("off", [0, 1, 3])
def test_decode_host_into_page_locked_output(off):
    """Page-locked output (the form bench.py's end-to-end number uses): same
    values, and the words around the output untouched (offset views)."""
    v = inputs.one_two_byte_mix(200_003, seed=off)
    data = oracle.encode_delta(np.cumsum(v.astype(np.uint64)).astype(np.uint32))
    n = v.size
    pinned = torch.full((n + 8,), 0x3C3C3C3C, dtype=torch.int32).pin_memory()
    h = pinned.numpy().view(np.uint32)
    out = h[off:off + n]
    vbyte.decode_host(data, n, delta=True, prev=0, out=out)
    assert vbyte.get_status() == 0
    assert np.array_equal(out, oracle.decode_delta(data, prev=0))
    assert np.all(h[:off] == 0x3C3C3C3C) and np.all(h[off + n:] == 0x3C3C3C3C)


def test_two_streams_independent():
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    v1 = inputs.uniform_bits(200_000, seed=1)
    v2 = inputs.geometric_gaps(300_000, seed=2)
    d1 = torch.from_numpy(oracle.encode(v1)).cuda()
    d2 = torch.from_numpy(oracle.encode(v2)).cuda()
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        o1 = vbyte.decode(d1, v1.size, stream=s1)
    with torch.cuda.stream(s2):
        o2 = vbyte.decode_delta(d2, v2.size, stream=s2)
    torch.cuda.synchronize()
    assert vbyte.get_status(s1) == 0 and vbyte.get_status(s2) == 0
    assert np.array_equal(o1.cpu().numpy(), v1)
    assert np.array_equal(o2.cpu().numpy(), oracle.decode_delta(oracle.encode(v2)))


# ------------------------------------------------------ full-size workloads --

def _full(values, delta):
    data = oracle.encode(values)
    ref = oracle.decode_delta(data) if delta else oracle.decode(data)
    d_in = torch.from_numpy(data).cuda()
    out = (vbyte.decode_delta if delta else vbyte.decode)(d_in, ref.size)
    st = vbyte.get_status()
    assert st == 0
    got = out.cpu().numpy()
    assert np.array_equal(got, ref)


def test_full_uniform_bits_1e6():
    _full(inputs.uniform_bits(1_000_000, seed=0), delta=False)


@pytest.mark.slow
@pytest.mark.parametrize("gen", ["geometric", "uniform300"])
def test_full_differential_2_26(gen):
    g = inputs.geometric_gaps(1 << 26, seed=0) if gen == "geometric" else inputs.uniform_gaps(1 << 26, seed=1)
    _full(g, delta=True)


@pytest.mark.slow
@pytest.mark.parametrize("gen", ["one_two", "full_range"])
@pytest.mark.parametrize("delta", [False, True])
def test_full_roofline_stress_2_28(gen, delta):
    v = inputs.one_two_byte_mix(1 << 28, seed=0) if gen == "one_two" else inputs.full_range(1 << 28, seed=0)
    _full(v, delta)
