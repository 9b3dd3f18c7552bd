"""Property checks of the oracle on generated inputs (hypothesis; skipped where
it is not installed).  They widen the pins of test_oracle_pins.py: every
encoder round-trips through its decoder on arbitrary lists, the stored
integers of every differential form are the differences that form defines
(computed here with Python integers), and the byte-length rule of Sec. 1
holds for every value drawn."""
import numpy as np
import pytest

import oracle

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings

M32 = (1 << 32) - 1
M64 = (1 << 64) - 1
u32 = st.integers(0, M32)
u64 = st.integers(0, M64)
lists32 = st.lists(u32, max_size=300)
lists64 = st.lists(u64, max_size=200)


def length(v):
    """Sec. 1: seven bits per byte, at least one byte."""
    return max(1, (v.bit_length() + 6) // 7)


@settings(max_examples=200, deadline=None)
@given(lists32)
def test_plain_round_trip_and_lengths(xs):
    x = np.array(xs, dtype=np.uint32)
    enc = oracle.encode(x)
    assert enc.size == sum(length(v) for v in xs)
    assert oracle.decode(enc).tolist() == xs
    assert oracle.validate(enc, len(xs)) == 0


@settings(max_examples=200, deadline=None)
@given(lists32, u32)
def test_delta_stores_differences(xs, prev):
    x = np.array(xs, dtype=np.uint32)
    enc = oracle.encode_delta(x, prev)
    before = [prev] + xs[:-1]
    assert oracle.decode(enc).tolist() == [(a - b) & M32 for a, b in zip(xs, before)]
    assert oracle.decode_delta(enc, len(xs), prev).tolist() == xs


@settings(max_examples=200, deadline=None)
@given(lists32, u32)
def test_m1_stores_differences_minus_one(xs, prev):
    x = np.array(xs, dtype=np.uint32)
    enc = oracle.encode_delta_m1(x, prev)
    before = [prev] + xs[:-1]
    want = [(a - b - (1 if i else 0)) & M32 for i, (a, b) in enumerate(zip(xs, before))]
    assert oracle.decode(enc).tolist() == want
    assert oracle.decode_delta_m1(enc, len(xs), prev).tolist() == xs


@settings(max_examples=200, deadline=None)
@given(lists32, st.lists(u32, min_size=4, max_size=4))
def test_blocked_stores_differences_four_apart(xs, seed):
    x = np.array(xs, dtype=np.uint32)
    enc = oracle.encode_delta4(x, seed)
    ext = seed + xs
    assert oracle.decode(enc).tolist() == [(ext[i + 4] - ext[i]) & M32 for i in range(len(xs))]
    assert oracle.decode_delta4(enc, len(xs), seed).tolist() == xs


@settings(max_examples=200, deadline=None)
@given(lists64, u64)
def test_64_bit_round_trips(xs, prev):
    x = np.array(xs, dtype=np.uint64)
    enc = oracle.encode64(x)
    assert enc.size == sum(length(v) for v in xs)
    assert [int(v) for v in oracle.decode64(enc)] == xs
    assert oracle.validate64(enc, len(xs)) == 0
    d = oracle.encode_delta64(x, prev)
    before = [prev] + xs[:-1]
    assert [int(v) for v in oracle.decode64(d)] == [(a - b) & M64 for a, b in zip(xs, before)]
    assert [int(v) for v in oracle.decode_delta64(d, len(xs), prev)] == xs


@settings(max_examples=300, deadline=None)
@given(st.binary(max_size=64), st.integers(0, 70))
def test_validation_on_arbitrary_bytes(data, n):
    """The data-error contract restated over the bytes: runs of continuation
    bytes (five or more for uint32, ten or more for uint64), a final
    continuation byte, and the count of terminators."""
    runs, r = [], 0
    for b in data:
        r = r + 1 if b & 0x80 else 0
        runs.append(r)
    terms = sum(1 for b in data if not b & 0x80)
    tail = bool(data) and bool(data[-1] & 0x80)
    for lim, fn, bit in ((5, oracle.validate, 1), (10, oracle.validate64, 1)):
        want = (bit if any(x >= lim for x in runs) else 0) | (2 if tail else 0) | (4 if terms != n else 0)
        assert fn(data, n) == want
    if not any(x >= 5 for x in runs):
        assert oracle.decode(data).size == terms
