"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

Each test fixes the oracle to something other than itself: the byte strings
printed in Table 1 and Fig. 1, closed forms that follow from the format's
definition (Sec. 1), exhaustive enumeration on small ranges, numpy's own
cumulative sum for the differential rule, and the special cases Algorithm 1
(Sec. 2) fixes for the fifth byte.  A plausible slip in the oracle -- reversed
byte order, inverted continuation bit, a dropped 7-bit group, a wrong shift,
an off-by-one in the running sum -- fails at least one of them.
"""
import numpy as np
import pytest

import oracle
from conftest import read_golden
from paper_1503_07387_gb300 import inputs

MASK32 = (1 << 32) - 1


def _hex(bs):
    return bytes(int(x, 16) for x in bs)


# ------------------------------------------------------------ printed values --

def test_table1_encodings():
    """Table 1 (Sec. 1): the printed VByte forms of 1, 2, 4, 128, ..., 32768."""
    rows = read_golden("table1.txt")
    assert len(rows) == 8
    for row in rows:
        v, expect = int(row[0]), _hex(row[1:])
        assert oracle.encode_one(v) == expect
        assert oracle.encode([v]).tobytes() == expect
        assert oracle.decode(expect).tolist() == [v]


def test_table1_as_one_stream():
    rows = read_golden("table1.txt")
    vals = [int(r[0]) for r in rows]
    stream = b"".join(_hex(r[1:]) for r in rows)
    assert oracle.encode(vals).tobytes() == stream
    assert oracle.decode(stream).tolist() == vals


def test_fig1_example():
    """Fig. 1 (Sec. 4): 80 01 82 03 10 20 -> 128, 386, 16, 32."""
    rows = {r[0]: r[1:] for r in read_golden("fig1.txt")}
    data = _hex(rows["bytes"])
    vals = [int(x) for x in rows["values"]]
    assert oracle.decode(data).tolist() == vals
    assert oracle.encode(vals).tobytes() == data
    assert oracle.validate(data, 4) == 0


# ------------------------------------------------------------- closed forms --

def _length_closed_form(v):
    """Sec. 1: [0,2^7) -> 1 byte, [2^7,2^14) -> 2 bytes, and so on."""
    v = np.asarray(v, dtype=np.uint64)
    return (1 + (v >= 1 << 7).astype(int) + (v >= 1 << 14) + (v >= 1 << 21)
            + (v >= 1 << 28))


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_powers_of_128(k):
    """2^(7k) is k continuation bytes 0x80 followed by 0x01."""
    v = 1 << (7 * k)
    assert oracle.encode_one(v) == b"\x80" * k + b"\x01"
    assert oracle.decode(b"\x80" * k + b"\x01").tolist() == [v]


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_powers_of_128_minus_one(k):
    """2^(7k) - 1 is k-1 bytes 0xFF followed by 0x7F."""
    v = (1 << (7 * k)) - 1
    assert oracle.encode_one(v) == b"\xff" * (k - 1) + b"\x7f"
    assert oracle.decode(b"\xff" * (k - 1) + b"\x7f").tolist() == [v]


def test_max_uint32():
    """2^32 - 1: four full groups then the top four bits, 0x0F."""
    assert oracle.encode_one(MASK32) == b"\xff\xff\xff\xff\x0f"
    assert oracle.decode(b"\xff\xff\xff\xff\x0f").tolist() == [MASK32]


def test_brute_force_21_bits():
    """Every v in [0, 2^21): length rule, continuation bits, and the round trip."""
    v = np.arange(1 << 21, dtype=np.uint32)
    enc = oracle.encode(v)
    lens = _length_closed_form(v)
    assert enc.size == int(lens.sum())
    # continuation bit set on exactly the non-final byte of each integer
    ends = np.cumsum(lens) - 1
    msb = (enc >> 7).astype(bool)
    assert not msb[ends].any()
    assert msb.sum() == enc.size - v.size
    dec = oracle.decode(enc)
    assert np.array_equal(dec, v)


@pytest.mark.parametrize("lo,hi", [(1 << 21, 1 << 28), (1 << 28, 1 << 32)])
def test_random_round_trip_long_codes(lo, hi):
    rng = np.random.default_rng(7)
    v = rng.integers(lo, hi, size=200_000, dtype=np.uint64).astype(np.uint32)
    v[:4] = [lo, lo + 1, hi - 2, hi - 1]
    enc = oracle.encode(v)
    assert enc.size == int(_length_closed_form(v).sum())
    assert np.array_equal(oracle.decode(enc), v)


def test_group_sum_definition_small():
    """For a few thousand values, the bytes satisfy v = sum (b_k mod 128) 2^(7k)
    with Python integers, independently of Algorithm 1's loop structure."""
    rng = np.random.default_rng(3)
    for v in rng.integers(0, 1 << 32, size=3000, dtype=np.uint64).tolist():
        bs = oracle.encode_one(v)
        assert sum((b & 127) << (7 * k) for k, b in enumerate(bs)) == v


def test_round_trip_all_code_lengths_mixed():
    v = inputs.uniform_bits(200_000, seed=11)
    assert np.array_equal(oracle.decode(oracle.encode(v)), v)


# ------------------------------------------------- Algorithm 1 special cases --

def test_fifth_byte_keeps_low_four_bits():
    """Algorithm 1 appends c + b * 2^28 into a 32-bit array: only b's low four
    bits survive, and the fifth byte's high bit is never tested."""
    assert oracle.decode(b"\x80\x80\x80\x80\x7f").tolist() == [0xF0000000]
    assert oracle.decode(b"\x81\x82\x83\x84\x10").tolist() == [
        (1 + (2 << 7) + (3 << 14) + (4 << 21)) & MASK32]
    # fifth byte with the high bit set: still consumed as the last byte
    assert oracle.decode(b"\x80\x80\x80\x80\xff\x05").tolist() == [0xF0000000, 5]
    assert oracle.validate(b"\x80\x80\x80\x80\xff\x05", 2) & oracle.ERR_MALFORMED_LONG


def test_overlong_zero():
    """Non-canonical 0x80 0x00 decodes to 0 under Algorithm 1."""
    assert oracle.decode(b"\x80\x00").tolist() == [0]


def test_truncated_tail_drops_partial_integer():
    assert oracle.decode(b"\x05\x80").tolist() == [5]
    assert oracle.validate(b"\x05\x80", 1) == oracle.ERR_TRUNCATED
    assert oracle.decode(b"").tolist() == []
    assert oracle.validate(b"", 0) == 0


def test_validation_contract():
    assert oracle.validate(b"\x01\x02", 2) == 0
    assert oracle.validate(b"\x01\x02", 3) == oracle.ERR_COUNT_MISMATCH
    # four continuation bytes are fine, five are malformed
    assert oracle.validate(b"\x80\x80\x80\x80\x01", 1) == 0
    assert oracle.validate(b"\x80\x80\x80\x80\x80\x01", 1) & oracle.ERR_MALFORMED_LONG
    assert oracle.validate(b"\x01\x80\x80\x80\x80\x80", 1) == (
        oracle.ERR_MALFORMED_LONG | oracle.ERR_TRUNCATED)


# ------------------------------------------------------ differential coding --

def test_delta_equals_numpy_cumsum():
    """Sec. 1/2: decoding gaps with the running value equals the inclusive
    cumulative sum modulo 2^32 (numpy's cumsum in uint64, then wrapped)."""
    g = inputs.uniform_gaps(300_000, lo=0, hi=5_000_000, seed=5)
    ref = (np.cumsum(g.astype(np.uint64)) & MASK32).astype(np.uint32)
    assert np.array_equal(oracle.decode_delta(oracle.encode(g)), ref)
    assert int(g.astype(np.uint64).sum()) > MASK32  # the running sum really wraps


def test_delta_prev_seed():
    g = np.array([5, 1, 300, 0, 2**32 - 1], dtype=np.uint32)
    out = oracle.decode_delta(oracle.encode(g), prev=1000)
    ref = (1000 + np.cumsum(g.astype(np.uint64))) & MASK32
    assert out.tolist() == ref.tolist()


def test_fig1_as_gaps():
    rows = {r[0]: r[1:] for r in read_golden("fig1.txt")}
    assert oracle.decode_delta(_hex(rows["bytes"])).tolist() == [128, 514, 530, 562]


def test_encode_delta_round_trip_sorted_ids():
    ids, vo = inputs.posting_lists(num_lists=20, universe=1 << 30, cap=20_000, seed=2)
    x = ids[int(vo[0]):int(vo[1])]
    enc = oracle.encode_delta(x)
    gaps = np.diff(x.astype(np.int64), prepend=0).astype(np.uint32)
    assert np.array_equal(enc, oracle.encode(gaps))
    assert np.array_equal(oracle.decode_delta(enc), x)


def test_delta_wraps_modulo_2_32():
    x = np.array([2**32 - 10, 5, 7], dtype=np.uint32)  # not increasing: gaps wrap
    enc = oracle.encode_delta(x)
    assert np.array_equal(oracle.decode_delta(enc), x)


# ---------------------------------- differential coding, gaps minus one --
# Sec. 1 names a variant for lists without repeated values: x_1 - 0,
# x_2 - x_1 - 1, x_3 - x_2 - 1, ...

def test_m1_paper_form():
    """The stored integers are exactly the paper's list (x_1 - 0, x_2 - x_1 - 1, ...)."""
    x = np.array([3, 4, 7, 8, 100, 101], dtype=np.uint32)
    stored = [3, 4 - 3 - 1, 7 - 4 - 1, 8 - 7 - 1, 100 - 8 - 1, 101 - 100 - 1]
    enc = oracle.encode_delta_m1(x)
    assert oracle.decode(enc).tolist() == stored
    assert oracle.decode_delta_m1(enc).tolist() == x.tolist()


def test_m1_consecutive_ids_are_all_zero_bytes():
    """prev, prev+1, prev+2, ...: the first gap is 0 (x_1 - prev) and every
    later one 1 - 1 = 0, so the stream is n zero bytes."""
    x = (77 + np.arange(50_000, dtype=np.uint64)).astype(np.uint32)
    enc = oracle.encode_delta_m1(x, prev=77)
    assert enc.size == x.size and not enc.any()
    assert np.array_equal(oracle.decode_delta_m1(enc, prev=77), x)


def test_m1_generated_gaps_round_trip():
    """Ids built from chosen gaps G (x_0 = prev + G_0, x_i = x_{i-1} + 1 + G_i):
    the encoder stores exactly G and the decoder returns the ids, both checked
    against the construction rather than against each other."""
    rng = np.random.default_rng(9)
    G = rng.geometric(0.01, 200_000).astype(np.uint64) - 1
    prev = 12345
    x = ((prev + np.cumsum(G) + np.arange(G.size, dtype=np.uint64)) & MASK32).astype(np.uint32)
    enc = oracle.encode_delta_m1(x, prev=prev)
    assert np.array_equal(oracle.decode(enc), G.astype(np.uint32))
    assert np.array_equal(oracle.decode_delta_m1(enc, prev=prev), x)
    # the plain differential decoder of the same bytes lags by one per value
    lag = (oracle.decode_delta_m1(enc, prev=prev).astype(np.int64) -
           oracle.decode_delta(enc, prev=prev).astype(np.int64)) % (1 << 32)
    assert np.array_equal(lag, np.arange(G.size))


def test_m1_wraps_modulo_2_32():
    x = np.array([2**32 - 1, 0, 5, 5 + 2**31], dtype=np.uint32)   # 0 follows 2^32 - 1: gap 0
    enc = oracle.encode_delta_m1(x, prev=2**32 - 3)
    assert oracle.decode(enc).tolist() == [2, 0, 4, 2**31 - 1]
    assert np.array_equal(oracle.decode_delta_m1(enc, prev=2**32 - 3), x)


# ------------------------------------------------------------------ batched --

def test_batched_matches_per_list_and_concatenation():
    ids, vo = inputs.length_class_lists(300, max_class=10, seed=4)
    enc, bo = oracle.encode_batched(ids, vo, delta=True)
    out, st = oracle.decode_batched(enc, bo, vo, delta=True)
    assert st == 0
    assert np.array_equal(out, ids)
    for j in range(0, 300, 37):
        seg = enc[int(bo[j]):int(bo[j + 1])]
        assert np.array_equal(oracle.decode_delta(seg), ids[int(vo[j]):int(vo[j + 1])])
    # plain mode: decoding the concatenation as one stream is the same thing
    penc, pbo = oracle.encode_batched(ids, vo, delta=False)
    pout, pst = oracle.decode_batched(penc, pbo, vo, delta=False)
    assert pst == 0
    assert np.array_equal(pout, oracle.decode(penc))


def test_batched_prev_and_threads():
    ids, vo = inputs.length_class_lists(64, max_class=8, seed=9)
    prev = np.arange(64, dtype=np.uint32) * 7
    shifted = ids.copy()
    for j in range(64):
        shifted[int(vo[j]):int(vo[j + 1])] += prev[j]
    enc, bo = oracle.encode_batched(shifted, vo, delta=True, prev=prev)
    out1, st = oracle.decode_batched(enc, bo, vo, delta=True, prev=prev)
    out4, _ = oracle.decode_batched(enc, bo, vo, delta=True, prev=prev, threads=4)
    assert st == 0
    assert np.array_equal(out1, shifted)
    assert np.array_equal(out4, shifted)


def test_batched_count_mismatch_per_list():
    enc = np.frombuffer(b"\x01\x02\x03", dtype=np.uint8)
    bo = np.array([0, 1, 3], dtype=np.uint64)
    vo = np.array([0, 2, 3], dtype=np.uint64)   # list 0 claims 2 values, holds 1
    _, st = oracle.decode_batched(enc, bo, vo, delta=False)
    assert st == oracle.ERR_COUNT_MISMATCH


# ----------------------------------------------------------- 64-bit integers --
# Sec. 1 notes that the format applies to 64-bit integers too.  The 64-bit
# oracle is pinned to the same definition: seven bits per byte from the least
# significant end, so up to ten bytes; Algorithm 1 with ten steps.

MASK64 = (1 << 64) - 1


def _length64(v):
    """1 + [v >= 2^7] + [v >= 2^14] + ... + [v >= 2^63], with Python ints."""
    return 1 + sum(v >= 1 << (7 * k) for k in range(1, 10))


@pytest.mark.parametrize("k", range(10))
def test64_powers_of_128(k):
    v = 1 << (7 * k)
    assert oracle.encode64_one(v) == b"\x80" * k + b"\x01"
    assert oracle.decode64(b"\x80" * k + b"\x01").tolist() == [v]


@pytest.mark.parametrize("k", range(1, 10))
def test64_powers_of_128_minus_one(k):
    v = (1 << (7 * k)) - 1
    assert oracle.encode64_one(v) == b"\xff" * (k - 1) + b"\x7f"
    assert oracle.decode64(b"\xff" * (k - 1) + b"\x7f").tolist() == [v]


def test64_max():
    """2^64 - 1: nine full groups, then the top bit alone, 0x01."""
    assert oracle.encode64_one(MASK64) == b"\xff" * 9 + b"\x01"
    assert oracle.decode64(b"\xff" * 9 + b"\x01").tolist() == [MASK64]


def test64_group_sum_and_length_every_width():
    """For values of every bit width 0..64, the bytes satisfy
    v = sum (b_k mod 128) 2^(7k), the length closed form, and the
    continuation bits, checked with Python integers."""
    rng = np.random.default_rng(17)
    vals = [0, 1, MASK64]
    for bits in range(1, 65):
        top = 1 << (bits - 1)
        vals += [top, (top << 1) - 1] + [top | int(x) for x in rng.integers(0, top, 40, dtype=np.uint64)]
    for v in vals:
        bs = oracle.encode64_one(v)
        assert len(bs) == _length64(v), v
        assert sum((b & 127) << (7 * k) for k, b in enumerate(bs)) == v
        assert all(b & 128 for b in bs[:-1]) and not bs[-1] & 128
    arr = np.array(vals, dtype=np.uint64)
    enc = oracle.encode64(arr)
    assert enc.size == sum(_length64(v) for v in vals)
    assert np.array_equal(oracle.decode64(enc), arr)


def test64_agrees_with_32_bit_below_2_32():
    """Below 2^32 the 64-bit form is the 32-bit one, byte for byte."""
    v = inputs.uniform_bits(100_000, seed=5)
    enc = oracle.encode(v)
    assert np.array_equal(oracle.encode64(v.astype(np.uint64)), enc)
    assert np.array_equal(oracle.decode64(enc), v.astype(np.uint64))


def test64_tenth_byte_taken_whole():
    """The tenth byte is the last of an integer whatever its high bit; only
    its low bit survives the multiplication by 2^63 modulo 2^64."""
    assert oracle.decode64(b"\x80" * 9 + b"\x7f").tolist() == [1 << 63]
    assert oracle.decode64(b"\x80" * 9 + b"\xff\x05").tolist() == [1 << 63, 5]
    assert oracle.validate64(b"\x80" * 9 + b"\xff\x05", 2) & oracle.ERR_MALFORMED_LONG
    assert oracle.validate64(b"\x80" * 9 + b"\x01", 1) == 0
    assert oracle.validate64(b"\x80" * 10 + b"\x01", 1) & oracle.ERR_MALFORMED_LONG
    # five continuation bytes, malformed for uint32, are fine here
    assert oracle.validate64(b"\x80" * 5 + b"\x01", 1) == 0
    assert oracle.decode64(b"\x80" * 5 + b"\x01").tolist() == [1 << 35]


def test64_truncated_and_count():
    assert oracle.decode64(b"\x05\x80\x80").tolist() == [5]
    assert oracle.validate64(b"\x05\x80", 1) == oracle.ERR_TRUNCATED
    assert oracle.validate64(b"\x01\x02", 3) == oracle.ERR_COUNT_MISMATCH
    assert oracle.decode64(b"").tolist() == [] and oracle.validate64(b"", 0) == 0


def test64_delta_wraps_modulo_2_64():
    """Differential coding on uint64: the decoded values are numpy's uint64
    cumulative sum of the stored gaps from prev, wrapping modulo 2^64."""
    rng = np.random.default_rng(9)
    x = rng.integers(0, 1 << 63, 50_000, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, 50_000, dtype=np.uint64)
    for prev in (0, MASK64, 1 << 40):
        enc = oracle.encode_delta64(x, prev=prev)
        gaps = oracle.decode64(enc)
        with np.errstate(over="ignore"):
            assert np.array_equal(gaps, x - np.concatenate([[np.uint64(prev)], x[:-1]]))
            assert np.array_equal(np.cumsum(np.concatenate([[np.uint64(prev)], gaps]))[1:], x)
        assert np.array_equal(oracle.decode_delta64(enc, x.size, prev=prev), x)
    ids = np.cumsum(inputs.geometric_gaps(100_000, seed=2).astype(np.uint64)) + np.uint64(1 << 40)
    enc = oracle.encode_delta64(ids)
    assert enc.size == sum(_length64(int(g)) for g in np.diff(np.concatenate([[0], ids])).tolist())
    assert np.array_equal(oracle.decode_delta64(enc, ids.size), ids)


# ------------------------------------------------------ blocked differences --
# Sec. 1: x_1, x_2, x_3, x_4, x_5 - x_1, x_6 - x_2, x_7 - x_3, x_8 - x_4, ...

def test_delta4_paper_form():
    """The stored integers are the paper's list for a small example."""
    x = np.array([3, 10, 20, 21, 40, 41, 60, 100, 107], dtype=np.uint32)
    g = oracle.decode(oracle.encode_delta4(x))
    assert g.tolist() == [3, 10, 20, 21, 40 - 3, 41 - 10, 60 - 20, 100 - 21, 107 - 40]
    assert oracle.decode_delta4(oracle.encode_delta4(x)).tolist() == x.tolist()


def test_delta4_lanes_are_numpy_cumsums():
    """Each residue class mod 4 of the decoded list is numpy's cumulative sum
    (mod 2^32) of that class's stored integers, from its seed."""
    rng = np.random.default_rng(21)
    g = rng.integers(0, 1 << 32, 40_003, dtype=np.uint64).astype(np.uint32)
    data = oracle.encode(g)
    for prev4 in (None, [5, 0xFFFFFFFF, 7, 1 << 31]):
        x = oracle.decode_delta4(data, g.size, prev4=prev4)
        seeds = [0, 0, 0, 0] if prev4 is None else prev4
        for r in range(4):
            want = (np.cumsum(g[r::4].astype(np.uint64)) + seeds[r]) & MASK32
            assert np.array_equal(x[r::4], want.astype(np.uint32)), r


def test_delta4_round_trip_and_small_gaps():
    """Four interleaved sorted lists: the stored integers are each list's own
    gaps, and the round trip gives the lists back."""
    rng = np.random.default_rng(8)
    lanes = [np.cumsum(inputs.geometric_gaps(10_000, seed=s).astype(np.uint64)) for s in range(4)]
    x = np.stack(lanes, axis=1).reshape(-1).astype(np.uint32)
    data = oracle.encode_delta4(x)
    g = oracle.decode(data)
    assert np.array_equal(g, np.concatenate([x[:4], x[4:] - x[:-4]]))
    assert np.array_equal(oracle.decode_delta4(data, x.size), x)
    for prev4 in ([1, 2, 3, 4], rng.integers(0, 1 << 32, 4, dtype=np.uint64).astype(np.uint32)):
        assert np.array_equal(oracle.decode_delta4(oracle.encode_delta4(x, prev4), x.size, prev4), x)


def test_delta4_short_lists_and_wrap():
    for n in range(0, 9):
        x = (np.arange(n, dtype=np.uint64) * 0x9E3779B9 & MASK32).astype(np.uint32)
        data = oracle.encode_delta4(x, prev4=[MASK32] * 4)
        assert np.array_equal(oracle.decode_delta4(data, n, prev4=[MASK32] * 4), x)
        g = oracle.decode(data)
        before = np.concatenate([np.full(4, MASK32, dtype=np.uint64), x.astype(np.uint64)])[:n]
        want = (x.astype(np.uint64) + np.uint64(1 << 32) - before) & np.uint64(MASK32)
        assert np.array_equal(g, want.astype(np.uint32))
