"""The table-driven step of Sec. 4 (Masked VByte), as the library builds it:
a 2^12-entry table from the 12-bit mask of the next 12 bytes' high bits to
(bytes consumed, one of 170 cases).  Pinned on the CPU to the paper's case
counts (2^6 + 3^4 + 5^2 = 64 + 81 + 25 = 170) and to Algorithm 1: for every
one of the 4096 masks, bytes with those high bits decode by the table's step
exactly as the oracle decodes them."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1503_07387_gb300 import vbyte

ENTRIES, CASES = vbyte.table()


def lengths_of(mask):
    """Lengths of the integers that end within the 12 bytes, in order."""
    out, start = [], 0
    for b in range(12):
        if not (mask >> b) & 1:
            out.append(b + 1 - start)
            start = b + 1
    return out


def case_lengths(i):
    d = int(CASES[i])
    return [(d >> (3 + 3 * t)) & 7 for t in range(d & 7)]


def test_exactly_170_cases_in_three_groups():
    ids = {int(e) >> 4 for e in ENTRIES if int(e) & 15 and int(e) >> 4 != 255}
    assert ids == set(range(170))
    assert len([i for i in ids if i < 64]) == 2 ** 6 == 64
    assert len([i for i in ids if 64 <= i < 145]) == 3 ** 4 == 81
    assert len([i for i in ids if 145 <= i < 170]) == 5 ** 2 == 25


def test_case_descriptors():
    # 64 patterns of six lengths in {1, 2}, 81 of four in {1, 2, 3}, 25 of two in 1..5, all distinct
    pats = [tuple(case_lengths(i)) for i in range(170)]
    assert len(set(pats)) == 170
    assert set(pats[:64]) == set(itertools.product((1, 2), repeat=6))
    assert set(pats[64:145]) == set(itertools.product((1, 2, 3), repeat=4))
    assert set(pats[145:]) == set(itertools.product(range(1, 6), repeat=2))
    for i, p in enumerate(pats):
        assert (int(CASES[i]) >> 24) & 15 == sum(p)


def test_every_mask_follows_the_rule():
    for m in range(4096):
        e = int(ENTRIES[m])
        consumed, case = e & 15, e >> 4
        L = lengths_of(m)
        if m == 0:
            assert (consumed, case) == (12, 255)
        elif len(L) >= 6 and max(L[:6]) <= 2:
            assert case < 64 and case_lengths(case) == L[:6]
        elif len(L) >= 4 and max(L[:4]) <= 3:
            assert 64 <= case < 145 and case_lengths(case) == L[:4]
        elif len(L) >= 2 and max(L[:2]) <= 5:
            assert 145 <= case < 170 and case_lengths(case) == L[:2]
        else:
            # an integer of more than five bytes: malformed, nothing consumed
            assert consumed == 0
            continue
        assert 2 <= consumed <= 12 and consumed == sum(case_lengths(case)) if case != 255 else True


def _bytes_for(mask, rng, tail=24):
    """12 bytes whose high bits are the mask, random payloads, then a valid tail."""
    payload = rng.integers(0, 128, 12, dtype=np.uint16)
    head = (payload | (np.array([(mask >> b) & 1 for b in range(12)], np.uint16) << 7)).astype(np.uint8)
    rest = oracle.encode(rng.integers(0, 1 << 32, tail, dtype=np.uint64).astype(np.uint32))
    return np.concatenate([head, rest])


def test_every_mask_decodes_as_algorithm_1():
    rng = np.random.default_rng(7)
    for m in range(4096):
        data = _bytes_for(m, rng)
        want = oracle.decode(data)
        got = vbyte.table_decode(data)
        assert np.array_equal(got, want), hex(m)


def test_fig1_and_table1():
    fig1 = np.array([0x80, 0x01, 0x82, 0x03, 0x10, 0x20], np.uint8)
    assert vbyte.table_decode(fig1).tolist() == [128, 386, 16, 32]
    t1 = np.array([1, 2, 4, 128, 256, 512, 16384, 32768], np.uint32)
    assert np.array_equal(vbyte.table_decode(oracle.encode(t1)), t1)


@pytest.mark.parametrize("seed", range(4))
def test_random_streams(seed):
    rng = np.random.default_rng(seed)
    b = rng.integers(1, 33, 20_000)
    v = rng.integers(0, np.left_shift(np.uint64(1), b.astype(np.uint64)), dtype=np.uint64).astype(np.uint32)
    data = oracle.encode(v)
    assert np.array_equal(vbyte.table_decode(data), v)
