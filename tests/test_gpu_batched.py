"""GPU parity of the batched entry points (lists laid end to end, one launch)
with the oracle's per-list Algorithm 1, bit for bit, values and status."""
import numpy as np
import pytest

import oracle
from paper_1503_07387_gb300 import inputs, vbyte

pytestmark = pytest.mark.gpu

SENTINEL = 0xA5A5A5A5
GUARD = 37


def _dev_bytes(b, offset=0):
    import torch
    t = torch.zeros(b.size + offset + 1, dtype=torch.uint8, device="cuda")
    if b.size:
        t[offset:offset + b.size] = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    return t[offset:offset + b.size]


def _dev_u64(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def _gpu(b, bo, vo, delta, prev=None, offset=0):
    import torch
    n = int(vo[-1])
    obuf = torch.from_numpy(np.full(n + GUARD, SENTINEL, np.uint32).view(np.int32)).cuda()
    out = obuf[:n]
    d = _dev_bytes(b, offset)
    if delta:
        dp = None if prev is None else torch.from_numpy(np.ascontiguousarray(prev, np.uint32).view(np.int32)).cuda()
        vbyte.decode_delta_batched(d, _dev_u64(bo), _dev_u64(vo), n, prev=dp, out=out)
    else:
        vbyte.decode_batched(d, _dev_u64(bo), _dev_u64(vo), n, out=out)
    status = vbyte.get_status()
    host = obuf.cpu().numpy().view(np.uint32)
    assert np.all(host[n:] == SENTINEL), "write past n"
    return host[:n], status


def _check(ids, vo, delta, prev=None, offset=0):
    b, bo = oracle.encode_batched(ids, vo, delta, prev)
    want, st = oracle.decode_batched(b, bo, vo, delta, prev)
    assert st == 0
    got, status = _gpu(b, bo, vo, delta, prev, offset)
    assert status == 0
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, (bad[:10], got[bad[:10]], want[bad[:10]])


def _tiny_lists(num_lists, max_len, seed):
    rng = np.random.default_rng(seed)
    lengths = rng.integers(0, max_len + 1, size=num_lists)
    vo = np.zeros(num_lists + 1, np.uint64)
    np.cumsum(lengths, out=vo[1:])
    ids = inputs.uniform_bits(int(vo[-1]), seed=seed + 1)
    return ids, vo


@pytest.mark.parametrize("delta", [False, True])
def test_zipf_posting_lists(delta):
    ids, vo = inputs.posting_lists(3000, universe=1 << 22, cap=20000, seed=4)
    _check(ids, vo, delta)


@pytest.mark.parametrize("delta", [False, True])
def test_tiny_lists_with_empty_ones(delta):
    # 0..3 values per list, codes of 1..5 bytes: several list heads per slice
    ids, vo = _tiny_lists(20000, 3, seed=5)
    prev = inputs.full_range(20000, seed=6) if delta else None
    _check(ids, vo, delta, prev)


def test_one_value_lists_of_one_byte():
    vo = np.arange(9001, dtype=np.uint64)
    ids = (inputs.uniform_bits(9000, seed=7) & 0x7F).astype(np.uint32)
    _check(ids, vo, False)
    _check(np.cumsum(ids, dtype=np.uint64).astype(np.uint32), vo, True, np.arange(9000, dtype=np.uint32))


@pytest.mark.parametrize("delta", [False, True])
def test_length_classes(delta):
    ids, vo = inputs.length_class_lists(400, max_class=12, seed=8)
    prev = np.full(400, 12345, np.uint32) if delta else None
    _check(ids, vo, delta, prev)


@pytest.mark.parametrize("offset", [0, 1, 3, 7, 8, 13, 15])
def test_unaligned_input(offset):
    ids, vo = _tiny_lists(3000, 40, seed=9)
    _check(ids, vo, True, inputs.full_range(3000, seed=10), offset)
    _check(ids, vo, False, None, offset)


def test_long_lists_across_chunks_with_tiny_ones_between():
    # two long lists (several 8 MiB chunks) with tiny lists and empty lists around them
    a = np.cumsum(inputs.uniform_gaps(5_000_000, seed=11), dtype=np.uint64).astype(np.uint32)
    c = np.cumsum(inputs.geometric_gaps(4_000_000, seed=12), dtype=np.uint64).astype(np.uint32)
    parts = [np.array([5], np.uint32), a, np.zeros(0, np.uint32), np.array([1, 2, 3], np.uint32), c,
             np.array([7], np.uint32), np.zeros(0, np.uint32)]
    ids = np.concatenate(parts)
    vo = np.zeros(len(parts) + 1, np.uint64)
    np.cumsum([p.size for p in parts], out=vo[1:])
    prev = np.array([0, 9, 0, 2**32 - 1, 100, 0, 3], np.uint32)
    _check(ids, vo, True, prev)
    _check(ids, vo, False)


def test_list_heads_at_every_offset_of_a_tile_boundary():
    # one-value lists of growing code lengths so that list heads fall on every
    # byte position around several 4 KiB tile boundaries
    rng = np.random.default_rng(13)
    lens = rng.integers(1, 4, size=30000)
    vo = np.zeros(lens.size + 1, np.uint64)
    np.cumsum(lens, out=vo[1:])
    ids = inputs.uniform_bits(int(vo[-1]), seed=14)
    for off in (0, 5, 11):
        _check(ids, vo, True, inputs.full_range(lens.size, seed=15), off)


def test_empty_batches():
    import torch
    z = torch.zeros(0, dtype=torch.uint8, device="cuda")
    one = _dev_u64(np.zeros(1, np.uint64))
    vbyte.decode_batched(z, one, one, 0)
    assert vbyte.get_status() == 0
    four = _dev_u64(np.zeros(4, np.uint64))
    vbyte.decode_delta_batched(z, four, four, 0)
    assert vbyte.get_status() == 0
    vo = _dev_u64(np.array([0, 0, 2], np.uint64))   # two values expected from no bytes
    vbyte.decode_batched(z, _dev_u64(np.zeros(3, np.uint64)), vo, 2)
    assert vbyte.get_status() & vbyte.ERR_COUNT_MISMATCH


def _valid_batch(seed=16):
    ids, vo = _tiny_lists(5000, 30, seed=seed)
    b, bo = oracle.encode_batched(ids, vo, True)
    return ids, vo, b, bo


def test_truncated_list_matches_oracle_status():
    ids, vo, b, bo = _valid_batch()
    # list j ends with a one-byte integer and list j+1 starts with one, so no
    # run of continuation bytes grows across the boundary
    e = bo[1:-1].astype(np.int64)
    ok = (np.diff(bo)[:-1] > 2) & (b[e - 2] < 0x80) & (b[np.minimum(e, b.size - 1)] < 0x80) & (e < b.size)
    cand = np.flatnonzero(ok)
    j = int(cand[cand.size // 2])
    b = b.copy()
    b[int(bo[j + 1]) - 1] |= 0x80   # list j now ends inside an integer
    _, st = oracle.decode_batched(b, bo, vo, True)
    _, status = _gpu(b, bo, vo, True)
    assert st & oracle.ERR_TRUNCATED and status == st


def test_count_mismatch_matches_oracle_status():
    ids, vo, b, bo = _valid_batch()
    vo = vo.copy()
    j = int(np.flatnonzero(np.diff(vo) > 1)[50])
    vo[j + 1] -= 1   # one value moves from list j to list j+1
    _, st = oracle.decode_batched(b, bo, vo, True)
    _, status = _gpu(b, bo, vo, True)
    assert st == oracle.ERR_COUNT_MISMATCH and status == st


def test_malformed_long_run_matches_oracle_status():
    ids, vo, b, bo = _valid_batch()
    b = b.copy()
    j = int(np.flatnonzero(np.diff(bo) > 8)[10])
    b[int(bo[j]):int(bo[j]) + 6] = 0x81   # six continuation bytes
    _, st = oracle.decode_batched(b, bo, vo, False)
    _, status = _gpu(b, bo, vo, False)
    assert st & oracle.ERR_MALFORMED_LONG
    assert status & vbyte.ERR_MALFORMED_LONG
    assert status == st


def test_bad_offsets_are_reported():
    ids, vo, b, bo = _valid_batch()
    bo2 = bo.copy()
    bo2[10], bo2[11] = bo2[11] + 1, bo2[10]   # not non-decreasing
    _, status = _gpu(b, bo2, vo, True)
    assert status & vbyte.ERR_BAD_OFFSETS
    bo3 = bo.copy()
    bo3[-1] -= 1                                # does not end at nbytes
    _, status = _gpu(b, bo3, vo, False)
    assert status & vbyte.ERR_BAD_OFFSETS


def test_full_size_posting_lists():
    # 100,000 rank-Zipf lists over a 5e7 universe (about 1.2e8 values)
    ids, vo = inputs.posting_lists()
    prev = inputs.full_range(vo.size - 1, seed=17)
    for delta in (True, False):
        b, bo = oracle.encode_batched(ids, vo, delta, prev if delta else None)
        want, _ = oracle.decode_batched(b, bo, vo, delta, prev if delta else None, threads=8)
        got, status = _gpu(b, bo, vo, delta, prev if delta else None)
        assert status == 0
        assert np.array_equal(got, want)


def test_plan_autotuned_graph_replay_and_cache():
    import torch
    ids, vo = inputs.posting_lists(2000, universe=1 << 22, cap=50000, seed=18)
    prev = inputs.full_range(2000, seed=19)
    b, bo = oracle.encode_batched(ids, vo, True, prev)
    want, _ = oracle.decode_batched(b, bo, vo, True, prev)
    d, dbo, dvo = _dev_bytes(b), _dev_u64(bo), _dev_u64(vo)
    dp = torch.from_numpy(prev.view(np.int32)).cuda()
    n = int(vo[-1])
    plan = vbyte.Plan(d, dbo, dvo, n, True, prev=dp)
    info = plan.describe()
    assert info["tuned"] in ("timed", "cached for the length class")
    for _ in range(2):
        plan.out.fill_(0)
        plan.launch()
        torch.cuda.synchronize()
        assert np.array_equal(plan.out.cpu().numpy().view(np.uint32), want)
    assert plan.get_status() == 0
    # a second plan of the same length class reuses the tuned parameters
    plan2 = vbyte.Plan(d, dbo, dvo, n, True, prev=dp)
    assert plan2.describe()["tuned"] == "cached for the length class"
    for key in ("kernel", "chunk_bytes", "threads_per_block", "ctas_per_sm"):
        assert plan2.describe().get(key) == info.get(key)
    plan2.launch()
    torch.cuda.synchronize()
    assert np.array_equal(plan2.out.cpu().numpy().view(np.uint32), want)
    plan.close()
    plan2.close()


def test_plan_status_is_its_own():
    ids, vo, b, bo = _valid_batch()
    vo = vo.copy()
    j = int(np.flatnonzero(np.diff(vo) > 1)[20])
    vo[j + 1] -= 1
    plan = vbyte.Plan(_dev_bytes(b), _dev_u64(bo), _dev_u64(vo), int(vo[-1]), False, autotune=False)
    plan.launch()
    assert plan.get_status() == vbyte.ERR_COUNT_MISMATCH
    assert vbyte.get_status() == 0
    plan.close()


@pytest.mark.parametrize("delta", [False, True])
def test_decode_each_matches_oracle(delta):
    ids, vo = inputs.posting_lists(500, universe=1 << 20, cap=5000, seed=20)
    prev = inputs.full_range(500, seed=21) if delta else None
    b, bo = oracle.encode_batched(ids, vo, delta, prev)
    want, _ = oracle.decode_batched(b, bo, vo, delta, prev)
    got = vbyte.decode_each(_dev_bytes(b), bo, vo, int(vo[-1]), delta, prev)
    assert vbyte.get_status() == 0
    assert np.array_equal(got.cpu().numpy().view(np.uint32), want)
