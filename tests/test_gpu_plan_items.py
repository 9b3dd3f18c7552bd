"""GPU parity of tuned batched plans, every candidate kernel forced in turn:
list items (whole lists of at most C bytes in one pass, longer ones cut into
C-byte chunks decoded after a count and a per-list scan) for several C and
both block sizes, and the segmented stream kernel -- values and status bits
against the oracle's per-list Algorithm 1 (with the running sum from each
list's x_0 in differential mode)."""
import numpy as np
import pytest

import oracle
from paper_1503_07387_gb300 import inputs, vbyte

pytestmark = pytest.mark.gpu

SENTINEL = 0xA5A5A5A5
GUARD = 37
CHOICES = [(1, 4096, 128), (1, 8 << 10, 256), (1, 32 << 10, 128), (1, 128 << 10, 256), (0, 0, 256),
           (2, 16 << 10, 256), (2, 4096, 128)]


def _cid(c):
    if c[0] == 0:
        return "segmented"
    return f"{'table' if c[0] == 2 else 'items'}{c[1] >> 10}k_t{c[2]}"


@pytest.fixture(params=CHOICES, ids=_cid)
def choice(request):
    vbyte.debug_force_plan(*request.param)
    yield request.param
    vbyte.debug_force_plan(-1)


def _plan(b, bo, vo, delta, prev=None, offset=0, autotune=False):
    import torch
    n = int(vo[-1])
    t = torch.zeros(b.size + offset + 1, dtype=torch.uint8, device="cuda")
    if b.size:
        t[offset:offset + b.size] = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    d = t[offset:offset + b.size]
    dbo = torch.from_numpy(np.ascontiguousarray(bo, np.uint64).view(np.int64)).cuda()
    dvo = torch.from_numpy(np.ascontiguousarray(vo, np.uint64).view(np.int64)).cuda()
    dp = None
    if delta and prev is not None:
        dp = torch.from_numpy(np.ascontiguousarray(prev, np.uint32).view(np.int32)).cuda()
    obuf = torch.from_numpy(np.full(n + GUARD, SENTINEL, np.uint32).view(np.int32)).cuda()
    plan = vbyte.Plan(d, dbo, dvo, n, delta, prev=dp, out=obuf[:n], autotune=autotune)
    return plan, obuf, (t, dbo, dvo, dp)


def _run(plan, obuf, n, reps=2):
    import torch
    for _ in range(reps):
        obuf[:n].fill_(0x12345678)
        plan.launch()
        torch.cuda.synchronize()
    st = plan.get_status()
    host = obuf.cpu().numpy().view(np.uint32)
    assert np.all(host[n:] == SENTINEL), "write past n"
    return host[:n], st


def _check(ids, vo, delta, prev=None, offset=0):
    b, bo = oracle.encode_batched(ids, vo, delta, prev)
    want, st = oracle.decode_batched(b, bo, vo, delta, prev)
    assert st == 0
    plan, obuf, keep = _plan(b, bo, vo, delta, prev, offset)
    got, status = _run(plan, obuf, int(vo[-1]))
    plan.close()
    assert status == 0
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, (bad[:10], got[bad[:10]], want[bad[:10]])


@pytest.mark.parametrize("delta", [False, True])
def test_length_classes(choice, delta):
    ids, vo = inputs.length_class_lists(3000, max_class=16, seed=50)
    prev = inputs.full_range(vo.size - 1, seed=51)
    _check(ids, vo, delta, prev)


@pytest.mark.parametrize("offset", [0, 1, 7, 15])
def test_unaligned_input_and_tiny_lists(choice, offset):
    rng = np.random.default_rng(52 + offset)
    lengths = rng.integers(0, 40, 5000)
    lengths[::97] = rng.integers(20000, 60000, lengths[::97].size)   # long ones among them
    vo = np.zeros(lengths.size + 1, np.uint64)
    np.cumsum(lengths, out=vo[1:])
    ids = inputs.uniform_bits(int(vo[-1]), seed=53)
    _check(ids, vo, True, inputs.full_range(lengths.size, seed=54), offset)
    _check(ids, vo, False, None, offset)


def test_zipf_posting_lists(choice):
    ids, vo = inputs.posting_lists(4000, universe=1 << 24, cap=400000, seed=55)
    _check(ids, vo, True, inputs.full_range(4000, seed=56))


def test_status_bits_match_the_oracle(choice):
    ids, vo = inputs.length_class_lists(400, max_class=15, seed=57)
    b, bo = oracle.encode_batched(ids, vo, True, None)
    L = vo.size - 1
    lens = np.diff(bo.astype(np.int64))
    long_j = int(np.argmax(lens))
    # truncate the longest list (its last byte gets the high bit) and miscount another
    b = b.copy()
    b[int(bo[long_j + 1]) - 1] |= 0x80
    vo2 = vo.copy()
    j2 = (long_j + 7) % L
    vo2[j2 + 1:] += 1
    vo2[-1] -= 1   # keep the total
    want, st = oracle.decode_batched(b, bo, vo2, True, None)
    plan, obuf, keep = _plan(b, bo, vo2, True)
    got, status = _run(plan, obuf, int(vo2[-1]), reps=1)
    plan.close()
    assert st & vbyte.ERR_TRUNCATED and st & vbyte.ERR_COUNT_MISMATCH
    assert status == st


def test_describe_reports_a_mode_per_class(choice):
    ids, vo = inputs.length_class_lists(500, max_class=16, seed=58)
    b, bo = oracle.encode_batched(ids, vo, False, None)
    plan, obuf, keep = _plan(b, bo, vo, False)
    info = plan.describe()
    plan.close()
    assert sum(c["lists"] for c in info["classes"]) == vo.size - 1
    assert sum(c["values"] for c in info["classes"]) == int(vo[-1])
    kernel, chunk, tpb = choice
    for c in info["classes"]:
        if kernel == 0:
            assert c["mode"] == "segmented stream"
        else:
            whole = (2 << c["bytes_class"]) - 1 <= chunk
            assert c["mode"] == ("single pass" if whole else "count then decode")
    if kernel >= 1:
        assert info["chunk_bytes"] == chunk and info["threads_per_block"] == tpb
        assert info["kernel"] == ("list items, table-driven" if kernel == 2 else "list items")


@pytest.mark.slow
def test_full_size_posting_lists_tuned():
    import torch
    ids, vo = inputs.posting_lists()
    prev = inputs.full_range(vo.size - 1, seed=17)
    b, bo = oracle.encode_batched(ids, vo, True, prev)
    del ids
    want, st = oracle.decode_batched(b, bo, vo, True, prev)
    assert st == 0
    plan, obuf, keep = _plan(b, bo, vo, True, prev, autotune=True)
    n = int(vo[-1])
    got, status = _run(plan, obuf, n, reps=1)
    info = plan.describe()
    plan.close()
    assert status == 0 and info["tuned"] in ("timed", "cached for the length class")
    assert np.array_equal(got, want)
