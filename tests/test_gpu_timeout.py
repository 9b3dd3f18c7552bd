"""The bounded waits between CTAs, made to run out on purpose.

A decode launch passes tile counts and running sums between CTAs through
published words (either kernel: count-then-decode or the single pass with a
decoupled look-back).  With vbyte_debug_inject one tile's words are never
published and every wait is bounded by 50 ms: the launch must then return
(no hang, no trap), record VBYTE_ERR_TIMEOUT in the status word, and write
nothing outside [0, n).  Afterwards, with the defaults restored, the same
calls must again decode exactly as the oracle (Algorithm 1, Sec. 2, with the
differential running sum of Sec. 1)."""
import time

import numpy as np
import pytest

import oracle
from paper_1503_07387_gb300 import inputs, vbyte

LIMIT_NS = 50_000_000
CANARY = 0x3C3C3C3C
PAD = 64


@pytest.fixture
def injected():
    yield vbyte.debug_inject
    vbyte.debug_inject(-1, 0)
    vbyte.debug_force_passes(0)


def _padded(n):
    import torch
    buf = torch.full((n + 2 * PAD,), CANARY, dtype=torch.int32, device="cuda")
    return buf, buf[PAD:PAD + n]


def _canaries_intact(buf):
    h = buf.cpu().numpy()
    return bool(np.all(h[:PAD] == CANARY) and np.all(h[-PAD:] == CANARY))


@pytest.mark.gpu
@pytest.mark.parametrize("passes", [1, 2])   # the split kernels have no waits
@pytest.mark.parametrize("n,skip", [(30_000_000, 2048 + 100),   # four chunks; a tile of the second goes missing
                                    (100_000, 3)])              # one chunk
def test_single_stream_wait_runs_out(injected, n, skip, passes):
    import torch
    vbyte.debug_force_passes(passes)
    g = inputs.geometric_gaps(n, seed=3)
    b = oracle.encode(g)
    d = torch.from_numpy(b).cuda()
    buf, out = _padded(n)
    assert vbyte.get_status() == 0
    injected(skip, LIMIT_NS)
    t0 = time.perf_counter()
    vbyte.decode_delta(d, n, prev=5, out=out)
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    st = vbyte.get_status()
    assert st & vbyte.ERR_TIMEOUT, st
    assert elapsed < 20.0
    assert _canaries_intact(buf), "written outside [0, n)"
    # the defaults back: the same call decodes exactly
    injected(-1, 0)
    vbyte.decode_delta(d, n, prev=5, out=out)
    assert vbyte.get_status() == 0
    assert np.array_equal(out.cpu().numpy().view(np.uint32), oracle.decode_delta(b, n, prev=5))
    assert _canaries_intact(buf)


@pytest.mark.gpu
def test_batched_wait_runs_out(injected):
    import torch
    ids, vo = inputs.length_class_lists(3000, max_class=13, seed=4)
    L = vo.size - 1
    prev = inputs.full_range(L, seed=5)
    b, bo = oracle.encode_batched(ids, vo, True, prev)
    want, st = oracle.decode_batched(b, bo, vo, True, prev)
    assert st == 0
    n = int(vo[-1])
    d = torch.from_numpy(b).cuda()
    dbo = torch.from_numpy(bo.view(np.int64)).cuda()
    dvo = torch.from_numpy(vo.view(np.int64)).cuda()
    dp = torch.from_numpy(prev.view(np.int32)).cuda()
    buf, out = _padded(n)
    ntiles = (b.size + 4095) // 4096
    injected(ntiles // 2, LIMIT_NS)
    vbyte.decode_delta_batched(d, dbo, dvo, n, prev=dp, out=out)
    torch.cuda.synchronize()
    assert vbyte.get_status() & vbyte.ERR_TIMEOUT
    assert _canaries_intact(buf)
    injected(-1, 0)
    vbyte.decode_delta_batched(d, dbo, dvo, n, prev=dp, out=out)
    assert vbyte.get_status() == 0
    assert np.array_equal(out.cpu().numpy().view(np.uint32), want)
    assert _canaries_intact(buf)


def test_limit_above_default_refused():
    # checked on the host, before any CUDA call
    with pytest.raises(vbyte.VByteError):
        vbyte.debug_inject(-1, 3_000_000_000)
