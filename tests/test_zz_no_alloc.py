"""vbyte_decode_noalloc: the decode entry point that allocates nothing and
keeps its scratch in the library's fixed device array.

Its output must equal that of vbyte_decode / vbyte_decode_delta on the same
input, call after call: every call shares the array, so a second call on a
different input would expose scratch state left over from the first."""
import ctypes

import numpy as np
import pytest

from paper_1503_07387_gb300 import inputs, vbyte


def test_rejects_inputs_above_the_maximum():
    # checked before any CUDA call, so no GPU is needed
    lib = vbyte.load()
    rc = lib.vbyte_decode_noalloc(None, vbyte.NOALLOC_MAX_BYTES + 1, None, 0, 0, 0, None, None)
    assert rc == vbyte.ETOOBIG
    assert b"VBYTE_NOALLOC_MAX_BYTES" in lib.vbyte_strerror(rc)


def _case(gen, n, delta, seed):
    v = getattr(inputs, gen)(n, seed=seed)
    if delta:
        x = np.cumsum(v.astype(np.uint64)).astype(np.uint32)
        return vbyte.encode_delta(x, prev=0), x.size
    return vbyte.encode(v), v.size


def _device(b, offset=0):
    import torch
    t = torch.zeros(b.size + offset, dtype=torch.uint8, device="cuda")
    t[offset:] = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    return t[offset:]


@pytest.mark.gpu
def test_two_calls_in_a_row_match_vbyte_decode():
    import torch
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    cases = [("geometric_gaps", 5_000_000, True, 11, 3),    # several chunks, unaligned input
             ("uniform_bits", 300_001, False, 12, 0),       # smaller, different: stale scratch shows
             ("one_two_byte_mix", 2_000_003, True, 13, 7),
             ("full_range", 77_777, False, 14, 1)]
    for gen, n, delta, seed, off in cases:
        b, nv = _case(gen, n, delta, seed)
        d = _device(b, off)
        prev = 0
        want = vbyte.decode_delta(d, nv, prev) if delta else vbyte.decode(d, nv)
        assert vbyte.get_status() == 0
        for _ in range(2):
            got = torch.full((nv,), 0xDEADBEEF & 0x7FFFFFFF, dtype=torch.int32, device="cuda")
            vbyte.decode_noalloc(d, nv, delta=delta, prev=prev, out=got, status=status)
            torch.cuda.synchronize()
            assert torch.equal(got, want.view(torch.int32)), (gen, n, delta)
        assert int(status.item()) == 0


@pytest.mark.gpu
def test_maximum_size_and_errors():
    import torch
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    # exactly the maximum, starting 15 bytes past a 16-byte boundary
    # (the largest tile count the scratch must hold)
    nb = vbyte.NOALLOC_MAX_BYTES
    g = torch.Generator(device="cuda").manual_seed(5)
    raw = torch.randint(0, 128, (nb + 15,), dtype=torch.uint8, device="cuda", generator=g)
    d = raw[15:]
    want = vbyte.decode(d, nb)
    got = vbyte.decode_noalloc(d, nb, status=status)
    torch.cuda.synchronize()
    assert torch.equal(got.view(torch.int32), want.view(torch.int32)) and int(status.item()) == 0
    assert vbyte.get_status() == 0
    # one byte more is refused before any work is queued
    big = torch.zeros(nb + 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(vbyte.VByteError, match="VBYTE_NOALLOC_MAX_BYTES"):
        vbyte.decode_noalloc(big, 1)
    # data errors land in the caller's status word
    bad = torch.tensor([0x81, 0x01, 0x85], dtype=torch.uint8, device="cuda")
    vbyte.decode_noalloc(bad, 2, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) & vbyte.ERR_TRUNCATED
    status.zero_()
    vbyte.decode_noalloc(bad[:2], 3, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == vbyte.ERR_COUNT_MISMATCH
    # without a status word the errors are discarded; the output is still written
    vbyte.decode_noalloc(bad[:2], 1, status=None)
    torch.cuda.synchronize()
