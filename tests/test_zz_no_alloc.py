"""vbyte_decode_noalloc: the decode entry point that allocates nothing and
keeps its scratch in the library's fixed device array.

Some callers cannot allocate device memory: every byte belongs to another
allocator, or a serving loop cannot take cudaMalloc's implicit device
synchronisation or an out-of-memory failure mid-request.  This form serves
them.  Its output must equal the oracle's decoding (Algorithm 1, Sec. 2, and
the differential running sum) and that of vbyte_decode / vbyte_decode_delta
on the same input, call after call: every call shares the array, so a second
call on a different input would expose scratch state left over from the
first.  The file is named so that pytest collects it last."""
import numpy as np
import pytest

import oracle
from paper_1503_07387_gb300 import inputs, vbyte


def test_rejects_inputs_above_the_maximum():
    # checked before any CUDA call, so no GPU is needed
    lib = vbyte.load()
    rc = lib.vbyte_decode_noalloc(None, vbyte.NOALLOC_MAX_BYTES + 1, None, 0, 0, 0, None, None)
    assert rc == vbyte.ETOOBIG
    assert b"VBYTE_NOALLOC_MAX_BYTES" in lib.vbyte_strerror(rc)


def _case(gen, n, delta, seed, prev):
    """Bytes from the oracle's encoder and the oracle's decoding of them."""
    v = getattr(inputs, gen)(n, seed=seed)
    b = oracle.encode(v)           # the integers (gaps, in delta mode) as stored
    want = oracle.decode_delta(b, v.size, prev=prev) if delta else oracle.decode(b, v.size)
    assert want.size == v.size
    return b, want


def _device(b, offset=0):
    import torch
    t = torch.zeros(b.size + offset, dtype=torch.uint8, device="cuda")
    t[offset:] = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    return t[offset:]


@pytest.mark.gpu
def test_two_calls_in_a_row_match_the_oracle_and_vbyte_decode():
    import torch
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    cases = [("geometric_gaps", 5_000_000, True, 11, 3, 0),          # several chunks, unaligned input
             ("uniform_bits", 300_001, False, 12, 0, 0),             # smaller, different: stale scratch shows
             ("one_two_byte_mix", 2_000_003, True, 13, 7, 0xFFFFFF00),
             ("full_range", 77_777, False, 14, 1, 0)]
    for gen, n, delta, seed, off, prev in cases:
        b, want = _case(gen, n, delta, seed, prev)
        d = _device(b, off)
        ref = vbyte.decode_delta(d, n, prev) if delta else vbyte.decode(d, n)
        assert vbyte.get_status() == 0
        assert np.array_equal(ref.cpu().numpy(), want), (gen, n, delta)
        for _ in range(2):
            got = torch.full((n + 8,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
            vbyte.decode_noalloc(d, n, delta=delta, prev=prev, out=got[:n], status=status)
            torch.cuda.synchronize()
            h = got.cpu().numpy().view(np.uint32)
            assert np.array_equal(h[:n], want), (gen, n, delta)
            assert np.all(h[n:] == 0x5A5A5A5A), "written past n"
        assert int(status.item()) == 0


@pytest.mark.gpu
def test_maximum_size_and_errors():
    import torch
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    # exactly the maximum, starting 15 bytes past a 16-byte boundary (the
    # largest tile count the scratch must hold); one-byte codes, so the
    # values are the bytes themselves (Algorithm 1's first step)
    nb = vbyte.NOALLOC_MAX_BYTES
    g = torch.Generator(device="cuda").manual_seed(5)
    raw = torch.randint(0, 128, (nb + 15,), dtype=torch.uint8, device="cuda", generator=g)
    d = raw[15:]
    ref = vbyte.decode(d, nb)
    got = vbyte.decode_noalloc(d, nb, status=status)
    torch.cuda.synchronize()
    assert torch.equal(got.view(torch.int32), ref.view(torch.int32)) and int(status.item()) == 0
    assert torch.equal(got.view(torch.int32), d.to(torch.int32))
    assert vbyte.get_status() == 0
    # one byte more is refused before any work is queued
    big = torch.zeros(nb + 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(vbyte.VByteError, match="VBYTE_NOALLOC_MAX_BYTES"):
        vbyte.decode_noalloc(big, 1)
    # data errors land in the caller's status word, with the oracle's bits
    bad = np.array([0x81, 0x01, 0x85], dtype=np.uint8)
    dbad = torch.from_numpy(bad).cuda()
    vbyte.decode_noalloc(dbad, 2, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == oracle.validate(bad, 2) == vbyte.ERR_TRUNCATED | vbyte.ERR_COUNT_MISMATCH
    status.zero_()
    vbyte.decode_noalloc(dbad[:2], 3, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == oracle.validate(bad[:2], 3) == vbyte.ERR_COUNT_MISMATCH
    # without a status word the errors are discarded: a truncated stream
    # still writes the values it defines, the stream's own status word sees
    # nothing, and a following call with a fresh word reads 0
    trunc = np.array([0x05, 0x81, 0x01, 0x7F, 0x83], dtype=np.uint8)   # 5, 129, 127, then a cut integer
    assert oracle.validate(trunc, 3) == vbyte.ERR_TRUNCATED
    out = torch.zeros(3, dtype=torch.int32, device="cuda")
    vbyte.decode_noalloc(torch.from_numpy(trunc).cuda(), 3, out=out, status=None)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), oracle.decode(trunc[:4]))
    assert vbyte.get_status() == 0
    fresh = torch.zeros(1, dtype=torch.int32, device="cuda")
    ok = np.array([0x05, 0x81, 0x01], dtype=np.uint8)
    vbyte.decode_noalloc(torch.from_numpy(ok).cuda(), 2, status=fresh)
    torch.cuda.synchronize()
    assert int(fresh.item()) == 0
