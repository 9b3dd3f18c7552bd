"""A caller-owned workspace (vbyte_set_workspace, vbyte_release_stream): the
decoders give the oracle's values with it, never grow it (a call that needs
more returns VBYTE_ENOMEM and queues nothing), keep the stream's status word
in its first bytes, and carry the status bits over when the workspace is
replaced or handed back."""
import numpy as np
import pytest

import oracle
from paper_1503_07387_gb300 import inputs, vbyte

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)


def aligned_buffer(nbytes):
    raw = torch.zeros(nbytes + 256, dtype=torch.uint8, device="cuda")
    off = (-raw.data_ptr()) % 256
    return raw, raw[off:off + nbytes]


def test_caller_workspace_round_trip():
    s = torch.cuda.Stream()
    gaps = inputs.uniform_gaps(300_001, seed=5)
    data = oracle.encode(gaps)
    want = oracle.decode_delta(data, gaps.size, prev=9)
    d = torch.from_numpy(data).cuda()
    out = torch.empty(gaps.size, dtype=torch.uint32, device="cuda")
    raw, ws = aligned_buffer(vbyte.workspace_size(data.size))
    s.wait_stream(torch.cuda.current_stream())
    try:
        vbyte.set_workspace(ws, stream=s)
        vbyte.decode_delta(d, gaps.size, prev=9, out=out, stream=s)
        assert vbyte.get_status(stream=s) == 0
        assert np.array_equal(out.cpu().numpy(), want)

        # a data error lands in the caller's buffer (its first word)
        bad = torch.from_numpy(np.array([5, 0x80, 0x80, 0x80, 0x80, 0x80, 1], dtype=np.uint8)).cuda()
        s.wait_stream(torch.cuda.current_stream())
        vbyte.decode(bad, 2, out=out[:2], stream=s)
        s.synchronize()
        word = int(ws[:4].cpu().numpy().view(np.uint32)[0])
        assert word & vbyte.ERR_MALFORMED_LONG

        # replacing the buffer carries the bits over
        raw2, ws2 = aligned_buffer(vbyte.workspace_size(data.size))
        vbyte.set_workspace(ws2, stream=s)
        assert vbyte.get_status(stream=s) == word

        # an input larger than the workspace is refused, nothing queued
        big = torch.zeros(64 * data.size, dtype=torch.uint8, device="cuda")
        s.wait_stream(torch.cuda.current_stream())
        with pytest.raises(vbyte.VByteError):
            vbyte.decode(big, big.numel(), stream=s)
        assert vbyte.get_status(stream=s) == 0

        # 64-bit decoding with the same workspace
        v = inputs.uniform_bits64(50_000, seed=2)
        d64 = torch.from_numpy(oracle.encode64(v)).cuda()
        s.wait_stream(torch.cuda.current_stream())
        o64 = vbyte.decode64(d64, v.size, stream=s)
        assert vbyte.get_status(stream=s) == 0
        assert np.array_equal(o64.cpu().numpy().view(np.uint64), v)

        # handed back, the library grows its own workspace again
        vbyte.decode(bad, 2, out=out[:2], stream=s)
        vbyte.set_workspace(None, stream=s)
        assert vbyte.get_status(stream=s) & vbyte.ERR_MALFORMED_LONG
        big_vals = inputs.geometric_gaps(1 << 22, seed=1)
        hb = oracle.encode(big_vals)
        db = torch.from_numpy(hb).cuda()
        ob = torch.empty(big_vals.size, dtype=torch.uint32, device="cuda")
        s.wait_stream(torch.cuda.current_stream())
        vbyte.decode(db, big_vals.size, out=ob, stream=s)
        assert vbyte.get_status(stream=s) == 0
        assert np.array_equal(ob.cpu().numpy(), big_vals)
    finally:
        s.synchronize()
        vbyte.release_stream(stream=s)
