"""vbyte_decode_host on inputs of 128 MiB or more: the input goes to the
device in pieces while earlier pieces are counted, decoded and copied back,
and the values must equal the oracle's (Algorithm 1, Sec. 2, with the
differential running sum from prev), with the status bits of the data-error
contract."""
import numpy as np
import pytest

import oracle
from paper_1503_07387_gb300 import inputs, vbyte

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _pinned(a):
    t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    return t, t.numpy()


@pytest.mark.parametrize("delta,prev", [(False, 0), (True, 0), (True, 0xFFFFFF00)])
def test_geometric_gaps(delta, prev):
    n = 150_000_000   # more than two pieces
    g = inputs.geometric_gaps(n, seed=21)
    data = oracle.encode(g)
    want = oracle.decode_delta(data, n, prev=prev) if delta else oracle.decode(data, n)
    keep, h_in = _pinned(data)
    out_t = torch.empty(n, dtype=torch.int32).pin_memory()
    out = out_t.numpy().view(np.uint32)
    vbyte.decode_host(h_in, n, delta=delta, prev=prev, out=out)
    assert vbyte.get_status() == 0
    bad = np.flatnonzero(out != want)
    assert bad.size == 0, (bad[:5], out[bad[:5]], want[bad[:5]])


def test_mixed_lengths_pageable_and_offset():
    n = 60_000_000
    v = inputs.uniform_bits(n, seed=22)
    data = oracle.encode(v)                          # about 160 MB, pageable host memory
    src = np.zeros(data.size + 3, np.uint8)
    src[3:] = data
    out = np.zeros(n + 5, np.uint32)
    vbyte.decode_host(src[3:], n, delta=True, prev=7, out=out[1:n + 1])
    assert vbyte.get_status() == 0
    assert np.array_equal(out[1:n + 1], oracle.decode_delta(data, n, prev=7))
    assert out[0] == 0 and np.all(out[n + 1:] == 0)


def test_count_mismatch_and_truncation():
    n = 140_000_000
    g = (inputs.uniform_bits(n, seed=23) & 0x3FFF).astype(np.uint32)
    data = oracle.encode(g)
    out = np.zeros(n, np.uint32)
    vbyte.decode_host(data, n - 1000, out=out[:n - 1000])
    assert vbyte.get_status() == oracle.validate(data, n - 1000) == vbyte.ERR_COUNT_MISMATCH
    assert np.array_equal(out[:n - 1000], g[:n - 1000])
    cut = data[:-1].copy()
    cut[-1] |= 0x80
    vbyte.decode_host(cut, n, out=out)
    assert vbyte.get_status() == oracle.validate(cut, n)
