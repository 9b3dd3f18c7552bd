"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers; it holds none of the method's
arithmetic (no encoding, no gap formation, no prefix sums).  Both the library's
tests/benchmark and the CPU oracle consume what it returns.

The paper measured on ClueWeb09 category-B posting lists (Sec. 5): about 50M
documents, one sorted list of document ids per frequent word, grouped by length
class 2^K..2^(K+1)-1, 8 to 16 bits per integer after compression.  That data set
is not available here; the generators below stand in for its shapes.

Every generator takes a ``seed`` and sizes, and returns numpy arrays:
  * ``uniform_bits``      values below 2^b with b uniform in {1..32}
  * ``geometric_gaps``    gaps 1 + Geometric(p) (support of Geometric is k >= 1),
                          first gap 0 (so x_1 = 0)
  * ``uniform_gaps``      gaps uniform in [lo, hi]
  * ``one_two_byte_mix``  per value, a fair coin picks [0, 2^7) or [2^7, 2^14)
  * ``full_range``        uniform uint32
  * ``posting_lists``     rank-Zipf list lengths max(1, floor(cap / r)), each list
                          a sorted sample without replacement from [0, universe)
  * ``query_stream``      Poisson arrival times; each query names k distinct
                          lists drawn with probability proportional to length
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "uniform_bits", "geometric_gaps", "uniform_gaps", "one_two_byte_mix",
    "full_range", "posting_lists", "query_stream", "length_class_lists",
]


def uniform_bits(n: int = 1_000_000, seed: int = 0) -> np.ndarray:
    """Each value uniform below 2^b, b uniform in {1..32} (code lengths 1..5)."""
    rng = np.random.default_rng(seed)
    b = rng.integers(1, 33, size=n, dtype=np.int64)
    hi = np.left_shift(np.uint64(1), b.astype(np.uint64))
    return rng.integers(0, hi, dtype=np.uint64).astype(np.uint32)


def geometric_gaps(n: int = 1 << 26, p: float = 0.1, seed: int = 0) -> np.ndarray:
    """Gaps 1 + G with G ~ Geometric(p) on {1, 2, ...}; the first gap is 0."""
    rng = np.random.default_rng(seed)
    g = rng.geometric(p, size=n).astype(np.uint32)
    g += np.uint32(1)
    if n:
        g[0] = 0
    return g


def uniform_gaps(n: int = 1 << 26, lo: int = 1, hi: int = 300, seed: int = 1) -> np.ndarray:
    """Gaps uniform in [lo, hi] (a dense mix of one- and two-byte codes)."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=n, dtype=np.uint32)


def one_two_byte_mix(n: int = 1 << 28, seed: int = 0) -> np.ndarray:
    """Per value a fair coin: uniform in [0, 2^7) or uniform in [2^7, 2^14)."""
    rng = np.random.default_rng(seed)
    coin = rng.integers(0, 2, size=n, dtype=np.uint8).astype(bool)
    small = rng.integers(0, 1 << 7, size=n, dtype=np.uint32)
    big = rng.integers(1 << 7, 1 << 14, size=n, dtype=np.uint32)
    return np.where(coin, big, small).astype(np.uint32)


def full_range(n: int = 1 << 28, seed: int = 0) -> np.ndarray:
    """Uniform over all of uint32 (mostly five-byte codes)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)


def uniform_bits64(n: int = 1 << 26, seed: int = 0) -> np.ndarray:
    """uint64 values of every bit width 0..64, equally often (code lengths
    1..10 of the 64-bit form)."""
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 65, size=n).astype(np.uint64)
    top = rng.integers(0, 1 << 63, size=n, dtype=np.uint64) * np.uint64(2) \
        + rng.integers(0, 2, size=n, dtype=np.uint64)
    v = top >> (np.uint64(64) - np.maximum(bits, np.uint64(1)))
    v[bits == 0] = 0
    return v


def posting_lists(num_lists: int = 100_000, universe: int = 50_000_000,
                  cap: int = 10_000_000, seed: int = 0, min_len: int = 1):
    """Rank-Zipf(s=1) posting lists.

    List lengths are max(min_len, floor(cap / r)) for ranks r = 1..num_lists,
    clamped to [1, min(cap, universe)], in an order shuffled by the seed.  Each
    list is a sorted sample without replacement from [0, universe).

    Returns (ids, val_off): ids is uint32 with all lists laid end to end,
    val_off is uint64 of length num_lists + 1.
    """
    rng = np.random.default_rng(seed)
    r = np.arange(1, num_lists + 1, dtype=np.int64)
    lengths = np.maximum(cap // r, min_len)
    lengths = np.clip(lengths, 1, min(cap, universe))
    lengths = lengths[rng.permutation(num_lists)]
    val_off = np.zeros(num_lists + 1, dtype=np.uint64)
    np.cumsum(lengths, out=val_off[1:])
    ids = np.empty(int(val_off[-1]), dtype=np.uint32)
    for j in range(num_lists):
        s = rng.choice(universe, size=int(lengths[j]), replace=False)
        s.sort()
        ids[int(val_off[j]):int(val_off[j + 1])] = s
    return ids, val_off


def length_class_lists(num_lists: int, max_class: int = 12, universe: int = 1 << 22,
                       seed: int = 0):
    """Small posting lists spread over length classes 2^K..2^(K+1)-1 (Sec. 5)."""
    rng = np.random.default_rng(seed)
    k = rng.integers(0, max_class + 1, size=num_lists)
    lengths = rng.integers(np.left_shift(1, k), np.left_shift(1, k + 1))
    lengths = np.minimum(lengths, universe)
    val_off = np.zeros(num_lists + 1, dtype=np.uint64)
    np.cumsum(lengths, out=val_off[1:])
    ids = np.empty(int(val_off[-1]), dtype=np.uint32)
    for j in range(num_lists):
        s = rng.choice(universe, size=int(lengths[j]), replace=False)
        s.sort()
        ids[int(val_off[j]):int(val_off[j + 1])] = s
    return ids, val_off


def query_stream(list_lengths, num_queries: int, rate_qps: float, kmin: int = 2,
                 kmax: int = 8, seed: int = 0):
    """Poisson arrivals at rate_qps; each query names k ~ U{kmin..kmax} distinct
    lists drawn with probability proportional to list length.

    Returns (arrival_s, query_off, query_lists): arrival times in seconds from
    0, CSR offsets into query_lists (int64 list indices)."""
    rng = np.random.default_rng(seed)
    lens = np.asarray(list_lengths, dtype=np.float64)
    cdf = np.cumsum(lens / lens.sum())
    cdf[-1] = 1.0
    arrivals = np.cumsum(rng.exponential(1.0 / rate_qps, size=num_queries))
    ks = rng.integers(kmin, kmax + 1, size=num_queries)
    qoff = np.zeros(num_queries + 1, dtype=np.int64)
    np.cumsum(ks, out=qoff[1:])
    qlists = np.empty(int(qoff[-1]), dtype=np.int64)
    for q in range(num_queries):
        # draws proportional to length, repeated draws of the same list rejected
        picked: list[int] = []
        while len(picked) < ks[q]:
            for c in np.searchsorted(cdf, rng.random(2 * kmax), side="right"):
                c = int(min(c, lens.size - 1))
                if c not in picked:
                    picked.append(c)
                    if len(picked) == ks[q]:
                        break
        qlists[qoff[q]:qoff[q + 1]] = picked
    return arrivals, qoff, qlists
