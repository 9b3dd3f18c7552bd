"""Plain scalar CPU oracle for VByte decoding (arXiv 1503.07387).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / reference leg may import this package.  It
shares no code with the CUDA path and does not import the library package.

The arithmetic lives in ``vbyte_oracle.c`` (Algorithm 1 of Sec. 2, the
differential rule of Sec. 1/2, and the data-error contract); this module only
compiles it with the host C compiler and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "vbyte_oracle.c"), os.path.join(_HERE, "vbyte_oracle.h")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

ERR_MALFORMED_LONG = 1
ERR_TRUNCATED = 2
ERR_COUNT_MISMATCH = 4

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` with gcc (no SIMD flags)."""
    stale = force or not os.path.exists(_LIB_PATH) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB_PATH) for s in _SRC)
    if stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
               _SRC[0], "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    S = ctypes.c_size_t
    U32 = ctypes.c_uint32
    lib.oracle_encode_one.argtypes = [U32, P]
    lib.oracle_encode_one.restype = S
    lib.oracle_encode.argtypes = [P, S, P]
    lib.oracle_encode.restype = S
    lib.oracle_encode_delta.argtypes = [P, S, U32, P]
    lib.oracle_encode_delta.restype = S
    lib.oracle_decode.argtypes = [P, S, P, S]
    lib.oracle_decode.restype = S
    lib.oracle_decode_delta.argtypes = [P, S, P, S, U32]
    lib.oracle_decode_delta.restype = S
    lib.oracle_encode_delta_m1.argtypes = [P, S, U32, P]
    lib.oracle_encode_delta_m1.restype = S
    lib.oracle_decode_delta_m1.argtypes = [P, S, P, S, U32]
    lib.oracle_decode_delta_m1.restype = S
    lib.oracle_validate.argtypes = [P, S, S]
    lib.oracle_validate.restype = U32
    lib.oracle_encode_delta4.argtypes = [P, S, P, P]
    lib.oracle_encode_delta4.restype = S
    lib.oracle_decode_delta4.argtypes = [P, S, P, S, P]
    lib.oracle_decode_delta4.restype = S
    U64 = ctypes.c_uint64
    lib.oracle_encode64_one.argtypes = [U64, P]
    lib.oracle_encode64_one.restype = S
    lib.oracle_encode64.argtypes = [P, S, P]
    lib.oracle_encode64.restype = S
    lib.oracle_encode_delta64.argtypes = [P, S, U64, P]
    lib.oracle_encode_delta64.restype = S
    lib.oracle_decode64.argtypes = [P, S, P, S]
    lib.oracle_decode64.restype = S
    lib.oracle_decode_delta64.argtypes = [P, S, P, S, U64]
    lib.oracle_decode_delta64.restype = S
    lib.oracle_validate64.argtypes = [P, S, S]
    lib.oracle_validate64.restype = U32
    lib.oracle_decode_batched.argtypes = [P, P, P, S, ctypes.c_int, P, P]
    lib.oracle_decode_batched.restype = U32
    lib.oracle_encode_batched.argtypes = [P, P, S, ctypes.c_int, P, P, P]
    lib.oracle_encode_batched.restype = S
    lib.oracle_decode_batched_mt.argtypes = [P, P, P, S, ctypes.c_int, P, P, ctypes.c_int]
    lib.oracle_decode_batched_mt.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a.size else None


def _u8(b) -> np.ndarray:
    if isinstance(b, (bytes, bytearray)):
        return np.frombuffer(bytes(b), dtype=np.uint8)
    a = np.ascontiguousarray(b, dtype=np.uint8)
    return a


def encode(values) -> np.ndarray:
    """VByte-encode uint32 values (Sec. 1, Table 1)."""
    v = np.ascontiguousarray(values, dtype=np.uint32)
    out = np.empty(5 * v.size, dtype=np.uint8)
    nb = _load().oracle_encode(_ptr(v), v.size, _ptr(out))
    return out[:nb].copy()


def encode_delta(values, prev: int = 0) -> np.ndarray:
    """Encode the gaps x_i - x_{i-1} (mod 2^32), x_0 = prev (Sec. 1)."""
    v = np.ascontiguousarray(values, dtype=np.uint32)
    out = np.empty(5 * v.size, dtype=np.uint8)
    nb = _load().oracle_encode_delta(_ptr(v), v.size, ctypes.c_uint32(prev & 0xFFFFFFFF), _ptr(out))
    return out[:nb].copy()


def decode(data, n: int | None = None) -> np.ndarray:
    """Algorithm 1.  Returns every integer it appends (n is only a capacity hint)."""
    b = _u8(data)
    cap = b.size if n is None else max(n, 0)
    out = np.empty(max(cap, 1), dtype=np.uint32)
    cnt = _load().oracle_decode(_ptr(b), b.size, _ptr(out), cap)
    if cnt > cap:
        out = np.empty(cnt, dtype=np.uint32)
        cnt = _load().oracle_decode(_ptr(b), b.size, _ptr(out), cnt)
    return out[:cnt].copy()


def decode_delta(data, n: int | None = None, prev: int = 0) -> np.ndarray:
    """Algorithm 1 with the running sum of Sec. 2 (uint32 wrap-around)."""
    b = _u8(data)
    cap = b.size if n is None else max(n, 0)
    out = np.empty(max(cap, 1), dtype=np.uint32)
    p = ctypes.c_uint32(prev & 0xFFFFFFFF)
    cnt = _load().oracle_decode_delta(_ptr(b), b.size, _ptr(out), cap, p)
    if cnt > cap:
        out = np.empty(cnt, dtype=np.uint32)
        cnt = _load().oracle_decode_delta(_ptr(b), b.size, _ptr(out), cnt, p)
    return out[:cnt].copy()


def encode_delta_m1(values, prev: int = 0) -> np.ndarray:
    """The differential variant of Sec. 1 for lists without repeated values:
    store x_1 - x_0, then x_i - x_{i-1} - 1 (mod 2^32), x_0 = prev."""
    v = np.ascontiguousarray(values, dtype=np.uint32)
    out = np.empty(5 * v.size, dtype=np.uint8)
    nb = _load().oracle_encode_delta_m1(_ptr(v), v.size, ctypes.c_uint32(prev & 0xFFFFFFFF), _ptr(out))
    return out[:nb].copy()


def decode_delta_m1(data, n: int | None = None, prev: int = 0) -> np.ndarray:
    """Algorithm 1 with the running sum of that variant: one more for every
    value after the first (uint32 wrap-around)."""
    b = _u8(data)
    cap = b.size if n is None else max(n, 0)
    out = np.empty(max(cap, 1), dtype=np.uint32)
    p = ctypes.c_uint32(prev & 0xFFFFFFFF)
    cnt = _load().oracle_decode_delta_m1(_ptr(b), b.size, _ptr(out), cap, p)
    if cnt > cap:
        out = np.empty(cnt, dtype=np.uint32)
        cnt = _load().oracle_decode_delta_m1(_ptr(b), b.size, _ptr(out), cnt, p)
    return out[:cnt].copy()


def validate(data, n: int) -> int:
    """Status bits of the data-error contract for a stream expected to hold n values."""
    b = _u8(data)
    return int(_load().oracle_validate(_ptr(b), b.size, n))


def _prev4(prev4):
    if prev4 is None:
        return None
    p = np.ascontiguousarray(prev4, dtype=np.uint32)
    if p.size != 4:
        raise ValueError("prev4 holds the four values before the list")
    return p


def encode_delta4(values, prev4=None) -> np.ndarray:
    """The blocked differences of Sec. 1: x_i - x_{i-4} (mod 2^32), the four
    values before the list being prev4 (zeros: the paper's x_1..x_4 as is)."""
    v = np.ascontiguousarray(values, dtype=np.uint32)
    p = _prev4(prev4)
    out = np.empty(5 * v.size, dtype=np.uint8)
    nb = _load().oracle_encode_delta4(_ptr(v), v.size, None if p is None else _ptr(p), _ptr(out))
    return out[:nb].copy()


def decode_delta4(data, n: int | None = None, prev4=None) -> np.ndarray:
    """Algorithm 1, then x_i = g_i + x_{i-4} (mod 2^32)."""
    b = _u8(data)
    p = _prev4(prev4)
    cap = b.size if n is None else max(n, 0)
    out = np.empty(max(cap, 1), dtype=np.uint32)
    pp = None if p is None else _ptr(p)
    cnt = _load().oracle_decode_delta4(_ptr(b), b.size, _ptr(out), cap, pp)
    if cnt > cap:
        out = np.empty(cnt, dtype=np.uint32)
        cnt = _load().oracle_decode_delta4(_ptr(b), b.size, _ptr(out), cnt, pp)
    return out[:cnt].copy()


MASK64 = (1 << 64) - 1


def encode64(values) -> np.ndarray:
    """VByte-encode uint64 values (Sec. 1: the format read for 64-bit
    integers, up to ten bytes each)."""
    v = np.ascontiguousarray(values, dtype=np.uint64)
    out = np.empty(10 * v.size, dtype=np.uint8)
    nb = _load().oracle_encode64(_ptr(v), v.size, _ptr(out))
    return out[:nb].copy()


def encode_delta64(values, prev: int = 0) -> np.ndarray:
    """Encode the gaps x_i - x_{i-1} (mod 2^64), x_0 = prev."""
    v = np.ascontiguousarray(values, dtype=np.uint64)
    out = np.empty(10 * v.size, dtype=np.uint8)
    nb = _load().oracle_encode_delta64(_ptr(v), v.size, ctypes.c_uint64(prev & MASK64), _ptr(out))
    return out[:nb].copy()


def _decode64(fn, data, n, *extra):
    b = _u8(data)
    cap = b.size if n is None else max(n, 0)
    out = np.empty(max(cap, 1), dtype=np.uint64)
    cnt = fn(_ptr(b), b.size, _ptr(out), cap, *extra)
    if cnt > cap:
        out = np.empty(cnt, dtype=np.uint64)
        cnt = fn(_ptr(b), b.size, _ptr(out), cnt, *extra)
    return out[:cnt].copy()


def decode64(data, n: int | None = None) -> np.ndarray:
    """Algorithm 1 read for uint64 (ten steps, the tenth byte taken whole)."""
    return _decode64(_load().oracle_decode64, data, n)


def decode_delta64(data, n: int | None = None, prev: int = 0) -> np.ndarray:
    """decode64 with the running sum from prev (uint64 wrap-around)."""
    return _decode64(_load().oracle_decode_delta64, data, n, ctypes.c_uint64(prev & MASK64))


def validate64(data, n: int) -> int:
    """The data-error contract for uint64 streams: a run of ten or more bytes
    with the high bit set, a final byte with it set, a terminator count other
    than n."""
    b = _u8(data)
    return int(_load().oracle_validate64(_ptr(b), b.size, n))


def encode64_one(v: int) -> bytes:
    buf = (ctypes.c_uint8 * 10)()
    k = _load().oracle_encode64_one(ctypes.c_uint64(v & MASK64), buf)
    return bytes(buf[:k])


def encode_batched(values, val_off, delta: bool, prev=None):
    """Encode lists laid end to end; returns (bytes, byte_off)."""
    v = np.ascontiguousarray(values, dtype=np.uint32)
    vo = np.ascontiguousarray(val_off, dtype=np.uint64)
    L = vo.size - 1
    pv = None if prev is None else np.ascontiguousarray(prev, dtype=np.uint32)
    out = np.empty(5 * v.size + 1, dtype=np.uint8)
    bo = np.empty(L + 1, dtype=np.uint64)
    nb = _load().oracle_encode_batched(_ptr(v), _ptr(vo), L, int(delta),
                                       None if pv is None else _ptr(pv), _ptr(out), _ptr(bo))
    return out[:nb].copy(), bo


def decode_batched(data, byte_off, val_off, delta: bool, prev=None, threads: int = 1):
    """Decode every list on its own (Algorithm 1 per list).  Returns (values, status);
    status is computed only on the single-threaded path."""
    b = _u8(data)
    bo = np.ascontiguousarray(byte_off, dtype=np.uint64)
    vo = np.ascontiguousarray(val_off, dtype=np.uint64)
    L = bo.size - 1
    pv = None if prev is None else np.ascontiguousarray(prev, dtype=np.uint32)
    out = np.zeros(int(vo[-1]) if vo.size else 0, dtype=np.uint32)
    lib = _load()
    if threads <= 1:
        st = lib.oracle_decode_batched(_ptr(b), _ptr(bo), _ptr(vo), L, int(delta),
                                       None if pv is None else _ptr(pv), _ptr(out))
        return out, int(st)
    lib.oracle_decode_batched_mt(_ptr(b), _ptr(bo), _ptr(vo), L, int(delta),
                                 None if pv is None else _ptr(pv), _ptr(out), int(threads))
    return out, None


def encode_one(v: int) -> bytes:
    buf = (ctypes.c_uint8 * 5)()
    k = _load().oracle_encode_one(ctypes.c_uint32(v & 0xFFFFFFFF), buf)
    return bytes(buf[:k])


if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv)
    print(_LIB_PATH)
