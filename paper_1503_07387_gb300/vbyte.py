"""Python binding of libvbyte (ctypes).  Argument marshalling only.

Every step of decoding runs in the library's CUDA kernels; PyTorch supplies
device memory (tensors) and streams.  There is no CPU fallback: if the shared
library cannot be built or loaded, every call raises.

Names mirror the C ABI in ``include/vbyte.h``:

    encode / encode_delta / encode_batched      host encoder (numpy in, numpy out)
    decode(d_bytes, n)                          Algorithm 1 on the GPU (Sec. 2)
    decode_delta(d_bytes, n, prev)              ... plus the prefix sum of Sec. 1/4
    decode_host(h_bytes, n, delta, prev)        host buffers in and out
    decode_noalloc(d_bytes, n, delta, prev)     fixed library scratch, no allocation
    decode_batched(d_bytes, d_bo, d_vo)         lists laid end to end, one launch
    decode_delta_batched(d_bytes, d_bo, d_vo, d_prev)   ... each list differential
    get_status()                                data-error bits of a stream
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import _build

OK, EINVAL, ECUDA, ENOMEM, ETOOBIG = 0, 1, 2, 3, 4
NOALLOC_MAX_BYTES = 128 << 20
ERR_MALFORMED_LONG = 1
ERR_TRUNCATED = 2
ERR_COUNT_MISMATCH = 4
ERR_TIMEOUT = 8
ERR_BAD_OFFSETS = 16

HEADER = os.path.join(_build.INCLUDE, "vbyte.h")
HEADERS = [HEADER, os.path.join(_build.INCLUDE, "vbyte64.h"), os.path.join(_build.INCLUDE, "vbyte_debug.h")]

_lib = None


class VByteError(RuntimeError):
    pass


def _signatures(lib):
    P, S, U32, I = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_int
    sig = {
        "vbyte_max_encoded_size": ([S], S),
        "vbyte_encode": ([P, S, P], S),
        "vbyte_encode_delta": ([P, S, U32, P], S),
        "vbyte_encode_delta_m1": ([P, S, U32, P], S),
        "vbyte_encode_delta_m1_device": ([P, S, U32, P, P, P], I),
        "vbyte_decode_delta_m1": ([P, S, P, S, U32, P], I),
        "vbyte_decode_delta4": ([P, S, P, S, P, P], I),
        "vbyte_encode_delta4": ([P, S, P, P], S),
        "vbyte_encode_batched": ([P, P, S, I, P, P, P], S),
        "vbyte_encode_device": ([P, S, P, P, P], I),
        "vbyte_encode_delta_device": ([P, S, U32, P, P, P], I),
        "vbyte_decode": ([P, S, P, S, P], I),
        "vbyte_decode_delta": ([P, S, P, S, U32, P], I),
        "vbyte_decode_host": ([P, S, P, S, I, U32, P], I),
        "vbyte_decode_batched": ([P, S, P, P, S, P, S, P], I),
        "vbyte_decode_delta_batched": ([P, S, P, P, S, P, S, P, P], I),
        "vbyte_decode_noalloc": ([P, S, P, S, I, U32, P, P], I),
        "vbyte_plan_create": ([P, P, S, P, P, S, P, S, P, I, I, P], I),
        "vbyte_plan_launch": ([P, P], I),
        "vbyte_plan_get_status": ([P, P, P], I),
        "vbyte_plan_describe": ([P, P, P, P, P], I),
        "vbyte_plan_destroy": ([P], None),
        "vbyte_plan_choice": ([P, P, P, P], I),
        "vbyte_plan_class": ([P, I, P, P, P], I),
        "vbyte_debug_force_plan": ([I, ctypes.c_uint64, I], I),
        "vbyte_table": ([P, P], I),
        "vbyte_table_decode": ([P, S, P, S], S),
        "vbyte_decode_each": ([P, P, P, P, S, I, P, P], I),
        "vbyte_server_create": ([P, P, S, P, P, S, I, P, P], I),
        "vbyte_server_submit": ([P, P, S, P], I),
        "vbyte_server_wait": ([P, ctypes.c_uint64, P, P], I),
        "vbyte_server_result": ([P, ctypes.c_uint64, P, P, P], I),
        "vbyte_server_release": ([P, ctypes.c_uint64], I),
        "vbyte_server_replay": ([P, P, P, S, P, P, P], I),
        "vbyte_server_stats": ([P, P, P, P, P], I),
        "vbyte_server_destroy": ([P], None),
        "vbyte_get_status": ([P, P], I),
        "vbyte_strerror": ([I], ctypes.c_char_p),
        "vbyte_workspace_size": ([S], S),
        "vbyte_set_workspace": ([P, P, S], I),
        "vbyte_release_stream": ([P], I),
        "vbyte_debug_inject": ([ctypes.c_longlong, ctypes.c_uint64], I),
        "vbyte_debug_force_passes": ([I], I),
        "vbyte_debug_passes_for": ([S, S, I], I),
        "vbyte_max_encoded_size64": ([S], S),
        "vbyte_encode64": ([P, S, P], S),
        "vbyte_encode_delta64": ([P, S, ctypes.c_uint64, P], S),
        "vbyte_decode64": ([P, S, P, S, P], I),
        "vbyte_decode_delta64": ([P, S, P, S, ctypes.c_uint64, P], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res


def load(build: bool = True):
    """Load (building first if needed) the in-tree libvbyte.so."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise VByteError(f"libvbyte.so not found at {_build.LIB}; run __graft_entry__.build()")
    lib = ctypes.CDLL(_build.LIB)
    _signatures(lib)
    _lib = lib
    return lib


def declared_symbols() -> list[str]:
    """Function names declared in the public headers (vbyte.h, vbyte64.h)."""
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vbyte_[a-z0-9_]+)\s*\(", text)))


def _check(rc: int, what: str):
    if rc != OK:
        msg = load().vbyte_strerror(rc).decode()
        raise VByteError(f"{what} failed: {msg} (code {rc})")


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _np_ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else None


# ------------------------------------------------------------------ encoder --

def encode(values) -> np.ndarray:
    v = np.ascontiguousarray(values, dtype=np.uint32)
    out = np.empty(max(5 * v.size, 1), dtype=np.uint8)
    nb = load().vbyte_encode(_np_ptr(v), v.size, _np_ptr(out))
    return out[:nb]


def encode_delta(values, prev: int = 0) -> np.ndarray:
    v = np.ascontiguousarray(values, dtype=np.uint32)
    out = np.empty(max(5 * v.size, 1), dtype=np.uint8)
    nb = load().vbyte_encode_delta(_np_ptr(v), v.size, ctypes.c_uint32(prev & 0xFFFFFFFF), _np_ptr(out))
    return out[:nb]


def encode_batched(values, val_off, delta: bool, prev=None):
    v = np.ascontiguousarray(values, dtype=np.uint32)
    vo = np.ascontiguousarray(val_off, dtype=np.uint64)
    L = vo.size - 1
    pv = None if prev is None else np.ascontiguousarray(prev, dtype=np.uint32)
    out = np.empty(max(5 * v.size, 1), dtype=np.uint8)
    bo = np.empty(L + 1, dtype=np.uint64)
    nb = load().vbyte_encode_batched(_np_ptr(v), _np_ptr(vo), L, int(delta),
                                     None if pv is None else _np_ptr(pv), _np_ptr(out), _np_ptr(bo))
    return out[:nb], bo


# ------------------------------------------------------------------ decoder --

def _device_args(data, n, out):
    import torch
    if not isinstance(data, torch.Tensor) or data.dtype != torch.uint8 or not data.is_cuda:
        raise TypeError("data must be a CUDA uint8 tensor")
    if not data.is_contiguous():
        raise ValueError("data must be contiguous")
    if out is None:
        out = torch.empty(n, dtype=torch.uint32, device=data.device)
    elif out.dtype not in (torch.uint32, torch.int32) or not out.is_contiguous() or out.numel() < n:
        raise ValueError("out must be a contiguous 32-bit CUDA tensor with at least n elements")
    return out


def encode_delta_m1(values, prev: int = 0) -> np.ndarray:
    """Host encoding of the gaps-minus-one variant: x_0 - prev, then
    x_i - x_{i-1} - 1 (mod 2^32)."""
    v = np.ascontiguousarray(values, dtype=np.uint32)
    out = np.empty(max(5 * v.size, 1), dtype=np.uint8)
    nb = load().vbyte_encode_delta_m1(_np_ptr(v), v.size, ctypes.c_uint32(prev & 0xFFFFFFFF), _np_ptr(out))
    return out[:nb]


def encode_device(values, delta: bool = False, prev: int = 0, out=None, nbytes=None, stream=None,
                  minus_one: bool = False):
    """Encode the CUDA uint32/int32 tensor `values` on the device (delta: its
    gaps from prev; minus_one: every gap after the first one less).  Returns
    (out, nbytes): `out` is a uint8 tensor of 5 * n bytes whose first nbytes
    hold the encoding, `nbytes` a one-element int64 CUDA tensor written when
    the stream gets there (no synchronisation)."""
    import torch
    if not isinstance(values, torch.Tensor) or not values.is_cuda or not values.is_contiguous() \
            or values.dtype not in (torch.int32, torch.uint32):
        raise TypeError("values must be a contiguous CUDA int32/uint32 tensor")
    n = values.numel()
    if out is None:
        out = torch.empty(max(5 * n, 1), dtype=torch.uint8, device=values.device)
    elif out.dtype != torch.uint8 or not out.is_cuda or out.numel() < 5 * n or not out.is_contiguous():
        raise TypeError("out must be a contiguous CUDA uint8 tensor of at least 5 * n bytes")
    if nbytes is None:
        nbytes = torch.empty(1, dtype=torch.int64, device=values.device)
    lib, st = load(), _stream_handle(stream)
    if minus_one:
        rc = lib.vbyte_encode_delta_m1_device(ctypes.c_void_p(values.data_ptr()), n,
                                              ctypes.c_uint32(prev & 0xFFFFFFFF), ctypes.c_void_p(out.data_ptr()),
                                              ctypes.c_void_p(nbytes.data_ptr()), st)
        _check(rc, "vbyte_encode_delta_m1_device")
        return out, nbytes
    if delta:
        rc = lib.vbyte_encode_delta_device(ctypes.c_void_p(values.data_ptr()), n, ctypes.c_uint32(prev & 0xFFFFFFFF),
                                           ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(nbytes.data_ptr()), st)
    else:
        rc = lib.vbyte_encode_device(ctypes.c_void_p(values.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(nbytes.data_ptr()), st)
    _check(rc, "vbyte_encode_delta_device" if delta else "vbyte_encode_device")
    return out, nbytes


def decode(data, n: int, out=None, stream=None):
    """Decode the VByte stream in the CUDA uint8 tensor `data` into n uint32."""
    out = _device_args(data, n, out)
    rc = load().vbyte_decode(ctypes.c_void_p(data.data_ptr()), data.numel(),
                             ctypes.c_void_p(out.data_ptr()), n, _stream_handle(stream))
    _check(rc, "vbyte_decode")
    return out


def decode_delta(data, n: int, prev: int = 0, out=None, stream=None):
    """Decode gaps and return their prefix sums from prev (uint32 wrap-around)."""
    out = _device_args(data, n, out)
    rc = load().vbyte_decode_delta(ctypes.c_void_p(data.data_ptr()), data.numel(),
                                   ctypes.c_void_p(out.data_ptr()), n,
                                   ctypes.c_uint32(prev & 0xFFFFFFFF), _stream_handle(stream))
    _check(rc, "vbyte_decode_delta")
    return out


def decode_delta_m1(data, n: int, prev: int = 0, out=None, stream=None):
    """Decode the gaps-minus-one variant: prefix sums from prev plus each
    value's rank (uint32 wrap-around)."""
    out = _device_args(data, n, out)
    rc = load().vbyte_decode_delta_m1(ctypes.c_void_p(data.data_ptr()), data.numel(),
                                      ctypes.c_void_p(out.data_ptr()), n,
                                      ctypes.c_uint32(prev & 0xFFFFFFFF), _stream_handle(stream))
    _check(rc, "vbyte_decode_delta_m1")
    return out


def _prev4(prev4):
    if prev4 is None:
        return None
    p = np.ascontiguousarray(prev4, dtype=np.uint32)
    if p.size != 4:
        raise ValueError("prev4 holds the four values before the list")
    return p


def encode_delta4(values, prev4=None) -> np.ndarray:
    """Host encoding of the blocked differences x_i - x_{i-4} (mod 2^32),
    x_{-4..-1} = prev4 (zeros: the paper's list)."""
    v = np.ascontiguousarray(values, dtype=np.uint32)
    p = _prev4(prev4)
    out = np.empty(max(5 * v.size, 1), dtype=np.uint8)
    nb = load().vbyte_encode_delta4(_np_ptr(v), v.size, None if p is None else _np_ptr(p), _np_ptr(out))
    return out[:nb]


def decode_delta4(data, n: int, prev4=None, out=None, stream=None):
    """Decode blocked differences: out[i] = g_i + out[i-4] (mod 2^32) with
    out[-4..-1] = prev4 (four values; None for zeros)."""
    out = _device_args(data, n, out)
    p = _prev4(prev4)
    rc = load().vbyte_decode_delta4(ctypes.c_void_p(data.data_ptr()), data.numel(), ctypes.c_void_p(out.data_ptr()),
                                    n, None if p is None else _np_ptr(p), _stream_handle(stream))
    _check(rc, "vbyte_decode_delta4")
    return out


def _offsets(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype not in (torch.int64, torch.uint64) \
            or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA int64/uint64 tensor")
    return ctypes.c_void_p(t.data_ptr())


def _batched_args(data, byte_off, val_off, n, out):
    import torch
    if not isinstance(data, torch.Tensor) or data.dtype != torch.uint8 or not data.is_cuda \
            or not data.is_contiguous():
        raise TypeError("data must be a contiguous CUDA uint8 tensor")
    if byte_off.numel() != val_off.numel() or byte_off.numel() < 1:
        raise ValueError("byte_off and val_off must both hold num_lists + 1 entries")
    if out is None:
        out = torch.empty(n, dtype=torch.uint32, device=data.device)
    elif out.dtype not in (torch.uint32, torch.int32) or not out.is_contiguous() or out.numel() < n:
        raise ValueError("out must be a contiguous 32-bit CUDA tensor with at least n elements")
    return out, _offsets(byte_off, "byte_off"), _offsets(val_off, "val_off")


def decode_batched(data, byte_off, val_off, n: int, out=None, stream=None):
    """Decode the lists laid end to end in `data` (list j: bytes
    byte_off[j]..byte_off[j+1], values val_off[j]..val_off[j+1]); n = val_off[-1]."""
    out, bo, vo = _batched_args(data, byte_off, val_off, n, out)
    rc = load().vbyte_decode_batched(ctypes.c_void_p(data.data_ptr()), data.numel(), bo,
                                     ctypes.c_void_p(out.data_ptr()), n, vo, byte_off.numel() - 1,
                                     _stream_handle(stream))
    _check(rc, "vbyte_decode_batched")
    return out


def decode_delta_batched(data, byte_off, val_off, n: int, prev=None, out=None, stream=None):
    """As decode_batched, each list differentially coded from prev[j] (0 if prev is None)."""
    import torch
    out, bo, vo = _batched_args(data, byte_off, val_off, n, out)
    pp = None
    if prev is not None:
        if not prev.is_cuda or prev.dtype not in (torch.int32, torch.uint32) or not prev.is_contiguous() \
                or prev.numel() != byte_off.numel() - 1:
            raise TypeError("prev must be a contiguous 32-bit CUDA tensor with num_lists entries")
        pp = ctypes.c_void_p(prev.data_ptr())
    rc = load().vbyte_decode_delta_batched(ctypes.c_void_p(data.data_ptr()), data.numel(), bo,
                                           ctypes.c_void_p(out.data_ptr()), n, vo, byte_off.numel() - 1,
                                           pp, _stream_handle(stream))
    _check(rc, "vbyte_decode_delta_batched")
    return out


class Plan:
    """A batched decode tuned once and replayed from a CUDA graph
    (vbyte_plan_*).  Keeps references to every tensor it points at."""

    def __init__(self, data, byte_off, val_off, n: int, delta: bool, prev=None, out=None,
                 autotune: bool = True, stream=None):
        import torch
        out, bo, vo = _batched_args(data, byte_off, val_off, n, out)
        pp = None
        if delta and prev is not None:
            if not prev.is_cuda or prev.dtype not in (torch.int32, torch.uint32) or \
                    prev.numel() != byte_off.numel() - 1:
                raise TypeError("prev must be a 32-bit CUDA tensor with num_lists entries")
            pp = ctypes.c_void_p(prev.data_ptr())
        self._keep = (data, byte_off, val_off, prev, out)
        self.out = out
        h = ctypes.c_void_p()
        rc = load().vbyte_plan_create(ctypes.byref(h), ctypes.c_void_p(data.data_ptr()), data.numel(), bo,
                                      ctypes.c_void_p(out.data_ptr()), n, vo, byte_off.numel() - 1, pp,
                                      int(delta), int(autotune), _stream_handle(stream))
        _check(rc, "vbyte_plan_create")
        self._h = h

    def launch(self, stream=None):
        _check(load().vbyte_plan_launch(self._h, _stream_handle(stream)), "vbyte_plan_launch")
        return self.out

    def get_status(self, stream=None) -> int:
        v = ctypes.c_uint32(0)
        _check(load().vbyte_plan_get_status(self._h, _stream_handle(stream), ctypes.byref(v)),
               "vbyte_plan_get_status")
        return int(v.value)

    def describe(self) -> dict:
        c, sl, ms, tu = ctypes.c_int(0), ctypes.c_uint64(0), ctypes.c_float(0), ctypes.c_int(0)
        _check(load().vbyte_plan_describe(self._h, ctypes.byref(c), ctypes.byref(sl), ctypes.byref(ms),
                                          ctypes.byref(tu)), "vbyte_plan_describe")
        k, cb, tpb = ctypes.c_int(0), ctypes.c_uint64(0), ctypes.c_int(0)
        _check(load().vbyte_plan_choice(self._h, ctypes.byref(k), ctypes.byref(cb), ctypes.byref(tpb)),
               "vbyte_plan_choice")
        classes = []
        modes = {1: "single pass", 2: "count then decode", 3: "segmented stream"}
        for kk in range(64):
            nl, nv, md = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_int(0)
            _check(load().vbyte_plan_class(self._h, kk, ctypes.byref(nl), ctypes.byref(nv), ctypes.byref(md)),
                   "vbyte_plan_class")
            if nl.value:
                classes.append({"bytes_class": kk, "lists": int(nl.value), "values": int(nv.value),
                                "mode": modes[md.value]})
        out = {"kernel": {0: "segmented stream", 1: "list items", 2: "list items, table-driven"}[k.value],
               "tuned_ms": round(ms.value, 5),
               "tuned": {0: "defaults", 1: "timed", 2: "cached for the length class"}[tu.value],
               "classes": classes}
        if k.value in (1, 2):
            out.update(chunk_bytes=int(cb.value), threads_per_block=tpb.value)
        else:
            out.update(ctas_per_sm=c.value, lead_slack_tiles=int(sl.value))
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().vbyte_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _ServerConfig(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_size_t), ("staging_bytes", ctypes.c_size_t),
                ("max_inflight", ctypes.c_int), ("max_batch_queries", ctypes.c_int),
                ("max_batch_lists", ctypes.c_int), ("per_list", ctypes.c_int)]


class _DeviceView:
    """A borrowed device buffer exposed through __cuda_array_interface__."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i4", "data": (ptr, False),
                                         "version": 2}


class Server:
    """vbyte_server_*: a resident pool of compressed lists and a continuous-
    batching request loop (the scheduler runs in a native thread).  form:
    "in_place" (batches decoded from the pool as list items), "per_list"
    (one single-stream call per list) or "gather" (lists gathered, then one
    segmented batched launch); per_list=True is form="per_list"."""

    FORMS = {"in_place": 0, "per_list": 1, "gather": 2}

    def __init__(self, pool, h_byte_off, h_val_off, delta: bool, h_prev=None, arena_bytes: int = 1 << 30,
                 staging_bytes: int = 256 << 20, max_inflight: int = 4, max_batch_queries: int = 64,
                 max_batch_lists: int = 512, per_list: bool = False, form: str | None = None):
        import torch
        if not isinstance(pool, torch.Tensor) or pool.dtype != torch.uint8 or not pool.is_cuda:
            raise TypeError("pool must be a CUDA uint8 tensor")
        self._bo = np.ascontiguousarray(h_byte_off, dtype=np.uint64)
        self._vo = np.ascontiguousarray(h_val_off, dtype=np.uint64)
        self._pv = None if h_prev is None else np.ascontiguousarray(h_prev, dtype=np.uint32)
        self._pool = pool
        mode = self.FORMS[form] if form is not None else int(bool(per_list))
        cfg = _ServerConfig(arena_bytes, staging_bytes, max_inflight, max_batch_queries, max_batch_lists, mode)
        h = ctypes.c_void_p()
        rc = load().vbyte_server_create(ctypes.byref(h), ctypes.c_void_p(pool.data_ptr()), pool.numel(),
                                        _np_ptr(self._bo), _np_ptr(self._vo), self._bo.size - 1, int(delta),
                                        None if self._pv is None else _np_ptr(self._pv), ctypes.byref(cfg))
        _check(rc, "vbyte_server_create")
        self._h = h

    def submit(self, lists) -> int:
        a = np.ascontiguousarray(lists, dtype=np.uint32)
        q = ctypes.c_uint64(0)
        _check(load().vbyte_server_submit(self._h, _np_ptr(a), a.size, ctypes.byref(q)), "vbyte_server_submit")
        return int(q.value)

    def wait(self, qid: int):
        lat, st = ctypes.c_double(0), ctypes.c_uint32(0)
        _check(load().vbyte_server_wait(self._h, qid, ctypes.byref(lat), ctypes.byref(st)), "vbyte_server_wait")
        return float(lat.value), int(st.value)

    def result(self, qid: int):
        """(values as a borrowed CUDA int32 tensor, queries in its batch); valid until release."""
        import torch
        p, n, bq = ctypes.c_void_p(), ctypes.c_size_t(0), ctypes.c_uint32(0)
        _check(load().vbyte_server_result(self._h, qid, ctypes.byref(p), ctypes.byref(n), ctypes.byref(bq)),
               "vbyte_server_result")
        if n.value == 0:
            return torch.zeros(0, dtype=torch.int32, device=self._pool.device), int(bq.value)
        return torch.as_tensor(_DeviceView(p.value, n.value), device=self._pool.device), int(bq.value)

    def release(self, qid: int):
        _check(load().vbyte_server_release(self._h, qid), "vbyte_server_release")

    def replay(self, arrival_s, query_off, query_lists):
        arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
        qo = np.ascontiguousarray(query_off, dtype=np.uint64)
        ql = np.ascontiguousarray(query_lists, dtype=np.uint32)
        lat = np.zeros(arr.size, dtype=np.float64)
        st = np.zeros(arr.size, dtype=np.uint32)
        _check(load().vbyte_server_replay(self._h, _np_ptr(qo), _np_ptr(ql), arr.size, _np_ptr(arr),
                                          _np_ptr(lat), _np_ptr(st)), "vbyte_server_replay")
        return lat, st

    def stats(self) -> dict:
        b, q, v, l_ = (ctypes.c_uint64(0) for _ in range(4))
        _check(load().vbyte_server_stats(self._h, ctypes.byref(b), ctypes.byref(q), ctypes.byref(v),
                                         ctypes.byref(l_)), "vbyte_server_stats")
        return {"batches": b.value, "queries": q.value, "values": v.value, "lists": l_.value}

    def close(self):
        if getattr(self, "_h", None):
            load().vbyte_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def decode_each(data, h_byte_off: np.ndarray, h_val_off: np.ndarray, n: int, delta: bool, h_prev=None,
                out=None, stream=None):
    """One single-stream call per list (host offsets): the form batching replaces."""
    import torch
    bo = np.ascontiguousarray(h_byte_off, dtype=np.uint64)
    vo = np.ascontiguousarray(h_val_off, dtype=np.uint64)
    pv = None if h_prev is None else np.ascontiguousarray(h_prev, dtype=np.uint32)
    if out is None:
        out = torch.empty(n, dtype=torch.uint32, device=data.device)
    rc = load().vbyte_decode_each(ctypes.c_void_p(data.data_ptr()), _np_ptr(bo), ctypes.c_void_p(out.data_ptr()),
                                  _np_ptr(vo), bo.size - 1, int(delta), None if pv is None else _np_ptr(pv),
                                  _stream_handle(stream))
    _check(rc, "vbyte_decode_each")
    return out


def decode_host(data: np.ndarray, n: int, delta: bool = False, prev: int = 0, out=None, stream=None):
    """Host bytes in, host uint32 out (copies in both directions inside the call)."""
    b = np.ascontiguousarray(data, dtype=np.uint8)
    if out is None:
        out = np.empty(n, dtype=np.uint32)
    rc = load().vbyte_decode_host(_np_ptr(b), b.size, _np_ptr(out), n, int(delta),
                                  ctypes.c_uint32(prev & 0xFFFFFFFF), _stream_handle(stream))
    _check(rc, "vbyte_decode_host")
    return out


def decode_noalloc(data, n: int, delta: bool = False, prev: int = 0, out=None, status=None,
                   stream=None):
    """vbyte_decode_noalloc: decode with the library's fixed scratch array.

    `status` is an optional CUDA int32/uint32 tensor of one element into which
    the data-error bits are OR-ed."""
    import torch
    out = _device_args(data, n, out)
    sp = None
    if status is not None:
        if not status.is_cuda or status.dtype not in (torch.int32, torch.uint32):
            raise TypeError("status must be a 32-bit CUDA tensor")
        sp = ctypes.c_void_p(status.data_ptr())
    rc = load().vbyte_decode_noalloc(ctypes.c_void_p(data.data_ptr()), data.numel(),
                                     ctypes.c_void_p(out.data_ptr()), n, int(delta),
                                     ctypes.c_uint32(prev & 0xFFFFFFFF), sp, _stream_handle(stream))
    _check(rc, "vbyte_decode_noalloc")
    return out


# ------------------------------------------------------- 64-bit integers --

MASK64 = (1 << 64) - 1


def encode64(values) -> np.ndarray:
    """Host encoding of uint64 values (up to ten bytes each)."""
    v = np.ascontiguousarray(values, dtype=np.uint64)
    out = np.empty(max(10 * v.size, 1), dtype=np.uint8)
    nb = load().vbyte_encode64(_np_ptr(v), v.size, _np_ptr(out))
    return out[:nb]


def encode_delta64(values, prev: int = 0) -> np.ndarray:
    """Host encoding of the uint64 gaps x_i - x_{i-1} (mod 2^64), x_0 = prev."""
    v = np.ascontiguousarray(values, dtype=np.uint64)
    out = np.empty(max(10 * v.size, 1), dtype=np.uint8)
    nb = load().vbyte_encode_delta64(_np_ptr(v), v.size, ctypes.c_uint64(prev & MASK64), _np_ptr(out))
    return out[:nb]


def _device_args64(data, n, out):
    import torch
    if not isinstance(data, torch.Tensor) or data.dtype != torch.uint8 or not data.is_cuda \
            or not data.is_contiguous():
        raise TypeError("data must be a contiguous CUDA uint8 tensor")
    if out is None:
        out = torch.empty(n, dtype=torch.int64, device=data.device)
    elif out.dtype not in (torch.int64, torch.uint64) or not out.is_contiguous() or out.numel() < n:
        raise ValueError("out must be a contiguous 64-bit CUDA tensor with at least n elements")
    return out


def decode64(data, n: int, out=None, stream=None):
    """Decode uint64 VByte integers into n 64-bit slots (int64 tensor by
    default; view its bits as uint64)."""
    out = _device_args64(data, n, out)
    rc = load().vbyte_decode64(ctypes.c_void_p(data.data_ptr()), data.numel(),
                               ctypes.c_void_p(out.data_ptr()), n, _stream_handle(stream))
    _check(rc, "vbyte_decode64")
    return out


def decode_delta64(data, n: int, prev: int = 0, out=None, stream=None):
    """Decode uint64 gaps and return their prefix sums from prev (mod 2^64)."""
    out = _device_args64(data, n, out)
    rc = load().vbyte_decode_delta64(ctypes.c_void_p(data.data_ptr()), data.numel(),
                                     ctypes.c_void_p(out.data_ptr()), n,
                                     ctypes.c_uint64(prev & MASK64), _stream_handle(stream))
    _check(rc, "vbyte_decode_delta64")
    return out


def debug_inject(skip_tile: int = -1, wait_limit_ns: int = 0):
    """vbyte_debug_inject: make later decode launches leave tile skip_tile's
    count unpublished and bound their waits by wait_limit_ns (tests of the
    timeout path; skip_tile < 0 and 0 restore the defaults)."""
    _check(load().vbyte_debug_inject(int(skip_tile), int(wait_limit_ns)), "vbyte_debug_inject")


def debug_force_passes(passes: int = 0):
    """vbyte_debug_force_passes: 1 = single-pass kernel, 2 = count then
    decode in one launch, 3 = split count / scan / decode, 4 = split with the
    table-driven steps of Sec. 4, 0 = the library's choice."""
    _check(load().vbyte_debug_force_passes(int(passes)), "vbyte_debug_force_passes")


def debug_force_plan(kernel: int = -1, chunk_bytes: int = 0, threads_per_block: int = 256):
    """vbyte_debug_force_plan: make later plans use kernel 0 (segmented
    stream), 1 (list items of chunk_bytes) or 2 (list items, table-driven
    steps); -1 restores the usual choice."""
    _check(load().vbyte_debug_force_plan(int(kernel), int(chunk_bytes), int(threads_per_block)),
           "vbyte_debug_force_plan")


def table():
    """The table-driven step's table (Sec. 4): (entries uint16[4096], cases
    uint32[170]) as vbyte_table documents them."""
    e = np.zeros(4096, dtype=np.uint16)
    c = np.zeros(170, dtype=np.uint32)
    _check(load().vbyte_table(_np_ptr(e), _np_ptr(c)), "vbyte_table")
    return e, c


def table_decode(data, n=None) -> np.ndarray:
    """Host decoding by the table-driven steps (vbyte_table_decode)."""
    b = np.ascontiguousarray(data, dtype=np.uint8)
    cap = b.size if n is None else n
    out = np.empty(max(cap, 1), dtype=np.uint32)
    cnt = load().vbyte_table_decode(_np_ptr(b), b.size, _np_ptr(out), cap)
    if cnt > cap:
        out = np.empty(cnt, dtype=np.uint32)
        cnt = load().vbyte_table_decode(_np_ptr(b), b.size, _np_ptr(out), cnt)
    return out[:cnt].copy()


def chosen_passes(nbytes: int, n: int, delta: bool) -> int:
    """The single-stream kernel (1 or 2 passes) a call on this input would use."""
    return int(load().vbyte_debug_passes_for(nbytes, n, int(delta)))


def get_status(stream=None) -> int:
    """Synchronise the stream, return and clear its data-error bits."""
    v = ctypes.c_uint32(0)
    rc = load().vbyte_get_status(_stream_handle(stream), ctypes.byref(v))
    _check(rc, "vbyte_get_status")
    return int(v.value)


def workspace_size(nbytes: int) -> int:
    return int(load().vbyte_workspace_size(nbytes))


def set_workspace(buf, stream=None):
    """vbyte_set_workspace: make the CUDA uint8 tensor `buf` (256-byte aligned,
    at least workspace_size(0) bytes) the stream's workspace, or with
    buf=None hand the stream back to library allocations.  The caller keeps
    `buf` alive while the stream uses it."""
    import torch
    if buf is None:
        _check(load().vbyte_set_workspace(_stream_handle(stream), None, 0), "vbyte_set_workspace")
        return
    if not isinstance(buf, torch.Tensor) or buf.dtype != torch.uint8 or not buf.is_cuda or not buf.is_contiguous():
        raise TypeError("buf must be a contiguous CUDA uint8 tensor")
    _check(load().vbyte_set_workspace(_stream_handle(stream), ctypes.c_void_p(buf.data_ptr()), buf.numel()),
           "vbyte_set_workspace")


def release_stream(stream=None):
    """vbyte_release_stream: free what the library holds for the stream."""
    _check(load().vbyte_release_stream(_stream_handle(stream)), "vbyte_release_stream")
