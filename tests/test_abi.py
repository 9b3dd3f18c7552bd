"""CPU-side checks of the C-ABI library: it builds, loads, exports every symbol
the public header declares, and its host encoder agrees byte for byte with
the oracle's (no GPU needed: the encoder is host code)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1503_07387_gb300 import _build, inputs, vbyte


def test_library_builds_and_loads():
    lib = vbyte.load()
    assert isinstance(lib, ctypes.CDLL)


def test_every_declared_symbol_is_exported():
    names = vbyte.declared_symbols()
    assert "vbyte_decode" in names and "vbyte_decode_delta" in names
    lib = vbyte.load()
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in names if n not in exported]
    assert not missing, missing


def test_strerror_and_sizes():
    lib = vbyte.load()
    assert lib.vbyte_strerror(0) == b"ok"
    assert b"invalid" in lib.vbyte_strerror(1)
    assert lib.vbyte_max_encoded_size(10) == 50
    assert vbyte.workspace_size(0) >= 256
    assert vbyte.workspace_size(1 << 30) >= 16 * ((1 << 30) // 4096)


@pytest.mark.parametrize("gen", ["uniform_bits", "geometric_gaps", "uniform_gaps",
                                 "one_two_byte_mix", "full_range"])
def test_host_encoder_matches_oracle(gen):
    v = getattr(inputs, gen)(100_000, seed=3)
    assert np.array_equal(vbyte.encode(v), oracle.encode(v))


def test_host_encoder_boundaries():
    v = np.array([0, 1, 127, 128, 16383, 16384, 2**21 - 1, 2**21, 2**28 - 1, 2**28,
                  2**32 - 1], dtype=np.uint32)
    assert np.array_equal(vbyte.encode(v), oracle.encode(v))
    assert vbyte.encode(np.zeros(0, np.uint32)).size == 0


def test_host_delta_and_batched_encoders_match_oracle():
    ids, vo = inputs.length_class_lists(200, max_class=9, seed=1)
    x = ids[int(vo[3]):int(vo[4])]
    assert np.array_equal(vbyte.encode_delta(x, prev=17), oracle.encode_delta(x, prev=17))
    prev = np.arange(200, dtype=np.uint32)
    for delta in (False, True):
        b1, o1 = vbyte.encode_batched(ids, vo, delta, prev if delta else None)
        b2, o2 = oracle.encode_batched(ids, vo, delta, prev if delta else None)
        assert np.array_equal(b1, b2) and np.array_equal(o1, o2)


def test_host_m1_encoder_matches_oracle():
    rng = np.random.default_rng(4)
    x = np.sort(rng.choice(1 << 31, 50_000, replace=False)).astype(np.uint32)
    for prev in (0, 5, 2**32 - 1):
        assert np.array_equal(vbyte.encode_delta_m1(x, prev=prev), oracle.encode_delta_m1(x, prev=prev))
    assert vbyte.encode_delta_m1(np.zeros(0, np.uint32)).size == 0


def test_argument_errors_before_any_device_work():
    """Null or misaligned arguments are refused on the host (no CUDA call is
    reached), so these run without a GPU."""
    lib = vbyte.load()
    P = ctypes.c_void_p
    einval = 1
    # a null input with bytes, a null output with values
    assert lib.vbyte_decode(None, 16, P(16), 4, None) == einval
    assert lib.vbyte_decode(P(16), 16, None, 4, None) == einval
    assert lib.vbyte_decode_delta(None, 16, P(16), 4, 0, None) == einval
    assert lib.vbyte_decode_delta_m1(None, 16, P(16), 4, 0, None) == einval
    # an output that is not 4-byte aligned
    assert lib.vbyte_decode(P(16), 16, P(18), 4, None) == einval
    # the device encoder: misaligned input, null count word
    assert lib.vbyte_encode_device(P(18), 4, P(64), P(128), None) == einval
    assert lib.vbyte_encode_device(P(16), 4, P(64), None, None) == einval
    assert lib.vbyte_encode_delta_m1_device(None, 4, 0, P(64), P(128), None) == einval
    # plans and servers need their out-parameters
    assert lib.vbyte_plan_create(None, P(16), 16, P(16), P(16), 4, P(16), 1, None, 0, 0, None) == einval
    # 64-bit decoding: null pointers, an output that is not 8-byte aligned
    assert lib.vbyte_decode64(None, 16, P(16), 4, None) == einval
    assert lib.vbyte_decode64(P(16), 16, None, 4, None) == einval
    assert lib.vbyte_decode64(P(16), 16, P(20), 4, None) == einval
    assert lib.vbyte_decode_delta64(P(16), 16, P(12), 4, 0, None) == einval
    # nothing to do: no bytes and no values
    assert lib.vbyte_decode64(None, 0, None, 0, None) == 0
    # a caller workspace must be 256-byte aligned and hold at least the head
    assert lib.vbyte_set_workspace(None, P(256 + 16), 1 << 20) == einval
    assert lib.vbyte_set_workspace(None, P(1 << 20), vbyte.workspace_size(0) - 1) == einval


def _all_widths64(n, seed):
    """uint64 values of every bit width 0..64, equally often."""
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 65, n).astype(np.uint64)
    hi = rng.integers(0, 1 << 63, n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        v = np.where(bits == 0, np.uint64(0), hi >> (np.uint64(64) - np.maximum(bits, np.uint64(1))))
    return v.astype(np.uint64)


def test_host_encoder64_matches_oracle():
    v = _all_widths64(100_000, 2)
    assert np.array_equal(vbyte.encode64(v), oracle.encode64(v))
    edges = [0, 1, (1 << 64) - 1] + [(1 << (7 * k)) + d for k in range(1, 10) for d in (-1, 0)]
    e = np.array(edges, dtype=np.uint64)
    assert np.array_equal(vbyte.encode64(e), oracle.encode64(e))
    assert vbyte.encode64(np.zeros(0, np.uint64)).size == 0
    assert vbyte.load().vbyte_max_encoded_size64(7) == 70
    for prev in (0, 12345, (1 << 64) - 1):
        assert np.array_equal(vbyte.encode_delta64(v, prev=prev), oracle.encode_delta64(v, prev=prev))


C_CONSUMER = r"""
#include <stdio.h>
#include <stdint.h>
#include "vbyte.h"
#include "vbyte64.h"
#include "vbyte_debug.h"
int main(void)
{
    const uint32_t v[3] = {1u, 300u, 0xFFFFFFFFu};
    uint8_t out[15];
    const uint64_t w[2] = {1u, 0xFFFFFFFFFFFFFFFFull};
    uint8_t o64[20];
    size_t nb = vbyte_encode(v, 3, out);
    size_t nb64 = vbyte_encode64(w, 2, o64);
    for (size_t i = 0; i < nb; ++i) printf("%02x", out[i]);
    printf(" ");
    for (size_t i = 0; i < nb64; ++i) printf("%02x", o64[i]);
    printf(" %d", vbyte_decode(NULL, 16, NULL, 4, NULL));
    printf(" %d\n", vbyte_debug_inject(-1, 3000000000ull));
    return 0;
}
"""


def test_plain_c_consumer(tmp_path):
    """The public headers compile as C99 with warnings as errors, and a C
    program links against libvbyte.so and calls its host entry points."""
    vbyte.load()
    src = tmp_path / "consumer.c"
    src.write_text(C_CONSUMER)
    exe = tmp_path / "consumer"
    libdir = os.path.dirname(_build.LIB)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", f"-I{_build.INCLUDE}", str(src),
                    f"-L{libdir}", "-lvbyte", f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert out[0] == bytes(oracle.encode(np.array([1, 300, 0xFFFFFFFF], np.uint32))).hex()
    assert out[1] == bytes(oracle.encode64(np.array([1, (1 << 64) - 1], np.uint64))).hex()
    assert out[2] == "1"   # VBYTE_EINVAL, before any CUDA call
    assert out[3] == "1"   # a wait bound above the default is refused


def test_kernel_choice_by_length_class():
    """The single-stream kernel the library picks (host logic, no GPU): the
    single pass for inputs under 16 MiB, count-then-decode for one-byte codes,
    the split launches else (long codes too, plain and differential); a
    forced choice wins until it is cleared."""
    M = 1 << 20
    assert vbyte.chosen_passes(4 * M, 3 * M, False) == 1
    assert vbyte.chosen_passes(64 * M, 64 * M, True) == 2
    assert vbyte.chosen_passes(300 * M, 60 * M, True) == 3
    assert vbyte.chosen_passes(300 * M, 60 * M, False) == 3
    assert vbyte.chosen_passes(96 * M, 64 * M, True) == 3
    try:
        vbyte.debug_force_passes(2)
        assert vbyte.chosen_passes(4 * M, 3 * M, False) == 2
    finally:
        vbyte.debug_force_passes(0)
    with pytest.raises(vbyte.VByteError):
        vbyte.debug_force_passes(5)


def test_host_encoder_delta4_matches_oracle():
    rng = np.random.default_rng(3)
    x = rng.integers(0, 1 << 32, 10_001, dtype=np.uint64).astype(np.uint32)
    for prev4 in (None, [1, 2, 3, 4], [0xFFFFFFFF] * 4):
        assert np.array_equal(vbyte.encode_delta4(x, prev4=prev4), oracle.encode_delta4(x, prev4=prev4))
    assert vbyte.encode_delta4(np.zeros(0, np.uint32)).size == 0
