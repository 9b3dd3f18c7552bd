"""Host-side pieces of bench.py, checked on the CPU: the kernel-source hash
that ties the committed ncu traffic figure to the code it was taken on, the
lookup of that figure, the clock-record parsing, and the prefix sizing of
the reference arm."""
import os
import sys

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_code_only_ignores_comments_and_spacing():
    a = "int f(int x) {  // add one\n    return x + 1; /* the\n successor */ }\n"
    b = "/* header */\nint f(int x)\n{\n    return x + 1;\n}\n"
    assert bench._code_only(a) == bench._code_only(b) == "int f(int x) { return x + 1; }"
    assert bench._code_only(a) != bench._code_only(a.replace("x + 1", "x + 2"))


def test_profiled_traffic_lookup(tmp_path):
    """A summary's traffic figure is reported only for the kernel source hash
    it names, per stream label."""
    p = tmp_path / "p.md"
    p.write_text("kernel source hash: `0123456789abcdef`\n"
                 "dram bytes per launch (full workload) [full_range_delta]: 1.5e6\n"
                 "dram bytes per launch (full workload) [one_two_byte_mix_plain]: 2.5e6\n")
    assert bench.profiled_traffic("0123456789abcdef", "full_range_delta", str(tmp_path)) == 1.5e6
    assert bench.profiled_traffic("0123456789abcdef", "one_two_byte_mix_plain", str(tmp_path)) == 2.5e6
    assert bench.profiled_traffic("0123456789abcdef", "geometric_gaps", str(tmp_path)) is None
    assert bench.profiled_traffic("f" * 16, "full_range_delta", str(tmp_path)) is None
    assert bench.profiled_traffic("0123456789abcdef", "x", str(tmp_path / "absent")) is None
    assert len(bench.kernel_source_hash()) == 16


def test_workloads_share_bytes_between_readings():
    """The headline's plain and differential streams read the same bytes."""
    wl = bench.WORKLOADS[bench.HEADLINE]
    assert len(wl) == 4 and {d for _, _, d in wl} == {False, True}
    assert len({src for _, src, _ in wl}) == 2
    assert set(bench.BLOCKS) <= set(bench.WORKLOADS)


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


class _FakeThread:
    def join(self, timeout=None):
        pass


def test_clock_sampler_parses_rows_inside_the_timed_region():
    s = bench.ClockSampler(0)
    s.proc, s.thread = _FakeProc(), _FakeThread()
    s.t_start, s.t_end = 100.0, 101.0
    row = "0, {sm}, 2070, 900.5, 0x{r}, Not Active, Not Active, Not Active, {cap}"
    s.rows = [(99.0, row.format(sm=300, r=0, cap="Not Active")),     # before: ignored
              (100.2, row.format(sm=2070, r=0, cap="Not Active")),
              (100.5, row.format(sm=2040, r=4, cap="Active")),
              (100.9, row.format(sm=2055, r=0, cap="Not Active")),
              (105.0, row.format(sm=500, r=0, cap="Not Active"))]    # after: ignored
    rec = s.stop()
    assert rec["sm_mhz"] == 2055 and rec["sm_max_mhz"] == 2070
    assert rec["reasons"] == ["sw_power_cap"] and rec["samples"] == 3
    assert rec["window"] == "timed region"


def test_clock_sampler_without_nvidia_smi():
    s = bench.ClockSampler(0)
    assert s.stop() is None


def test_prefix_bytes_is_the_end_of_the_mth_integer():
    v = np.array([1, 300, 70000, 5, 1 << 31], dtype=np.uint32)
    data = oracle.encode(v)
    ends = np.cumsum([len(oracle.encode_one(int(x))) for x in v])
    for m in range(1, v.size + 1):
        assert bench._prefix_bytes(data, m) == ends[m - 1]
    assert bench._prefix_bytes(data, 0) == 0


def test_whole_job_rate_is_weak_scaling():
    assert bench.whole_job_rate(10**9, 1, 1.0) == pytest.approx(1.0)
    assert bench.whole_job_rate(10**9, 4, 2.0) == pytest.approx(2.0)
