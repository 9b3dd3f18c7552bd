"""Benchmark: VByte decoding throughput on GB300 (Gints/s and % of HBM roofline).

One "step" is one pass of the whole hot path over one batch of synthetic
input.  The default (headline) workload is the roofline-stress configuration:
two single streams of 2^28 uint32 each, resident in HBM --
  * one- or two-byte codes by a fair coin (the branch-misprediction case of
    the paper's Sec. 2), about 0.375 GiB compressed;
  * uniform full-range uint32 (mostly five-byte codes), about 1.23 GiB --
each decoded plainly and differentially (the same bytes read as gaps and
prefix-summed back with uint32 wrap-around): four decode calls per step,
each the split decoder's count, scan and decode launches.  Inputs plus
outputs exceed the 129 MB L2, so no flush is needed between steps.

The same JSON line carries a block per other configuration, each with its own
roofline and single-core oracle baseline: 10^6 plain values of every code
length (about 6.7 MB, timed with L2 flushed before every step and warm beside
it), the two differential 2^26 streams (geometric and uniform [1, 300] gaps),
and every stream of the headline separately; then batched decoding of 100,000
rank-Zipf posting lists (a tuned plan replayed from a CUDA graph against one
call per list, with an all-cores oracle baseline), the serving loop at
Poisson query rates, the device encoder and the 64-bit decoder.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload roofline_stress_2^28 | ...]

Under torchrun (N > 1) every rank decodes its own replica of the workload
(the path shards into independent streams; no data-path collective); rank 0
prints one JSON line with the whole-job throughput.  ``--impl reference``
times the CPU oracle (Algorithm 1, one core) on the same workload instead.
``--profile-case NAME`` runs one small stream a few times (for ncu) and prints
nothing else.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1503_07387_gb300 import inputs  # noqa: E402

METRIC = "Gints/s decoded + % of HBM roofline"
UNIT = "Gints/s"
PROFILES = os.path.join(ROOT, "profiles")
L2_FLUSH_BYTES = 256 << 20   # about twice the GB300's 129 MB L2
NOMINAL_HBM_GBS = 8000.0


# ------------------------------------------------------------------ workloads --
#
# A workload is a list of streams (label, values-to-encode generator, delta).
# For differential streams the values are the gaps; streams with the same
# `src` share their bytes (plain and differential readings of one stream).

def _src(name: str):
    gens = {
        "uniform_bits_1e6": lambda: inputs.uniform_bits(1_000_000, seed=0),
        "geometric_gaps_2^26": lambda: inputs.geometric_gaps(1 << 26, seed=0),
        "uniform_gaps_1_300_2^26": lambda: inputs.uniform_gaps(1 << 26, seed=1),
        "one_two_byte_mix_2^28": lambda: inputs.one_two_byte_mix(1 << 28, seed=0),
        "full_range_2^28": lambda: inputs.full_range(1 << 28, seed=0),
    }
    return gens[name]()


WORKLOADS = {
    # config 5: the roofline stress streams, plain and differential (the headline)
    "roofline_stress_2^28": [("one_two_byte_mix_plain", "one_two_byte_mix_2^28", False),
                             ("one_two_byte_mix_delta", "one_two_byte_mix_2^28", True),
                             ("full_range_plain", "full_range_2^28", False),
                             ("full_range_delta", "full_range_2^28", True)],
    # config 1: plain decode of 10^6 values of every code length
    "plain_uniform_bits_1e6": [("uniform_bits", "uniform_bits_1e6", False)],
    # config 2: differential decode of two 2^26 document-id streams
    "differential_2x2^26": [("geometric_gaps", "geometric_gaps_2^26", True),
                            ("uniform_gaps_1_300", "uniform_gaps_1_300_2^26", True)],
    # single streams of config 5, for experiments and profiles
    "plain_one_two_2^28": [("one_two_byte_mix_plain", "one_two_byte_mix_2^28", False)],
    "delta_one_two_2^28": [("one_two_byte_mix_delta", "one_two_byte_mix_2^28", True)],
    "plain_full_range_2^28": [("full_range_plain", "full_range_2^28", False)],
    "delta_full_range_2^28": [("full_range_delta", "full_range_2^28", True)],
}
HEADLINE = "roofline_stress_2^28"
BLOCKS = ["plain_uniform_bits_1e6", "differential_2x2^26"]   # reported beside the headline

# Single streams for ncu captures, a few launches each: (generator, n,
# differential, seed, default 0), the seeds those of the workloads above.
# The 2^28 streams are the headline's own (at most 2.4 GB on the device);
# the 2^26 ones are smaller cases of the same kernels for --set full.
PROFILE_CASES = {
    "one_two_plain_2^28": ("one_two_byte_mix", 1 << 28, False),
    "one_two_delta_2^28": ("one_two_byte_mix", 1 << 28, True),
    "full_range_plain_2^28": ("full_range", 1 << 28, False),
    "full_range_delta_2^28": ("full_range", 1 << 28, True),
    "one_two_plain_2^26": ("one_two_byte_mix", 1 << 26, False),
    "one_two_delta_2^26": ("one_two_byte_mix", 1 << 26, True),
    "full_range_plain_2^26": ("full_range", 1 << 26, False),
    "full_range_delta_2^26": ("full_range", 1 << 26, True),
    "geometric_delta_2^26": ("geometric_gaps", 1 << 26, True),
    "uniform300_delta_2^26": ("uniform_gaps", 1 << 26, True, 1),
    "uniform_bits_plain_1e6": ("uniform_bits", 1_000_000, False),
}


def encode_workload(name: str, encoder):
    """[(label, n, delta, bytes)] with bytes shared between streams of one source."""
    cache = {}
    out = []
    for label, src, delta in WORKLOADS[name]:
        if src not in cache:
            v = _src(src)
            cache[src] = (int(v.size), encoder(v))
            del v
        n, b = cache[src]
        out.append((label, n, delta, b, src))
    return out


# --------------------------------------------------------------- environment --

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int, device: str) -> float:
    """The slowest rank's time: every rank's timed region ends at a barrier,
    and the job took as long as its slowest replica."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, ws: int, seconds: float) -> float:
    """Whole-job throughput in 10^9 units/s: every rank decodes its own replica
    (weak scaling), so the job processed ws times one rank's units."""
    return ws * units_per_rank / seconds / 1e9


# the translation units of the stream decode kernels, every header they
# include, and the dispatcher that picks a kernel per stream
KERNEL_SOURCES = ["paper_1503_07387_gb300/csrc/" + f for f in
                  ("vbyte_stream.cu", "vbyte_split.cu", "vbyte_device.cuh", "vbyte_emit.cuh",
                   "vbyte_table.cuh", "vbyte_internal.h", "vbyte_api.cu")] + ["include/vbyte.h"]


def _code_only(src: str) -> str:
    """The source with its comments removed and its whitespace collapsed, so
    that editing a comment does not invalidate a profile of unchanged code."""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        h.update(os.path.basename(rel).encode())
        h.update(_code_only(open(os.path.join(ROOT, rel)).read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(src_hash: str, label: str, profiles_dir: str = PROFILES):
    """DRAM bytes per launch of stream `label` at its full size, from a
    committed ncu summary taken on the kernel source that is built now (else
    None).  A summary names its source hash once and has lines
    ``dram bytes per launch (full workload) [label]: X``."""
    for path in sorted(glob.glob(os.path.join(profiles_dir, "*.md"))):
        text = open(path).read()
        m_hash = re.search(r"kernel source hash:\s*`?([0-9a-f]{16})", text)
        if not m_hash or m_hash.group(1) != src_hash:
            continue
        m = re.search(r"dram bytes per launch \(full workload\) \[" + re.escape(label) + r"\]:\s*([0-9.eE+]+)",
                      text)
        if m:
            return float(m.group(1))
    return None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return None


def hbm_peak():
    peaks = measured_peaks()
    if peaks and peaks.get("hbm_gbs"):
        return float(peaks["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6800.0, "of fallback (6.8 TB/s)"


class ClockSampler:
    """nvidia-smi clocks/throttle sampler running while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 100):
        self.gpu = gpu_index
        self.period = period_ms
        self.proc = None
        self.rows = []
        self.t_start = self.t_end = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", str(self.period)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), line.strip()))

    def mark(self, which):
        setattr(self, "t_" + which, time.time())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        rows = [r for t, r in self.rows if self.t_start <= t <= self.t_end + 0.15]
        window = "timed region"
        if not rows:
            rows = [r for _, r in self.rows]
            window = "whole run (timed region shorter than the sampling period)"
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [x.strip() for x in r.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                maxs.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxs),
                "reasons": sorted(reasons), "samples": len(sms), "window": window}


# --------------------------------------------------------------------- GPU arm --

def _gpu_streams(name: str):
    """Encode (the library's host encoder) and move a workload to the device."""
    import torch
    from paper_1503_07387_gb300 import vbyte
    dev = {}
    streams = []
    for label, n, delta, b, src in encode_workload(name, vbyte.encode):
        if src not in dev:
            dev[src] = torch.from_numpy(b).cuda()
        streams.append(dict(label=label, n=n, delta=delta, host=b, d_in=dev[src],
                            d_out=torch.empty(n, dtype=torch.uint32, device="cuda")))
    torch.cuda.synchronize()
    return streams


def _launch(vbyte, s, stream):
    if s["delta"]:
        vbyte.decode_delta(s["d_in"], s["n"], out=s["d_out"], stream=stream)
    else:
        vbyte.decode(s["d_in"], s["n"], out=s["d_out"], stream=stream)


def time_streams(streams, steps: int, warmup: int, stream, ws: int = 1, sampler=None):
    """W untimed steps, then K timed steps bracketed by a barrier and a device
    synchronisation on both sides, every launch with its own CUDA events on
    the launching stream.  A workload smaller than 256 MiB is timed with L2
    flushed before every step (a write larger than L2, outside the launches'
    events) and its time is the sum of the launches' event times; a warm-L2
    figure is taken beside it."""
    import torch
    import torch.distributed as dist
    from paper_1503_07387_gb300 import vbyte

    def step(events=None):
        for i, s in enumerate(streams):
            if events is not None:
                events[i][0].record(stream)
            _launch(vbyte, s, stream)
            if events is not None:
                events[i][1].record(stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if vbyte.get_status() != 0:
        raise SystemExit("data error during warm-up")
    algo = sum(int(s["host"].size) + 4 * s["n"] for s in streams)
    l2_resident = algo < L2_FLUSH_BYTES
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda") if l2_resident else None
    ev = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in streams]
          for _ in range(steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler is not None:
        sampler.mark("start")
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(steps):
        if flush is not None:
            flush.fill_(k & 0xFF)
        step(ev[k])
    t1.record(stream)
    torch.cuda.synchronize()
    if sampler is not None:
        sampler.mark("end")
    if ws > 1:
        dist.barrier()
    launch_ms = [[e[0].elapsed_time(e[1]) for e in row] for row in ev]
    elapsed = t0.elapsed_time(t1)
    warm = None
    if flush is not None:
        elapsed = sum(x for row in launch_ms for x in row)   # the flushes are not decoding
        del flush
        w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0.record(stream)
        for _ in range(steps):
            step()
        w1.record(stream)
        torch.cuda.synchronize()
        warm = w0.elapsed_time(w1)
    status = vbyte.get_status()
    return dict(elapsed_ms=elapsed, launch_ms=launch_ms, warm_ms=warm, status=status, l2_resident=l2_resident)


def roofline_of(streams, launch_ms, peak, peak_source, src_hash, kernel):
    """The decoder's roofline over a step: algorithmic bytes (input read once
    + 4 bytes per value written) per decode call over the call's CUDA-event
    duration (all its launches), averaged over the step's calls."""
    nl = len(launch_ms)
    per_stream_ms = [sum(row[i] for row in launch_ms) / nl for i in range(len(streams))]
    algo = [int(s["host"].size) + 4 * s["n"] for s in streams]
    bytes_per_launch = sum(algo) / len(streams)
    avg_ms = sum(per_stream_ms) / len(streams)
    achieved = bytes_per_launch / (avg_ms * 1e-3) / 1e9
    tr = [profiled_traffic(src_hash, s["label"]) for s in streams]
    traffic = sum(tr) / len(tr) if all(t is not None for t in tr) else None
    rows = []
    for s, ms, a, t in zip(streams, per_stream_ms, algo, tr):
        gbs = a / (ms * 1e-3) / 1e9
        rows.append({"label": s["label"], "n": s["n"], "nbytes": int(s["host"].size),
                     "mode": "differential" if s["delta"] else "plain", "avg_launch_ms": round(ms, 5),
                     "gints_per_s": round(s["n"] / (ms * 1e-3) / 1e9, 3), "achieved_gbs": round(gbs, 1),
                     "frac": round(gbs / peak, 4), "frac_of_nominal_8000_gbs": round(gbs / NOMINAL_HBM_GBS, 4),
                     "traffic": t})
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": peak_source,
            "frac_of_nominal_8000_gbs": round(achieved / NOMINAL_HBM_GBS, 4), "traffic": traffic,
            "kernel": kernel, "algorithmic_bytes_per_launch": bytes_per_launch,
            "avg_launch_ms": round(avg_ms, 5), "kernel_source_hash": src_hash, "streams": rows}


def launches_per_call(vbyte, s) -> int:
    """Kernels one decode call of stream s launches: the split decoder's count,
    scan and decode, else one (the workspace clears are memsets, not kernels)."""
    return 3 if vbyte.chosen_passes(int(s["host"].size), s["n"], s["delta"]) in (3, 4) else 1


def kernel_name(vbyte, streams):
    passes = {vbyte.chosen_passes(int(s["host"].size), s["n"], s["delta"]) for s in streams}
    names = {1: "onepass_kernel (single pass, decoupled look-back)", 2: "sdecode_kernel (count then decode)",
             3: "sp::count_kernel + sp::scan_kernel + sp::decode2_kernel (split)",
             4: "sp::count_kernel + sp::decode_kernel (split, table-driven step)"}
    return " + ".join(names[p] for p in sorted(passes))


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_1503_07387_gb300 import vbyte

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    vbyte.load()
    if args.passes:
        vbyte.debug_force_passes(args.passes)
    stream = torch.cuda.current_stream()
    peak, peak_source = hbm_peak()
    src_hash = kernel_source_hash()

    streams = _gpu_streams(args.workload)
    total_vals = sum(s["n"] for s in streams)
    launches = sum(launches_per_call(vbyte, s) for s in streams)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.5)
    t = time_streams(streams, args.steps, args.warmup, stream, ws, sampler)
    clocks = sampler.stop()
    elapsed_ms = max_over_ranks(t["elapsed_ms"], ws, "cuda")
    roof = roofline_of(streams, t["launch_ms"], peak, peak_source, src_hash, kernel_name(vbyte, streams))
    warm = None
    if t["warm_ms"] is not None:
        warm = {"value": round(whole_job_rate(total_vals * args.steps, 1, t["warm_ms"] * 1e-3), 3), "unit": UNIT,
                "ms_per_step": round(t["warm_ms"] / args.steps, 5),
                "note": "the same steps back to back with L2 warm (inputs and outputs resident)"}
    status = t["status"]

    # ---- end to end through the public host-buffer call (copies inside)
    e2e = run_e2e(args, streams, stream, ws)
    status |= e2e.pop("status")

    # ---- CPU baseline (rank 0, N = 1 only): the oracle as it stands
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(streams, budget_s=args.cpu_seconds)

    for s in streams:
        del s["d_in"], s["d_out"]
    del streams
    torch.cuda.empty_cache()

    # ---- the other single-stream configurations, each with its own roofline
    blocks = {}
    if ws == 1 and not args.no_blocks:
        for name in [b for b in BLOCKS if b != args.workload]:
            blocks[name] = run_block(args, name, stream, peak, peak_source, src_hash)

    encode = decode64 = batched = serving = delta4 = None
    if ws == 1:
        if not args.no_encode:
            encode = run_encode(args, stream, peak)
        if not args.no_delta4:
            delta4 = run_delta4(args, stream, peak)
        if not args.no_decode64:
            try:
                decode64 = run_decode64(args, stream, peak)
            except Exception as e:   # an auxiliary leg: report it, keep the headline line
                decode64 = {"error": f"{type(e).__name__}: {e}"}
        if not args.no_batched:
            batched, pool = run_batched(args, peak)
            if not args.no_serving:
                serving = run_serving(args, pool)
            del pool

    if rank != 0:
        dist.destroy_process_group()
        return
    value = whole_job_rate(total_vals * args.steps, ws, elapsed_ms * 1e-3)
    wl = WORKLOADS[args.workload]
    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": UNIT,
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(elapsed_ms / args.steps, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8->u32",
        "data": "synthetic (seeded generators shaped like the paper's posting lists)",
        "config": {
            "workload": args.workload,
            "streams": [{"label": lab, "source": src, "mode": "differential" if d else "plain"}
                        for lab, src, d in wl],
            "values_per_step": total_vals,
            "l2": ("L2 flushed before every step (a 256 MiB write outside the launches' events); "
                   "value from the launches' event times" if warm is not None else
                   "inputs and outputs larger than the 129 MB L2; no flush"),
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
            "kernel_choice": "forced" if args.passes else "library default",
        },
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": launches * args.steps,
        "warm": warm,
        "status": status,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "host_cores": os.cpu_count(),
        "configs": blocks,
        "batched": batched,
        "serving": serving,
        "encode": encode,
        "decode64": decode64,
        "delta4": delta4,
    }
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def run_e2e(args, streams, stream, ws):
    """The same metric through vbyte_decode_host: every step copies the inputs
    from page-locked host memory and the decoded values back, inside the call."""
    import torch
    from paper_1503_07387_gb300 import vbyte
    import torch.distributed as dist
    pinned = {}
    h_in, h_out = [], []
    for s in streams:
        key = id(s["host"])
        if key not in pinned:
            pinned[key] = torch.from_numpy(s["host"]).pin_memory()
        h_in.append(pinned[key].numpy())
        h_out.append(torch.empty(s["n"], dtype=torch.int32).pin_memory().numpy().view(np.uint32))
    e2e_steps = max(3, min(args.steps, args.e2e_steps))
    for i, s in enumerate(streams):
        vbyte.decode_host(h_in[i], s["n"], delta=s["delta"], out=h_out[i], stream=stream)
    if ws > 1:
        dist.barrier()
    te = time.perf_counter()
    marks = [te]
    for _ in range(e2e_steps):
        for i, s in enumerate(streams):
            vbyte.decode_host(h_in[i], s["n"], delta=s["delta"], out=h_out[i], stream=stream)
        marks.append(time.perf_counter())
    e2e_s = max_over_ranks(marks[-1] - te, ws, "cuda")
    status = vbyte.get_status()
    total = sum(s["n"] for s in streams)
    return {"value": round(whole_job_rate(total * e2e_steps, ws, e2e_s), 3), "unit": UNIT,
            "h2d_bytes_per_step": int(sum(s["host"].size for s in streams)),
            "d2h_bytes_per_step": int(4 * total), "steps": e2e_steps,
            "step_ms": [round(1e3 * (b - a), 2) for a, b in zip(marks, marks[1:])],
            "api": "vbyte_decode_host (pinned host buffers, copies inside the call)", "status": status}


def run_block(args, name, stream, peak, peak_source, src_hash):
    """One more configuration: its own timing, roofline and oracle baseline."""
    import torch
    from paper_1503_07387_gb300 import vbyte
    streams = _gpu_streams(name)
    steps = max(5, min(args.steps, 200))
    t = time_streams(streams, steps, 3, stream)
    total = sum(s["n"] for s in streams)
    res = {"value": round(whole_job_rate(total * steps, 1, t["elapsed_ms"] * 1e-3), 3), "unit": UNIT,
           "steps": steps, "ms_per_step": round(t["elapsed_ms"] / steps, 5), "status": t["status"],
           "l2": "flushed before every step; value from the launches' event times" if t["l2_resident"]
           else "inputs and outputs larger than L2; no flush",
           "roofline": roofline_of(streams, t["launch_ms"], peak, peak_source, src_hash, kernel_name(vbyte, streams))}
    if t["warm_ms"] is not None:
        res["warm"] = {"value": round(whole_job_rate(total * steps, 1, t["warm_ms"] * 1e-3), 3), "unit": UNIT}
    if not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(streams, budget_s=max(1.0, args.cpu_seconds / 4))
    for s in streams:
        del s["d_in"], s["d_out"]
    torch.cuda.empty_cache()
    return res


def run_encode(args, stream, peak):
    """Device encoding of the two differential 2^26 streams' document ids,
    checked byte for byte against the host encoder and timed with CUDA events:
    Gints/s and the HBM roofline (4n read + bytes written)."""
    import torch
    from paper_1503_07387_gb300 import vbyte
    cases = []
    for gen, seed in (("geometric_gaps", 0), ("uniform_gaps", 1)):
        g = getattr(inputs, gen)(1 << 26, seed=seed)
        x = np.cumsum(g.astype(np.uint64)).astype(np.uint32)
        want = vbyte.encode_delta(x, prev=0)
        cases.append(dict(n=x.size, want=torch.from_numpy(want).cuda(), nb=int(want.size),
                          x=torch.from_numpy(x.view(np.int32)).cuda(),
                          buf=torch.empty(5 * x.size, dtype=torch.uint8, device="cuda"),
                          d_nb=torch.empty(1, dtype=torch.int64, device="cuda")))

    def step():
        for c in cases:
            vbyte.encode_device(c["x"], delta=True, out=c["buf"], nbytes=c["d_nb"], stream=stream)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    exact = all(int(c["d_nb"].item()) == c["nb"] and torch.equal(c["buf"][:c["nb"]], c["want"]) for c in cases)
    reps = max(5, min(args.steps, 200))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    n = sum(c["n"] for c in cases)
    algo = sum(4 * c["n"] + c["nb"] for c in cases)
    achieved = algo / (ms * 1e-3) / 1e9
    del cases
    return {"value": round(n / (ms * 1e-3) / 1e9, 3), "unit": "Gints/s", "ms_per_step": round(ms, 5),
            "form": "vbyte_encode_delta_device, one launch per stream (2 x 2^26 document ids)",
            "bit_exact_with_host_encoder": bool(exact), "status": int(vbyte.get_status()),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "algorithmic_bytes_per_step": algo}}


def run_decode64(args, stream, peak):
    """64-bit VByte decoding (the format read for uint64): 2^26 sorted uint64
    document ids from 1 + Geometric(0.1) gaps above 2^40 (differential, almost
    all one-byte codes) and 2^26 values of every bit width 0..64 (plain, code
    lengths 1..10), checked bit for bit against the values the streams were
    built from and timed with CUDA events: Gints/s and the HBM roofline
    (input bytes + 8n per call)."""
    import torch
    from paper_1503_07387_gb300 import vbyte
    n = 1 << 26
    ids = np.cumsum(inputs.geometric_gaps(n, seed=0).astype(np.uint64)) + np.uint64(1 << 40)
    vals = inputs.uniform_bits64(n, seed=1)
    cases = [{"label": "geometric_ids_delta", "x": ids, "delta": True, "host": vbyte.encode_delta64(ids)},
             {"label": "uniform_bits64_plain", "x": vals, "delta": False, "host": vbyte.encode64(vals)}]
    for c in cases:
        c["d_in"] = torch.from_numpy(c["host"]).cuda()
        c["out"] = torch.empty(n, dtype=torch.int64, device="cuda")

    def call(c):
        if c["delta"]:
            vbyte.decode_delta64(c["d_in"], n, out=c["out"], stream=stream)
        else:
            vbyte.decode64(c["d_in"], n, out=c["out"], stream=stream)

    reps = max(5, min(args.steps, 200))
    res = []
    for c in cases:
        for _ in range(3):
            call(c)
        torch.cuda.synchronize()
        exact = torch.equal(c["out"], torch.from_numpy(c["x"].view(np.int64)).cuda())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            call(c)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        algo = int(c["host"].size) + 8 * n
        achieved = algo / (ms * 1e-3) / 1e9
        res.append({"label": c["label"], "n": n, "nbytes": int(c["host"].size), "ms": round(ms, 5),
                    "value": round(n / (ms * 1e-3) / 1e9, 3), "unit": "Gints/s", "bit_exact": bool(exact),
                    "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                                 "frac": round(achieved / peak, 4), "algorithmic_bytes_per_call": algo}})
    status = int(vbyte.get_status())
    for c in cases:
        del c["d_in"], c["out"]
    return {"form": "vbyte_decode_delta64 / vbyte_decode64", "status": status, "streams": res}


def run_delta4(args, stream, peak):
    """Blocked differences (x_i - x_{i-4}, Sec. 1): 2^26 values of four
    interleaved sorted id lists, so each stored integer is one list's gap;
    checked bit for bit against the ids and timed with CUDA events: Gints/s
    and the HBM roofline (input bytes + 4n per call)."""
    import torch
    from paper_1503_07387_gb300 import vbyte
    n = 1 << 26
    g = inputs.geometric_gaps(n, seed=3).astype(np.uint64) + 1
    x = np.zeros(n, dtype=np.uint64)
    for k in range(4):
        x[k::4] = np.cumsum(g[k::4])
    x = x.astype(np.uint32)
    b = vbyte.encode_delta4(x)
    d = torch.from_numpy(b).cuda()
    out = torch.empty(n, dtype=torch.uint32, device="cuda")
    for _ in range(3):
        vbyte.decode_delta4(d, n, out=out, stream=stream)
    torch.cuda.synchronize()
    exact = bool(torch.equal(out.view(torch.int32), torch.from_numpy(x.view(np.int32)).cuda()))
    reps = max(5, min(args.steps, 200))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        vbyte.decode_delta4(d, n, out=out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    algo = int(b.size) + 4 * n
    achieved = algo / (ms * 1e-3) / 1e9
    res = {"workload": "2^26 values of four interleaved sorted id lists (gaps 2 + Geometric(0.1))",
           "n": n, "nbytes": int(b.size), "ms": round(ms, 5), "value": round(n / (ms * 1e-3) / 1e9, 3),
           "unit": "Gints/s", "bit_exact": exact, "status": int(vbyte.get_status(stream)),
           "form": "vbyte_decode_delta4 (split count, scan and decode launches)",
           "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(achieved / peak, 4), "algorithmic_bytes_per_call": algo}}
    del d, out
    return res


def run_batched(args, peak):
    """Batched differential decoding of 100,000 rank-Zipf posting lists (about
    1.2e8 values): a tuned plan replayed from a CUDA graph against one
    vbyte_decode_delta call per list, both checked against the oracle's
    per-list decoding and timed with CUDA events on the same stream; the
    oracle itself timed on all host cores."""
    import torch
    import oracle
    from paper_1503_07387_gb300 import vbyte
    ids, vo = inputs.posting_lists()
    L = vo.size - 1
    prev = inputs.full_range(L, seed=17)
    hb, hbo = vbyte.encode_batched(ids, vo, True, prev)
    n = int(vo[-1])
    del ids
    want, _ = oracle.decode_batched(hb, hbo, vo, True, prev, threads=os.cpu_count() or 1)
    d = torch.from_numpy(hb).cuda()
    dbo = torch.from_numpy(hbo.view(np.int64)).cuda()
    dvo = torch.from_numpy(vo.view(np.int64)).cuda()
    dp = torch.from_numpy(prev.view(np.int32)).cuda()
    dwant = torch.from_numpy(want.view(np.int32)).cuda()
    out_b = torch.empty(n, dtype=torch.uint32, device="cuda")
    out_e = torch.empty(n, dtype=torch.uint32, device="cuda")
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = vbyte.Plan(d, dbo, dvo, n, True, prev=dp, out=out_b, stream=stream)
    tune_s = time.perf_counter() - t0
    steps = max(5, min(args.steps, 200))
    for _ in range(3):
        plan.launch(stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for e0, e1 in ev:
        e0.record(stream)
        plan.launch(stream)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = sorted(e0.elapsed_time(e1) for e0, e1 in ev)
    st_b = plan.get_status(stream)
    # the per-list form: 100,000 single-stream calls back to back
    vbyte.decode_each(d, hbo, vo, n, True, prev, out=out_e, stream=stream)
    torch.cuda.synchronize()
    reps = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        vbyte.decode_each(d, hbo, vo, n, True, prev, out=out_e, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    each_ms = e0.elapsed_time(e1) / reps
    st_e = vbyte.get_status(stream)
    exact_b = bool(torch.equal(out_b.view(torch.int32), dwant))
    exact_e = bool(torch.equal(out_e.view(torch.int32), dwant))
    # the lean per-list form: the same 100,000 calls captured once into a
    # CUDA graph (one memset and one kernel per list, no host work per call)
    graph = None
    if not args.no_graph_each:
        gs = torch.cuda.Stream()
        out_g = torch.empty(n, dtype=torch.uint32, device="cuda")
        torch.cuda.synchronize()
        vbyte.decode_each(d, hbo, vo, n, True, prev, out=out_g, stream=gs)   # grows the stream's workspace
        gs.synchronize()
        g = torch.cuda.CUDAGraph()
        t0 = time.perf_counter()
        with torch.cuda.graph(g, stream=gs):
            vbyte.decode_each(d, hbo, vo, n, True, prev, out=out_g, stream=gs)
        cap_s = time.perf_counter() - t0
        g.replay()
        torch.cuda.synchronize()
        ge0, ge1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ge0.record(stream)
        for _ in range(reps):
            g.replay()
        ge1.record(stream)
        torch.cuda.synchronize()
        g_ms = ge0.elapsed_time(ge1) / reps
        graph = {"value": round(n / (g_ms * 1e-3) / 1e9, 3), "unit": UNIT, "ms": round(g_ms, 3),
                 "capture_s": round(cap_s, 2), "bit_exact_vs_oracle": bool(torch.equal(out_g.view(torch.int32), dwant)),
                 "status": int(vbyte.get_status(gs)),
                 "form": "the 100,000 vbyte_decode_delta calls captured into one CUDA graph, replayed"}
        del g, out_g
    med = ms[len(ms) // 2]
    algo = hb.size + 4 * n + 16 * (L + 1)
    # the oracle on every host core, lists split between threads
    cores = os.cpu_count() or 1
    reps_c, tc = 0, time.perf_counter()
    while True:
        oracle.decode_batched(hb, hbo, vo, True, prev, threads=cores)
        reps_c += 1
        if time.perf_counter() - tc >= args.cpu_seconds / 4:
            break
    cpu_s = (time.perf_counter() - tc) / reps_c
    res = {
        "workload": "100,000 rank-Zipf posting lists, universe 5e7, differential, per-list prev",
        "lists": L, "values": n, "nbytes": int(hb.size),
        "batched": {"value": round(n / (med * 1e-3) / 1e9, 3), "unit": UNIT, "ms_median": round(med, 5),
                    "ms_best": round(ms[0], 5), "launches": steps, "form": "vbyte_plan (CUDA graph)",
                    "plan": plan.describe(), "plan_create_s": round(tune_s, 3),
                    "roofline": {"bound": "hbm", "achieved": round(algo / (med * 1e-3) / 1e9, 1),
                                 "peak": peak, "unit": "GB/s",
                                 "frac": round(algo / (med * 1e-3) / 1e9 / peak, 4),
                                 "algorithmic_bytes": algo}},
        "per_list": {"value": round(n / (each_ms * 1e-3) / 1e9, 3), "unit": UNIT, "ms": round(each_ms, 3),
                     "form": "vbyte_decode_each (one vbyte_decode_delta per list)"},
        "per_list_graph": graph,
        "speedup": round(each_ms / med, 2),
        "speedup_vs_graph": round(graph["ms"] / med, 2) if graph else None,
        "bit_exact_vs_oracle": {"batched": exact_b, "per_list": exact_e},
        "status": st_b | st_e,
        "cpu_baseline": {"value": round(n / cpu_s / 1e9, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"the whole batch, {reps_c} pass(es), lists split over {cores} threads"},
    }
    plan.close()
    del dwant
    pool = dict(d=d, bo=hbo, vo=vo, prev=prev, lens=np.diff(vo).astype(np.int64))
    return res, pool


def run_serving(args, pool):
    """Open-loop Poisson query streams against the resident 100,000-list pool:
    each query names 2..8 lists drawn proportionally to length; continuous
    batching (each batch decoded in place from the pool as list items)
    against the same loop decoding every list with its own call.  Per rate, at least
    args.serve_seconds of arrivals or args.serve_queries queries, whichever is
    fewer, after an untimed warm-up.  Latency runs from a query's scheduled
    arrival to the scheduler seeing its batch complete."""
    import torch
    from paper_1503_07387_gb300 import vbyte
    free, _ = torch.cuda.mem_get_info()
    arena = int(min(free * 0.25, 8 << 30)) // 4096 * 4096
    cfg = dict(arena_bytes=arena, staging_bytes=512 << 20, max_inflight=4, max_batch_queries=64,
               max_batch_lists=512)
    rows = []
    for rate in args.serve_rates:
        nq = int(max(200, min(rate * args.serve_seconds, args.serve_queries)))
        arr, qoff, ql = inputs.query_stream(pool["lens"], nq, float(rate), seed=40)
        vals = int(sum(int(pool["lens"][ql[qoff[i]:qoff[i + 1]]].sum()) for i in range(nq)))
        row = {"rate_qps": rate, "queries": nq, "seconds_of_arrivals": round(float(arr[-1]), 2), "values": vals}
        for form, per_list in (("batched", False), ("per_list", True)):
            srv = vbyte.Server(pool["d"], pool["bo"], pool["vo"], True, pool["prev"],
                               form="per_list" if per_list else "in_place", **cfg)
            w = min(nq, max(100, int(rate * 0.2)))   # untimed warm-up: 0.2 s at the same rate
            srv.replay(arr[:w], qoff[:w + 1], ql[:int(qoff[w])])
            s0 = srv.stats()
            t0 = time.perf_counter()
            lat, st = srv.replay(arr, qoff, ql)
            span = time.perf_counter() - t0
            s = srv.stats()
            s["batches"] -= s0["batches"]
            srv.close()
            lat_ms = np.sort(lat) * 1e3
            row[form] = {"p50_ms": round(float(np.percentile(lat_ms, 50)), 3),
                         "p99_ms": round(float(np.percentile(lat_ms, 99)), 3),
                         "qps": round(nq / span, 1), "gints_per_s": round(vals / span / 1e9, 3),
                         "batches": s["batches"], "status": int(np.bitwise_or.reduce(st)) if st.size else 0}
        rows.append(row)
    return {"pool": "the 100,000-list batch above, resident in HBM", "arena_bytes": arena,
            "config": {k: v for k, v in cfg.items() if k != "arena_bytes"},
            "latency": "scheduled arrival -> batch completion seen by the scheduler thread",
            "rates": rows}


def cpu_baseline(streams, budget_s=10.0):
    """The oracle (scalar Algorithm 1, one core) over bounded prefixes of the
    same streams: each stream gets an equal share of about budget_s seconds
    (the prefix's byte length is found before the clock starts)."""
    import oracle
    per = budget_s / len(streams)
    done, spent = 0, 0.0
    parts = []
    for s in streams:
        # calibrate on a small prefix, then time a prefix worth `per` seconds
        m0 = min(s["n"], 1 << 18)
        nb0 = _prefix_bytes(s["host"], m0)
        t0 = time.perf_counter()
        _oracle_prefix(oracle, s, m0, nb0)
        rate = m0 / max(time.perf_counter() - t0, 1e-6)
        m = max(1, min(s["n"], int(rate * per)))
        nb = _prefix_bytes(s["host"], m)
        t0 = time.perf_counter()
        _oracle_prefix(oracle, s, m, nb)
        dt = time.perf_counter() - t0
        done += m
        spent += dt
        parts.append(f"{s['label']}: first {m} of {s['n']} values")
    return {"value": round(done / spent / 1e9, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "; ".join(parts) + f" ({spent:.1f} s, single thread)"}


def _oracle_prefix(oracle, s, m, nb):
    if s["delta"]:
        oracle.decode_delta(s["host"][:nb], m)
    else:
        oracle.decode(s["host"][:nb], m)


# --------------------------------------------------------------- profile case --

# Other kernels' cases: the batched plan on the 100,000-list workload, the
# device encoder and the 64-bit decoder on their bench inputs.
OTHER_PROFILE_CASES = ["batched_plan_1e5_lists", "encode_delta_geometric_2^26", "decode64_geometric_ids_2^26",
                       "decode64_uniform_bits_2^26"]


def _profile_other(args):
    import torch
    from paper_1503_07387_gb300 import vbyte
    case = args.profile_case
    launches = args.warmup + args.steps
    if case == "batched_plan_1e5_lists":
        ids, vo = inputs.posting_lists()
        prev = inputs.full_range(vo.size - 1, seed=17)
        hb, hbo = vbyte.encode_batched(ids, vo, True, prev)
        n = int(vo[-1])
        d = torch.from_numpy(hb).cuda()
        dbo = torch.from_numpy(hbo.view(np.int64)).cuda()
        dvo = torch.from_numpy(vo.view(np.int64)).cuda()
        dp = torch.from_numpy(prev.view(np.int32)).cuda()
        out = torch.empty(n, dtype=torch.uint32, device="cuda")
        # the tuner's choice on this batch, forced so that no tuning launches
        # come before the captured ones: list items of 32 KiB, 128 threads
        vbyte.debug_force_plan(1, 32 << 10, 128)
        plan = vbyte.Plan(d, dbo, dvo, n, True, prev=dp, out=out)
        vbyte.debug_force_plan(-1)
        for _ in range(launches):
            plan.launch()
        torch.cuda.synchronize()
        st = plan.get_status()
        info = {"nbytes": int(hb.size), "n": n, "plan": plan.describe()}
    elif case == "encode_delta_geometric_2^26":
        x = np.cumsum(inputs.geometric_gaps(1 << 26, seed=0).astype(np.uint64)).astype(np.uint32)
        dx = torch.from_numpy(x.view(np.int32)).cuda()
        buf = torch.empty(5 * x.size, dtype=torch.uint8, device="cuda")
        nb = torch.empty(1, dtype=torch.int64, device="cuda")
        for _ in range(launches):
            vbyte.encode_device(dx, delta=True, out=buf, nbytes=nb)
        torch.cuda.synchronize()
        st = vbyte.get_status()
        info = {"n": int(x.size), "nbytes": int(nb.item())}
    else:
        n = 1 << 26
        if case == "decode64_geometric_ids_2^26":
            x = np.cumsum(inputs.geometric_gaps(n, seed=0).astype(np.uint64)) + np.uint64(1 << 40)
            host, delta = vbyte.encode_delta64(x), True
        else:
            x, delta = inputs.uniform_bits64(n, seed=1), False
            host = vbyte.encode64(x)
        d = torch.from_numpy(host).cuda()
        out = torch.empty(n, dtype=torch.int64, device="cuda")
        for _ in range(launches):
            (vbyte.decode_delta64 if delta else vbyte.decode64)(d, n, out=out)
        torch.cuda.synchronize()
        st = vbyte.get_status()
        info = {"n": n, "nbytes": int(host.size), "delta": delta}
    print(json.dumps({"profile_case": case, "launches": launches, "status": st, **info}))
    if st:
        raise SystemExit(1)


def run_profile_case(args):
    """One small stream decoded a few times (the command ncu captures)."""
    import torch
    from paper_1503_07387_gb300 import vbyte
    if args.profile_case in OTHER_PROFILE_CASES:
        _profile_other(args)
        return
    gen, n, delta, *seed = PROFILE_CASES[args.profile_case]
    v = getattr(inputs, gen)(n, seed=seed[0] if seed else 0)
    b = vbyte.encode(v)
    if args.passes:
        vbyte.debug_force_passes(args.passes)
    d = torch.from_numpy(b).cuda()
    out = torch.empty(n, dtype=torch.uint32, device="cuda")
    for _ in range(args.warmup + args.steps):
        (vbyte.decode_delta if delta else vbyte.decode)(d, n, out=out)
    torch.cuda.synchronize()
    st = vbyte.get_status()
    print(json.dumps({"profile_case": args.profile_case, "n": n, "nbytes": int(b.size), "delta": delta,
                      "launches": args.warmup + args.steps, "status": st,
                      "kernel_source_hash": kernel_source_hash()}))
    if st:
        raise SystemExit(1)


# --------------------------------------------------------------- reference arm --

def _prefix_bytes(data: np.ndarray, m: int) -> int:
    """Byte length of the first m integers of a well-formed stream (at most
    five bytes each, so only the first 5m bytes are scanned)."""
    if m <= 0:
        return 0
    ends = np.flatnonzero(data[:5 * m] < 128)
    return int(ends[m - 1]) + 1


def run_reference(args):
    """The CPU oracle (scalar Algorithm 1, one core) on the same workload,
    encoded by the oracle's own encoder.  Each step decodes a bounded prefix
    of every stream, sized so that the whole --steps/--warmup run stays
    within about args.ref_seconds."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    streams = [dict(label=lab, n=n, delta=d, host=b) for lab, n, d, b, _ in
               encode_workload(args.workload, oracle.encode)]
    # calibrate the oracle's speed on the first 2^20 values of each stream
    cal = [(s, min(s["n"], 1 << 20)) for s in streams]
    cal = [(s, m, _prefix_bytes(s["host"], m)) for s, m in cal]
    t0 = time.perf_counter()
    for s, m, nb in cal:
        _oracle_prefix(oracle, s, m, nb)
    rate = sum(m for _, m, _ in cal) / max(time.perf_counter() - t0, 1e-6)
    per_step = args.ref_seconds / (args.steps + args.warmup)
    frac = min(1.0, per_step * rate / sum(s["n"] for s in streams))
    for s in streams:
        s["m"] = max(1, int(s["n"] * frac))
        s["nb"] = _prefix_bytes(s["host"], s["m"])

    def step():
        for s in streams:
            (oracle.decode_delta if s["delta"] else oracle.decode)(s["host"][:s["nb"]], s["m"])

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    per = sum(s["m"] for s in streams)
    total = args.steps * per
    value = total / dt / 1e9
    sample = (f"each step decodes the first {frac:.4f} of every stream ({per} values), "
              f"single thread; bytes from the oracle's encoder")
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": round(value, 4),
        "unit": UNIT,
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3 / args.steps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8->u32",
        "data": "synthetic (seeded generators shaped like the paper's posting lists)",
        "config": {"workload": args.workload,
                   "streams": [{"label": s["label"], "n": s["n"], "nbytes": int(s["host"].size),
                                "mode": "differential" if s["delta"] else "plain"} for s in streams]},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=HEADLINE)
    ap.add_argument("--passes", type=int, choices=[0, 1, 2, 3, 4], default=0,
                    help="single-stream kernel: 1 single pass, 2 count then decode, 3 split, "
                         "4 split with the table-driven step, 0 the library default")
    ap.add_argument("--profile-case", choices=sorted(PROFILE_CASES) + OTHER_PROFILE_CASES, default=None)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=120.0)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-blocks", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-encode", action="store_true")
    ap.add_argument("--no-decode64", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-delta4", action="store_true")
    ap.add_argument("--no-graph-each", action="store_true")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[2000, 5000, 10000, 20000, 50000])
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-queries", type=int, default=100_000)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.profile_case:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
