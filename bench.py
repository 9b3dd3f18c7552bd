"""Benchmark: VByte decoding throughput on GB300 (Gints/s and % of HBM roofline).

Default workload (one "step" = one pass of the whole hot path over one batch):
differential decoding of two single streams of 2^26 uint32 each --
  stream A: gaps 1 + Geometric(0.1) (first gap 0), almost all one-byte codes;
  stream B: gaps uniform in [1, 300], a dense mix of one- and two-byte codes --
VByte-encoded on the host, resident in HBM, decoded and prefix-summed back to
document ids (uint32 wrap-around).  Inputs plus outputs exceed the 129 MB L2,
so no flush is needed between steps.  A smaller workload (--workload
plain_uniform_bits_1e6, about 6.7 MB) is timed with L2 flushed before every
step, its value taken from the launches' own events, and a warm-L2 figure
beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload differential_2x2^26 | ...]

Under torchrun (N > 1) every rank decodes its own replica of the workload
(the path shards into independent streams; no data-path collective); rank 0
prints one JSON line with the whole-job throughput.  ``--impl reference`` times
the CPU oracle (Algorithm 1, one core) on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1503_07387_gb300 import inputs  # noqa: E402

METRIC = "Gints/s decoded + % of HBM roofline"
UNIT = "Gints/s"
PROFILE_FILE = os.path.join(ROOT, "profiles", "decode_delta_differential_2x2^26.md")
L2_FLUSH_BYTES = 256 << 20   # about twice the GB300's 129 MB L2


# ------------------------------------------------------------------ workloads --

def workload(name: str):
    """Returns a list of (label, values_to_encode, delta) streams."""
    if name == "differential_2x2^26":
        return [("geometric_gaps", inputs.geometric_gaps(1 << 26, seed=0), True),
                ("uniform_gaps_1_300", inputs.uniform_gaps(1 << 26, seed=1), True)]
    if name == "plain_uniform_bits_1e6":
        return [("uniform_bits", inputs.uniform_bits(1_000_000, seed=0), False)]
    if name == "plain_one_two_2^28":
        return [("one_two_byte_mix", inputs.one_two_byte_mix(1 << 28, seed=0), False)]
    if name == "delta_one_two_2^28":
        return [("one_two_byte_mix", inputs.one_two_byte_mix(1 << 28, seed=0), True)]
    if name == "plain_full_range_2^28":
        return [("full_range", inputs.full_range(1 << 28, seed=0), False)]
    if name == "delta_full_range_2^28":
        return [("full_range", inputs.full_range(1 << 28, seed=0), True)]
    raise SystemExit(f"unknown workload {name}")


WORKLOADS = ["differential_2x2^26", "plain_uniform_bits_1e6", "plain_one_two_2^28",
             "delta_one_two_2^28", "plain_full_range_2^28", "delta_full_range_2^28"]


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


# the translation unit of the decode kernels and every header it includes
KERNEL_SOURCES = ["paper_1503_07387_gb300/csrc/vbyte_stream.cu", "paper_1503_07387_gb300/csrc/vbyte_device.cuh",
                  "paper_1503_07387_gb300/csrc/vbyte_internal.h", "include/vbyte.h"]


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


def profiled_traffic(src_hash: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the kernel source that is built now (else None)."""
    try:
        text = open(PROFILE_FILE).read()
    except OSError:
        return None
    m_hash = re.search(r"kernel source hash:\s*`?([0-9a-f]{16})", text)
    m_traffic = re.search(r"dram bytes per launch \(full workload\):\s*([0-9.eE+]+)", text)
    if m_hash and m_traffic and m_hash.group(1) == src_hash:
        return float(m_traffic.group(1))
    return None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return None


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
                 "--format=csv,noheader,nounits", f"-lms", str(self.period)],
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

def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_1503_07387_gb300 import vbyte

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    vbyte.load()

    streams = []
    for label, vals, delta in workload(args.workload):
        # values are the integers to code; for differential streams they are the gaps
        data = vbyte.encode(vals)
        streams.append(dict(label=label, n=int(vals.size), delta=delta, host=data,
                            d_in=torch.from_numpy(data).cuda(),
                            d_out=torch.empty(vals.size, dtype=torch.uint32, device="cuda")))
        del vals
    torch.cuda.synchronize()
    total_vals = sum(s["n"] for s in streams)
    algo_bytes = sum(s["host"].size + 4 * s["n"] for s in streams)
    stream = torch.cuda.current_stream()

    def step(events=None):
        for i, s in enumerate(streams):
            if events is not None:
                events[i][0].record(stream)
            if s["delta"]:
                vbyte.decode_delta(s["d_in"], s["n"], out=s["d_out"], stream=stream)
            else:
                vbyte.decode(s["d_in"], s["n"], out=s["d_out"], stream=stream)
            if events is not None:
                events[i][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if vbyte.get_status() != 0:
        raise SystemExit("data error during warm-up")
    # A workload whose inputs and outputs fit in L2 is timed with L2 flushed
    # before every step (a write larger than L2, outside the launches' events).
    l2_resident = algo_bytes < L2_FLUSH_BYTES
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda") if l2_resident else None

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.5)
    per_launch = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
                   for _ in streams] for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.mark("start")
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        if flush is not None:
            flush.fill_(k & 0xFF)
        step(per_launch[k])
    t1.record(stream)
    torch.cuda.synchronize()
    sampler.mark("end")
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    elapsed_ms = t0.elapsed_time(t1)
    launch_ms = [[ev[0].elapsed_time(ev[1]) for ev in row] for row in per_launch]
    warm = None
    if flush is not None:
        elapsed_ms = sum(x for row in launch_ms for x in row)   # the flushes are not decoding
        w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0.record(stream)
        for _ in range(args.steps):
            step()
        w1.record(stream)
        torch.cuda.synchronize()
        warm_ms = w0.elapsed_time(w1)
        warm = {"value": round(whole_job_rate(total_vals * args.steps, 1, warm_ms * 1e-3), 3), "unit": UNIT,
                "ms_per_step": round(warm_ms / args.steps, 5),
                "note": "the same steps back to back with L2 warm (inputs and outputs resident)"}
        del flush
    status = vbyte.get_status()

    elapsed_ms = max_over_ranks(elapsed_ms, ws, "cuda")

    # ---- end to end through the public host-buffer call (copies inside)
    pinned_in = [torch.from_numpy(s["host"]).pin_memory() for s in streams]
    pinned_out = [torch.empty(s["n"], dtype=torch.int32).pin_memory() for s in streams]
    h_in = [p.numpy() for p in pinned_in]
    h_out = [p.numpy().view(np.uint32) for p in pinned_out]
    e2e_steps = max(3, min(args.steps, 20))
    for i, s in enumerate(streams):
        vbyte.decode_host(h_in[i], s["n"], delta=s["delta"], out=h_out[i], stream=stream)
    if ws > 1:
        dist.barrier()
    te = time.perf_counter()
    for _ in range(e2e_steps):
        for i, s in enumerate(streams):
            vbyte.decode_host(h_in[i], s["n"], delta=s["delta"], out=h_out[i], stream=stream)
    e2e_s = time.perf_counter() - te
    e2e_s = max_over_ranks(e2e_s, ws, "cuda")
    status |= vbyte.get_status()

    # ---- the device encoder on the same streams (the step before the path)
    encode = None
    if not args.no_encode:
        encode = run_encode(args, streams, stream, measured_peaks())

    # ---- 64-bit integers
    decode64 = None
    if not args.no_decode64:
        try:
            decode64 = run_decode64(args, stream, measured_peaks())
        except Exception as e:   # an auxiliary leg: report it, keep the headline line
            decode64 = {"error": f"{type(e).__name__}: {e}"}

    # ---- batched lists: one tuned, graph-replayed launch vs one call per list
    batched = serving = None
    if ws == 1 and not args.no_batched:
        batched, pool = run_batched(args, measured_peaks())
        if not args.no_serving:
            serving = run_serving(args, pool)
        del pool

    # ---- CPU baseline (rank 0, N = 1 only): the oracle as it stands
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(streams, budget_s=args.cpu_seconds)

    if rank != 0:
        dist.destroy_process_group()
        return
    peaks = measured_peaks()
    peak_gbs = peaks["hbm_gbs"] if peaks else 6800.0
    launches = [x for row in launch_ms for x in row]
    avg_launch_ms = sum(launches) / len(launches)
    bytes_per_launch = algo_bytes / len(streams)
    achieved = bytes_per_launch / (avg_launch_ms * 1e-3) / 1e9
    src_hash = kernel_source_hash()
    traffic = profiled_traffic(src_hash)
    value = whole_job_rate(total_vals * args.steps, ws, elapsed_ms * 1e-3)
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
            "streams": [{"label": s["label"], "n": s["n"], "nbytes": int(s["host"].size),
                         "mode": "differential" if s["delta"] else "plain"} for s in streams],
            "values_per_step": total_vals,
            "l2": ("L2 flushed before every step (a 256 MiB write outside the launches' events); "
                   "value from the launches' event times" if warm is not None else
                   "inputs and outputs larger than the 129 MB L2; no flush"),
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
        },
        "roofline": {
            "bound": "hbm",
            "achieved": round(achieved, 1),
            "peak": peak_gbs,
            "unit": "GB/s",
            "frac": round(achieved / peak_gbs, 4),
            "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "of fallback",
            "frac_of_nominal_8000_gbs": round(achieved / 8000.0, 4),
            "traffic": traffic,
            "kernel": "sdecode_kernel<delta>" if all(s["delta"] for s in streams) else "sdecode_kernel",
            "algorithmic_bytes_per_launch": bytes_per_launch,
            "avg_launch_ms": round(avg_launch_ms, 5),
            "kernel_source_hash": src_hash,
        },
        "e2e": {
            "value": round(whole_job_rate(total_vals * e2e_steps, ws, e2e_s), 3),
            "unit": UNIT,
            "h2d_bytes_per_step": int(sum(s["host"].size for s in streams)),
            "d2h_bytes_per_step": int(4 * total_vals),
            "api": "vbyte_decode_host (pinned host buffers, copies inside the call)",
        },
        "gpu_launches": len(streams) * args.steps,
        "warm": warm,
        "encode": encode,
        "decode64": decode64,
        "batched": batched,
        "serving": serving,
        "status": status,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def run_encode(args, streams, stream, peaks):
    """Device encoding of the decoded streams (differential streams from their
    document ids), checked byte for byte against the encoded input and timed
    with CUDA events: Gints/s and the HBM roofline (4n read + bytes written)."""
    import torch
    from paper_1503_07387_gb300 import vbyte
    bufs = [torch.empty(5 * s["n"], dtype=torch.uint8, device="cuda") for s in streams]
    nbs = [torch.empty(1, dtype=torch.int64, device="cuda") for _ in streams]

    def step():
        for s, b, nb in zip(streams, bufs, nbs):
            vbyte.encode_device(s["d_out"], delta=s["delta"], out=b, nbytes=nb, stream=stream)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    exact = all(int(nb.item()) == s["host"].size and torch.equal(b[:s["host"].size], s["d_in"])
                for s, b, nb in zip(streams, bufs, nbs))
    reps = max(5, min(args.steps, 200))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    n = sum(s["n"] for s in streams)
    algo = sum(4 * s["n"] + s["host"].size for s in streams)
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = algo / (ms * 1e-3) / 1e9
    del bufs
    return {"value": round(n / (ms * 1e-3) / 1e9, 3), "unit": "Gints/s", "ms_per_step": round(ms, 5),
            "form": "vbyte_encode_device / vbyte_encode_delta_device, one launch per stream",
            "bit_exact_with_input": bool(exact), "status": int(vbyte.get_status()),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "algorithmic_bytes_per_step": algo}}


def run_decode64(args, stream, peaks):
    """64-bit VByte decoding (the format read for uint64): 2^26 sorted uint64
    document ids from 1 + Geometric(0.1) gaps above 2^40 (differential, almost
    all one-byte codes) and 2^26 values of every bit width 0..64 (plain, code
    lengths 1..10), checked bit for bit against the values the streams were
    built from and timed with CUDA events over the three launches of each
    call: Gints/s and the HBM roofline (input bytes + 8n per call)."""
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

    peak = peaks["hbm_gbs"] if peaks else 6800.0
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
    return {"form": "vbyte_decode_delta64 / vbyte_decode64 (count, scan and decode launches per call)",
            "status": status, "streams": res}


def run_batched(args, peaks):
    """Batched differential decoding of 100,000 rank-Zipf posting lists (about
    1.2e8 values): a tuned plan replayed from a CUDA graph against one
    vbyte_decode_delta call per list, both bit-exact and timed with CUDA
    events on the same stream."""
    import torch
    from paper_1503_07387_gb300 import vbyte
    ids, vo = inputs.posting_lists()
    L = vo.size - 1
    prev = inputs.full_range(L, seed=17)
    hb, hbo = vbyte.encode_batched(ids, vo, True, prev)
    n = int(vo[-1])
    del ids
    d = torch.from_numpy(hb).cuda()
    dbo = torch.from_numpy(hbo.view(np.int64)).cuda()
    dvo = torch.from_numpy(vo.view(np.int64)).cuda()
    dp = torch.from_numpy(prev.view(np.int32)).cuda()
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
    same = bool(torch.equal(out_b.view(torch.int32), out_e.view(torch.int32)))
    med = ms[len(ms) // 2]
    algo = hb.size + 4 * n + 16 * (L + 1)
    peak = peaks["hbm_gbs"] if peaks else 6800.0
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
        "speedup": round(each_ms / med, 2),
        "bit_exact_between_forms": same,
        "status": st_b | st_e,
    }
    plan.close()
    pool = dict(d=d, bo=hbo, vo=vo, prev=prev, lens=np.diff(vo).astype(np.int64))
    return res, pool


def run_serving(args, pool):
    """Open-loop Poisson query streams against the resident 100,000-list pool:
    each query names 2..8 lists drawn proportionally to length; continuous
    batching (gather + one batched launch per batch) against the same loop
    decoding every list with its own call.  Latency runs from a query's
    scheduled arrival to the scheduler seeing its batch complete."""
    import torch
    from paper_1503_07387_gb300 import vbyte
    # a query's output is about 27 MB (lists drawn in proportion to length):
    # 8 GiB holds four full batches of 64 queries in flight
    free, _ = torch.cuda.mem_get_info()
    arena = int(min(free * 0.25, 8 << 30)) // 4096 * 4096
    cfg = dict(arena_bytes=arena, staging_bytes=512 << 20, max_inflight=4, max_batch_queries=64,
               max_batch_lists=512)
    rows = []
    for rate in args.serve_rates:
        nq = int(min(max(rate * args.serve_seconds, 200), 40000))
        arr, qoff, ql = inputs.query_stream(pool["lens"], nq, float(rate), seed=40)
        vals = int(sum(int(pool["lens"][ql[qoff[i]:qoff[i + 1]]].sum()) for i in range(nq)))
        row = {"rate_qps": rate, "queries": nq, "values": vals}
        for form, per_list in (("batched", False), ("per_list", True)):
            srv = vbyte.Server(pool["d"], pool["bo"], pool["vo"], True, pool["prev"], per_list=per_list, **cfg)
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
    """The oracle (scalar Algorithm 1, one core) over the same streams, repeated
    until about budget_s seconds of CPU work."""
    import oracle
    reps = 0
    t0 = time.perf_counter()
    while True:
        for s in streams:
            if s["delta"]:
                oracle.decode_delta(s["host"], s["n"])
            else:
                oracle.decode(s["host"], s["n"])
        reps += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    total = reps * sum(s["n"] for s in streams)
    return {"value": round(total / dt / 1e9, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{reps} full pass(es) over every stream of the workload "
                      f"({total} values, {dt:.1f} s, single thread)"}


# --------------------------------------------------------------- reference arm --

def _prefix_bytes(data: np.ndarray, m: int) -> int:
    """Byte length of the first m integers of a well-formed stream."""
    if m <= 0:
        return 0
    ends = np.flatnonzero(data < 128)
    return int(ends[m - 1]) + 1


def run_reference(args):
    """The CPU oracle (scalar Algorithm 1, one core) on the same workload.  Each
    step decodes a bounded prefix of every stream, sized so that the whole
    --steps/--warmup run stays within about args.ref_seconds."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1503_07387_gb300 import vbyte
    oracle.build()
    streams = []
    for label, vals, delta in workload(args.workload):
        streams.append(dict(label=label, n=int(vals.size), delta=delta, host=vbyte.encode(vals)))
    # calibrate the oracle's speed on the first 2^20 values of each stream
    t0 = time.perf_counter()
    cal = 0
    for s in streams:
        m = min(s["n"], 1 << 20)
        nb = _prefix_bytes(s["host"], m)
        (oracle.decode_delta if s["delta"] else oracle.decode)(s["host"][:nb], m)
        cal += m
    rate = cal / max(time.perf_counter() - t0, 1e-6)
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
              f"single thread")
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
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=WORKLOADS, default="differential_2x2^26")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-seconds", type=float, default=120.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-encode", action="store_true")
    ap.add_argument("--no-decode64", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[2000, 5000, 10000, 20000, 50000])
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
