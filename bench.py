#!/usr/bin/env python3
"""Throughput of OblivGM's secure predicate evaluation (secEval, Alg. 3) on GB300.

One step = one fused evaluation of the bulk vertex filter: 1,048,576 vertices
with 4 uint32 attributes (uniform), secret-shared three ways and resident in
HBM; 8 predicates (4 equality / DPF, 4 range / 2 DCF each) at n = 32, each
evaluated by all three simulated servers (6 key halves), re-shared to RSS and
ANDed.  Metric: element-predicate evaluations per second (one unit = one
predicate on one element, all three servers, re-share included).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank evaluates its own replica of the workload (weak
scaling; the element filter needs no exchange between GPUs), timed between
barriers, max over ranks.  --impl reference times the CPU oracle on the host
cores on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workload as W  # noqa: E402

METRIC = "FSS predicate evals/s (element-predicate evaluations per second, 3 simulated servers)"
UNIT = "element-predicates/s"
N_VERTICES = 1 << 20
PRF = bytes(range(48))
KEY_SEED = bytes(range(16))
LOOKUPS_PER_AES = 160          # T-table AES-128: 16 table reads per round, 10 rounds
LDS_LANES_PER_CLK = 32         # shared-memory data path: one 4-byte word per lane per clock per SM


def aes_per_element(preds, n_bits=32):
    """FSS + re-share AES blocks one element costs for an AND-group of predicates."""
    fss = sum(6 * n_bits if p["kind"] == W.PRED_EQ else 6 * 2 * 2 * n_bits for p in preds)
    reshares = len(preds) + (len(preds) - 1)
    return fss + 3 * reshares


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def oracle_rate(wl, toks, seconds: float, threads: int, rng_seed: int = 0):
    """Time the oracle on a bounded sample of the workload; returns (units/s, sample size, seconds)."""
    import oracle
    tabs = [(t["shares"], t["bits"]) for t in wl["tables"]]
    g = W.rng(rng_seed)
    n = wl["tables"][0]["values"].shape[1]
    probe = g.integers(0, n, 4 * threads)
    t0 = time.perf_counter()
    oracle.filter_group(toks, 1, PRF, tabs, 0, probe, threads=threads)
    dt = time.perf_counter() - t0
    per_elem = dt / len(probe)
    size = max(threads, int(seconds / per_elem))
    sample = g.integers(0, n, size)
    t0 = time.perf_counter()
    oracle.filter_group(toks, 1, PRF, tabs, 0, sample, threads=threads)
    dt = time.perf_counter() - t0
    return size * len(wl["preds"]) / dt, size, dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    wl = W.bulk_vertex_filter(n_vertices=N_VERTICES, seed=2)
    toks = oracle.keygen(wl["preds"], 32, KEY_SEED)
    cores = os.cpu_count() or 1
    per_step_s = min(10.0, max(1.0, 120.0 / max(1, args.steps + args.warmup)))
    rates = []
    sample_desc = None
    for s in range(args.warmup + args.steps):
        r, size, dt = oracle_rate(wl, toks, per_step_s, cores, rng_seed=100 + s)
        if s >= args.warmup:
            rates.append(r)
            sample_desc = f"{size} random vertices of the 1,048,576-vertex table per step, all 8 predicates"
    value = statistics.mean(rates)
    units = len(wl["preds"]) * N_VERTICES
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": units / value * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": wl["name"], "elements": N_VERTICES, "predicates": 8,
                                            "n_bits": 32, "servers": 3},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample_desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import paper_2209_03526_gb300 as P

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    wl = W.bulk_vertex_filter(n_vertices=N_VERTICES, seed=2)
    preds = wl["preds"]
    units = len(preds) * N_VERTICES
    aes_step = aes_per_element(preds) * N_VERTICES
    toks = P.keygen(preds, 32, KEY_SEED)
    shares_dev = [torch.from_numpy(s.view(np.int32)).to(dev) for s in wl["tables"][0]["shares"]]
    ctx = P.Context(local, prf_keys=PRF)
    ctx.load_shares(0, shares_dev, 32)
    if args.schedule:
        threads, ept = (int(v) for v in args.schedule.split(","))
        ctx.set_schedule(threads, ept)
    else:
        threads, ept = ctx.autotune()
    outs = [[torch.empty(N_VERTICES, dtype=torch.int32, device=dev) for _ in range(3)]]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    for _ in range(args.warmup):
        ctx.filter_and_combine(1, toks, outs, stream)
    ctx.sync(stream)
    barrier()

    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            gpu_index = int(vis.split(",")[local])
        except (ValueError, IndexError):
            pass
    sampler = ClockSampler(gpu_index)
    sampler.start()
    launches0 = ctx.launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)                      # evict the shares from L2 between timed steps
        evs[k][0].record(stream)
        ctx.filter_and_combine(1 + k, toks, outs, stream)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = ctx.launch_count() - launches0
    ctx.sync(stream)
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_s = sum(step_ms) / 1e3
    if pg:
        t = torch.tensor([total_s], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        total_s = float(t.item())
    value = units * args.steps * world / total_s
    ms_per_step = total_s / args.steps * 1e3

    # ---- end to end through the public API with host buffers (pinned), every step:
    # upload the three share sets and the tokens, evaluate, read the result shares back
    host_shares = [torch.from_numpy(s.view(np.int32)).pin_memory() for s in wl["tables"][0]["shares"]]
    host_out = [torch.empty(N_VERTICES, dtype=torch.int32).pin_memory() for _ in range(3)]
    h2d = sum(t.numel() * 4 for t in host_shares) + sum(len(t) for t in toks)
    d2h = sum(t.numel() * 4 for t in host_out)
    e2e_steps = max(2, min(args.steps, 5))
    barrier()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        ctx.load_shares(0, host_shares, 32)
        ctx.filter_and_combine(1000 + k, toks, outs, stream)
        for h, d in zip(host_out, outs[0]):
            h.copy_(d, non_blocking=True)
        stream.synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0
    if pg:
        t = torch.tensor([e2e_s], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = units * e2e_steps * world / e2e_s

    peaks = measured_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_aes = sm_count * LDS_LANES_PER_CLK * max_mhz * 1e6 / LOOKUPS_PER_AES / 1e9
    achieved_aes = aes_step / (ms_per_step / 1e3) / 1e9
    roofline = {"bound": "alu", "achieved": achieved_aes, "peak": peak_aes, "unit": "GAES/s",
                "frac": achieved_aes / peak_aes, "traffic": None,
                "kernel": "k_filter", "pipe": "shared-memory T-table lookups (LSU), 160 per AES block",
                "peak_basis": f"{sm_count} SMs x {LDS_LANES_PER_CLK} lookups/clk x {max_mhz:.0f} MHz / 160"}
    traffic = os.path.join(ROOT, "profiles", "k_filter_traffic.json")
    if os.path.exists(traffic):
        try:
            with open(traffic) as f:
                tr = json.load(f)
            if tr.get("kernel_source_hash") == kernel_hash():
                roofline["traffic"] = tr.get("bytes_per_launch")
        except (OSError, ValueError):
            pass

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": wl["name"], "elements": N_VERTICES, "attributes": 4, "predicates": 8,
                       "predicate_mix": "4 equality (DPF) + 4 range (2 DCF)", "n_bits": 32, "ring": "Z_2^32",
                       "servers": 3, "combine": "RSS AND of all 8", "l2": "flushed between timed steps",
                       "schedule": {"threads": threads, "elems_per_thread": ept},
                       "aes_blocks_per_step": aes_step, "parallelism": f"replica x{world}"},
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps},
            "gpu_launches": launches,
            "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        toks_o = oracle.keygen(preds, 32, KEY_SEED)
        r, size, dt = oracle_rate(wl, toks_o, args.cpu_seconds, cores)
        line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{size} random vertices of the 1,048,576-vertex table, all 8 predicates, "
                                          f"{dt:.1f} s on {cores} threads"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if pg:
        pg.destroy_process_group()
    return 0


def run_profile_case(args):
    import torch
    import paper_2209_03526_gb300 as P
    n = 1 << 22
    g = W.rng(9)
    tab = W.table(W.uniform_attrs(g, 1, n, 32), 32, g)
    v = int(tab["values"][0, 123])
    preds = [W.eq_pred(0, 0, 0, v), W.range_pred(0, 0, 0, v // 2, min(0xFFFFFFFF, v + (1 << 30)))]
    toks = P.keygen(preds, 32, KEY_SEED)
    with P.Context(0, prf_keys=PRF) as ctx:
        ctx.load_shares(0, [torch.from_numpy(s.view(np.int32)).cuda() for s in tab["shares"]], 32)
        if args.schedule:
            ctx.set_schedule(*(int(x) for x in args.schedule.split(",")))
        outs = [[torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(3)]]
        for k in range(2):
            ctx.filter_and_combine(1 + k, toks, outs)
        ctx.sync()
    print(json.dumps({"profile_case": True, "elements": n, "aes_blocks_per_launch": aes_per_element(preds) * n}))
    return 0


def kernel_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("device_fss.cuh", "oblivgm.cu"):
        with open(os.path.join(ROOT, "paper_2209_03526_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--schedule", default="", help="threads,elems_per_thread (skips the autotuner)")
    ap.add_argument("--profile-case", action="store_true",
                    help="one small fused launch for ncu: 4,194,304 elements, 1 attribute, 1 equality + 1 range "
                         "predicate, after one warm-up launch")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
