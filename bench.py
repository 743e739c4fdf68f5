#!/usr/bin/env python3
"""Throughput and latency of OblivGM's secure predicate evaluation (secEval, Alg. 3) on GB300.

One step = one fused evaluation of the bulk vertex filter: 1,048,576 vertices
with 4 uint32 attributes (uniform), secret-shared three ways and resident in
HBM; 8 predicates (4 equality / DPF, 4 range / 2 DCF each) at n = 32, each
evaluated by all three simulated servers (6 key halves), re-shared to RSS and
ANDed.  Metric: element-predicate evaluations per second (one unit = one
predicate on one element, all three servers, re-share included), beside the
plain one-query-per-launch GPU path and query p50/p99 latency.

The same JSON line carries, under "workloads", one record per other workload
of the metric, each timed on its own with its own clocks, roofline, plain-path
comparison and oracle leg: the 1k/4k path query (n = 16), the triangle +
pendant query on a 1M-vertex / 10M-edge graph, 256 mixed queries in one
persistent launch replayed from a CUDA graph, the serving loop on a
4M-vertex / 40M-edge graph under Poisson arrivals, and the paper's one-hot
secEval on 107,614 vertices with 2^16-position one-hot vectors; then one record
each of secFetch case I (1,048,576 candidates, 4 attributes), secShuffle
(1,048,576 records) and the GPU keygen (2^20 key pairs of each kind).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank evaluates its own replica of the workload (weak
scaling; the element filter needs no exchange between GPUs), timed between
barriers, max over ranks; the per-workload records run on rank 0 of a
one-GPU run only.  --impl reference times the CPU oracle on the host cores on
bounded samples of the same workload.
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
SEED_B = bytes(range(16, 32))
LOOKUPS_PER_AES = 160          # T-table AES-128: 16 table reads per round, 10 rounds
LOOKUPS_PER_AES_W0 = 148       # ... when only output word 0 is used (DCF value block, re-share PRF)
LDS_LANES_PER_CLK = 32         # shared-memory data path: one 4-byte word per lane per clock per SM


def aes_per_element(preds, n_bits=32):
    """FSS + re-share AES blocks one element costs for an AND-group of predicates."""
    fss = sum(6 * n_bits if p["kind"] == W.PRED_EQ else 6 * 2 * 2 * n_bits for p in preds)
    reshares = len(preds) + (len(preds) - 1)
    return fss + 3 * reshares


def lookups_per_element(preds, n_bits=32):
    """Shared-memory T-table lookups one element costs: DPF walks 160 per level, DCF walks
    160 + 148 per level (seed block + value word), re-shares 148 per PRF call."""
    fss = sum(6 * n_bits * LOOKUPS_PER_AES if p["kind"] == W.PRED_EQ
              else 12 * n_bits * (LOOKUPS_PER_AES + LOOKUPS_PER_AES_W0) for p in preds)
    return fss + 3 * (2 * len(preds) - 1) * LOOKUPS_PER_AES_W0


def keygen_blocks_per_pair(dcf: bool, n_bits: int = 32):
    """AES blocks (full, value-word-only) of one key pair's Gen on the GPU: the two root seeds
    from the client seed, then per level both parties' seeds expanded in both directions
    (4 blocks) and, for a DCF, the 4 value words of those children."""
    return 2 + 4 * n_bits, (4 * n_bits if dcf else 0)


def plain_and(preds, values):
    """Plaintext AND of a group's predicates (Def. 2), for the checks of the timed modes."""
    res = np.ones(values.shape[1], dtype=np.uint64)
    for p in preds:
        v = values[p["attr"]].astype(np.uint64)
        res &= ((v == p["lo"]) if p["kind"] == W.PRED_EQ else ((v >= p["lo"]) & (v <= p["hi"]))).astype(np.uint64)
    return res


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


def make_reduce_max(dist_mod, device):
    """max over ranks of a host float (all_reduce MAX on a one-element tensor)."""
    def reduce_max(x: float) -> float:
        import torch
        t = torch.tensor([float(x)], device=device, dtype=torch.float64)
        dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
        return float(t.item())
    return reduce_max


def aggregate_ranks(local_seconds: float, units_per_step: int, steps: int, world: int, reduce_max=None):
    """Whole-job throughput of weak-scaled replicas: every rank's units over the slowest rank's time."""
    t = reduce_max(local_seconds) if reduce_max else local_seconds
    return units_per_step * steps * world / t, t


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


def oracle_leg(run, units: float, unit: str, cores: int, sample: str, target_s: float = 4.0):
    """Time the oracle as it stands on a bounded sample: run(scale) does `scale` units' worth of
    oracle work (scale = 1 is the smallest sample); one probe, then a run of about target_s."""
    t0 = time.perf_counter()
    run(1)
    dt = time.perf_counter() - t0
    scale = 1
    if dt < 0.5 * target_s:               # a probe that already took long enough is the measurement
        scale = max(1, int(target_s / max(dt, 1e-6)))
        t0 = time.perf_counter()
        run(scale)
        dt = time.perf_counter() - t0
    return {"value": units * scale / dt, "unit": unit, "cores": cores, "kind": "oracle",
            "sample": f"{sample}, x{scale} ({dt:.1f} s)"}


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
    rates, secs, sizes = [], [], []
    for s in range(args.warmup + args.steps):
        r, size, dt = oracle_rate(wl, toks, per_step_s, cores, rng_seed=100 + s)
        if s >= args.warmup:
            rates.append(r)
            secs.append(dt)
            sizes.append(size)
    # a step is one bounded sample of the table (all 8 predicates on `size` random vertices);
    # value = element-predicates of the timed samples over their measured seconds
    units = len(wl["preds"]) * sum(sizes)
    value = units / sum(secs)
    sample_desc = (f"{min(sizes)}-{max(sizes)} random vertices of the 1,048,576-vertex table per step, all 8 "
                   f"predicates, {statistics.mean(secs):.2f} s per step on {cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(secs) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": wl["name"], "elements": N_VERTICES, "attributes": 4,
                                            "predicates": 8, "n_bits": 32, "servers": 3,
                                            "step": "one bounded random sample of the table (oracle, all host cores)"},
            "measured_seconds_per_step": statistics.mean(secs),
            "extrapolated_full_table_ms_per_step": len(wl["preds"]) * N_VERTICES / value * 1e3,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample_desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def gpu_index_of(local: int) -> int:
    """nvidia-smi index of this process's CUDA device (honours CUDA_VISIBLE_DEVICES)."""
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            return int(vis.split(",")[local])
        except (ValueError, IndexError):
            pass
    return local


LDS_PIPE = "shared-memory (LDS/MIO) AES T-table lookups, one 4-byte word per lane per clock per SM"


def lookup_roofline(lookups: float, seconds: float, peak_lu: float, aes: float | None = None) -> dict:
    """Roofline record of a filter run against the shared-memory T-table lookup ceiling."""
    ach = lookups / seconds / 1e9
    out = {"bound": "lds", "achieved": ach, "peak": peak_lu, "unit": "Glookup/s", "frac": ach / peak_lu,
           "traffic": None, "pipe": LDS_PIPE}
    if aes is not None:
        out["aes_blocks_per_s"] = aes / seconds
    return out


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
    # the autotuner's AES-layout dimension: the walks are built in the layout it measures faster
    lay, tt_rate, bs_rate = (None, None, None) if args.no_compare else ctx.autotune_aes_layout()
    outs = [[torch.empty(N_VERTICES, dtype=torch.int32, device=dev) for _ in range(3)]]
    stream = torch.cuda.current_stream(dev)
    flush = L2Flush(torch, dev, stream)

    for _ in range(args.warmup):
        ctx.filter_and_combine(1, toks, outs, stream)
    ctx.sync(stream)
    barrier()

    sampler = ClockSampler(gpu_index_of(local))
    sampler.start()
    launches0 = ctx.launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        flush()                                    # evict the shares from L2 between timed steps
        evs[k][0].record(stream)
        ctx.filter_and_combine(1 + k, toks, outs, stream)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = ctx.launch_count() - launches0
    ctx.sync(stream)
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    reduce_max = make_reduce_max(pg, dev) if pg else None
    value, total_s = aggregate_ranks(sum(step_ms) / 1e3, units, args.steps, world, reduce_max)
    ms_per_step = total_s / args.steps * 1e3
    rec = (sum(o.cpu().numpy().view(np.uint32).astype(np.uint64) for o in outs[0]) & 0xFFFFFFFF)
    parity_ok = bool(np.array_equal(rec, plain_and(preds, wl["tables"][0]["values"])))

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
    e2e_value, e2e_s = aggregate_ranks(time.perf_counter() - t0, units, e2e_steps, world, reduce_max)

    peaks = measured_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    lookups_step = lookups_per_element(preds) * N_VERTICES
    peak_lu = sm_count * LDS_LANES_PER_CLK * max_mhz * 1e6 / 1e9
    roofline = lookup_roofline(lookups_step, ms_per_step / 1e3, peak_lu, aes_step)
    roofline.update({"kernel": "k_filter", "peak_basis": f"{sm_count} SMs x {LDS_LANES_PER_CLK} lookups/clk x "
                                                         f"{max_mhz:.0f} MHz (sm_max_mhz of MEASURED_PEAKS.json)",
                     "lookups_per_step": lookups_step})
    rec_traffic = kernel_record("k_filter_traffic.json")
    if rec_traffic:
        roofline["traffic"] = rec_traffic.get("bytes_per_launch")
    rec_issue = kernel_record("k_filter_issue.json")
    if rec_issue:
        # every instruction the kernel issues, per AES block (ncu), against the SMs' issue slots
        # for 32-bit integer work: 128 lanes per clock per SM
        ipb = float(rec_issue["thread_inst_per_aes_block"])
        roofline["int32_issue_frac"] = roofline["aes_blocks_per_s"] * ipb / (sm_count * 128 * max_mhz * 1e6)
        roofline["int32_issue_basis"] = (f"AES blocks/s x {ipb:.1f} thread-instructions per block (ncu, "
                                         f"{rec_issue['source']}) / ({sm_count} SMs x 128 lanes x {max_mhz:.0f} MHz)")

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": wl["name"], "elements": N_VERTICES, "attributes": 4, "predicates": 8,
                       "predicate_mix": "4 equality (DPF) + 4 range (2 DCF)", "n_bits": 32, "ring": "Z_2^32",
                       "servers": 3, "combine": "RSS AND of all 8", "l2": "flushed between timed steps",
                       "schedule": {"threads": threads, "elems_per_thread": ept,
                                    "aes_layout": None if lay is None else {
                                        "chosen": "bitsliced" if lay == P.AES_BITSLICED else "T-table",
                                        "ttable_prg_blocks_per_s": tt_rate, "bitsliced_prg_blocks_per_s": bs_rate},
                                    "vector_width": "32-bit coalesced share loads and output stores: the "
                                                    "one-element-per-thread shape the autotuner picks; the "
                                                    "128-bit four-element shape spills and runs 1.5x slower, "
                                                    "and shares are ~1e-5 of the kernel's time"},
                       "aes_blocks_per_step": aes_step, "parallelism": f"replica x{world}",
                       "reconstructs_to_plaintext": parity_ok},
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps},
            "gpu_launches": launches,
            "clocks": clocks,
            # per element: 6 DPF key-half walks per equality predicate, 12 DCF walks per range
            "secondary_units": {
                "key_half_walks_per_s": sum(6 if p["kind"] == W.PRED_EQ else 12 for p in preds) * N_VERTICES
                / (ms_per_step / 1e3),
                "aes_blocks_per_s": roofline["aes_blocks_per_s"]}}
    # ---- the plain per-query GPU path on the same step (same shares, parity-tested)
    if not args.no_compare:
        l0 = ctx.launch_count()
        ctx.filter_plain(1, toks, outs, stream)          # warm-up
        stream.synchronize()
        plain_launches = ctx.launch_count() - l0
        plain_s = time_plain(ctx, [toks], [outs], stream, reps=2)
        line["plain_path"] = {"value": units / plain_s, "unit": UNIT, "ms_per_step": plain_s * 1e3,
                              "gpu_launches_per_step": plain_launches,
                              "what": "per predicate: open + one launch per key half (6 DPF / 12 DCF walks, "
                                      "global-memory AES tables) + sum/re-share + AND launches",
                              "fused_speedup": value / (units / plain_s)}
        line["latency"] = latency_leg(ctx, P, torch, dev, wl, roofline["aes_blocks_per_s"], stream,
                                      args.latency_queries, args.latency_plain)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        toks_o = oracle.keygen(preds, 32, KEY_SEED)
        r, size, dt = oracle_rate(wl, toks_o, args.cpu_seconds, cores)
        line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{size} random vertices of the 1,048,576-vertex table, all 8 predicates, "
                                          f"{dt:.1f} s on {cores} threads"}
    # context only (another method, machine and workload): the paper's Table 2 secEval time for
    # 10,000 candidates with an equality predicate, one-hot keys, 3 V100 servers and a network
    line["paper_context"] = {"secEval_10000_candidates_eq_s": 2.6, "candidate_predicates_per_s": 10000 / 2.6,
                             "hardware": "3 x Tesla V100 (one per server), 2.5 Gbps network",
                             "note": "not the same workload or metric; not used for vs_baseline"}
    ctx.close()
    del outs, shares_dev, flush
    torch.cuda.empty_cache()
    # ---- the metric's other workloads, one record each (one GPU only: they are not replicated)
    if not args.no_compare and world == 1 and args.workloads:
        line["workloads"] = {}
        for name in [w for w in args.workloads.split(",") if w]:
            t0 = time.perf_counter()
            line["workloads"][name] = WORKLOAD_RECORDS[name](P, torch, args, (threads, ept))
            line["workloads"][name]["wall_s"] = time.perf_counter() - t0
            torch.cuda.empty_cache()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def latency_leg(ctx, P, torch, dev, wl, aes_per_s, stream, n_queries: int, plain_k: int) -> dict:
    """Query latency under Poisson arrivals at half the fused path's measured capacity: queries
    of 1-8 predicates (one AND-group) on the resident 1,048,576-vertex table, served by the
    serving loop (continuous batching); the plain path serves the first plain_k arrivals as a
    FIFO at the same arrival times."""
    g = W.rng(77)
    tabs = wl["tables"]
    qlist = []
    for _ in range(n_queries):
        q = W.random_query(g, tabs, 32, int(g.integers(1, 9)), 1, vertex_table=0, edge_table=0)
        qlist.append(q["preds"])
    toks_q = [P.keygen(q, 32, struct_seed(i)) for i, q in enumerate(qlist)]
    table_n = {0: N_VERTICES}
    svc = [query_aes(q, table_n) / aes_per_s for q in qlist]
    rate = 0.5 / float(np.mean(svc))
    arrivals = np.cumsum(g.exponential(1.0 / rate, len(qlist)))
    arrivals -= arrivals[0]
    lat, tot, rej = serve_latency(ctx, toks_q, arrivals, P)
    k = min(plain_k, n_queries)
    plain_outs = [query_outs(torch, dev, q, table_n) for q in qlist[:k]]
    plat, ptot = plain_latency(ctx, toks_q[:k], plain_outs, arrivals[:k], stream)
    del plain_outs
    return {"queries": len(qlist), "arrival": "Poisson", "rate_qps": rate, "offered_load": "50% of fused capacity",
            "predicates_per_query": "1-8 (uniform), one AND-group on the resident table",
            "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "max_ms": float(np.max(lat) * 1e3),
            "completed_qps": len(qlist) / tot, "rejected": rej,
            "plain_queries": k, "plain_p50_ms": pct(plat, 50), "plain_p99_ms": pct(plat, 99),
            "fused_p50_ms_same_queries": pct(lat[:k], 50), "fused_p99_ms_same_queries": pct(lat[:k], 99),
            "plain_completed_qps": k / ptot}


def struct_seed(i: int) -> bytes:
    """16-byte client seed of query i."""
    return bytes([i % 256, (i >> 8) % 256]) + bytes(14)


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
    """Hash of the k_filter source: the device AES/FSS and async-copy headers and the kernel's
    part of oblivgm.cu (from the PTX helpers to the raw-batch section), so host-code edits
    elsewhere do not invalidate a capture."""
    import hashlib
    h = hashlib.sha256()
    for hdr in ("device_fss.cuh", "ptx_async.cuh"):
        with open(os.path.join(ROOT, "paper_2209_03526_gb300", "csrc", hdr), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(ROOT, "paper_2209_03526_gb300", "csrc", "oblivgm.cu"), "rb") as fh:
        src = fh.read()
    a = src.index(b"// ------------------------------------------------------------------ PTX helpers")
    b = src.index(b"// ------------------------------------------------------------------ raw batches")
    h.update(src[a:b])
    return h.hexdigest()[:16]


def kernel_record(name: str):
    """An ncu record under profiles/ taken on the current k_filter source, else None."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    return rec if rec.get("kernel_source_hash") == kernel_hash() else None


def query_aes(preds, table_n, n_bits=32):
    """Algorithmic AES blocks of one query: per AND-group, its per-element cost times its table's size."""
    groups = {}
    for p in preds:
        groups.setdefault(p["group"], []).append(p)
    return sum(aes_per_element(g, n_bits) * table_n[g[0]["table"]] for g in groups.values())


def query_lookups(preds, table_n, n_bits=32):
    groups = {}
    for p in preds:
        groups.setdefault(p["group"], []).append(p)
    return sum(lookups_per_element(g, n_bits) * table_n[g[0]["table"]] for g in groups.values())


def query_units(preds, table_n):
    return sum(table_n[p["table"]] for p in preds)


def query_outs(torch, dev, preds, table_n):
    ng = max(p["group"] for p in preds) + 1
    tab = {p["group"]: p["table"] for p in preds}
    return [[torch.empty(table_n[tab[g]], dtype=torch.int32, device=dev) for _ in range(3)] for g in range(ng)]


def serve_latency(ctx, toks_list, arrivals, P):
    """Real-time arrivals through submit/poll/release.  Latency runs from a query's scheduled
    arrival to the moment its completion is seen; a query the loop cannot admit yet waits in a
    client-side backlog (counted as rejected once) and is resubmitted as results are released."""
    from collections import deque
    n = len(toks_list)
    t0 = time.perf_counter()
    nxt, done = 0, 0
    backlog, inflight = deque(), {}
    lat = [0.0] * n
    rejected = set()
    while done < n:
        now = time.perf_counter() - t0
        while nxt < n and arrivals[nxt] <= now:
            backlog.append(nxt)
            nxt += 1
        while backlog:
            i = backlog[0]
            try:
                tk = ctx.submit(toks_list[i])
            except P.OblivgmError as e:
                if e.status != P.EAGAIN:
                    raise
                rejected.add(i)
                break
            backlog.popleft()
            inflight[tk] = i
        progressed = False
        for tk in list(inflight):
            if ctx.poll(tk, 0) is not None:
                i = inflight.pop(tk)
                lat[i] = time.perf_counter() - t0 - arrivals[i]
                ctx.release(tk)
                done += 1
                progressed = True
        if not progressed:
            if not inflight and not backlog and nxt < n:
                time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
            else:
                time.sleep(0.0002)
    return lat, time.perf_counter() - t0, len(rejected)


def plain_latency(ctx, toks_list, outs_list, arrivals, stream):
    """The plain per-query path as a FIFO server: one query at a time, in arrival order."""
    t0 = time.perf_counter()
    lat = []
    for i, toks in enumerate(toks_list):
        wait = arrivals[i] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        ctx.filter_plain(5000 + i, toks, outs_list[i], stream)
        stream.synchronize()
        lat.append(time.perf_counter() - t0 - arrivals[i])
    return lat, time.perf_counter() - t0


def pct(xs, q):
    return float(np.percentile(np.asarray(xs) * 1e3, q))


class L2Flush:
    """Reads a buffer larger than the 129 MB L2 on `stream` (None: the current stream), so
    that the next timed step starts with its inputs in HBM; called between timed steps,
    outside the events.  A read leaves clean lines behind: a write would leave the L2 full
    of dirty lines whose write-back the next step would pay for."""

    def __init__(self, torch, dev, stream=None):
        self.torch, self.stream = torch, stream
        self.buf = torch.zeros(64 << 20, dtype=torch.int32, device=dev)     # 256 MB

    def __call__(self):
        s = self.stream if self.stream is not None else self.torch.cuda.current_stream()
        with self.torch.cuda.stream(s):
            self.buf.max()


def time_plain(ctx, toks_list, outs_list, stream, reps=1):
    """Seconds the plain path takes for the listed queries, run one after another."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        for i, toks in enumerate(toks_list):
            ctx.filter_plain(7000 + i, toks, outs_list[i], stream)
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / 1e3 / reps


def _load_graph(ctx, torch, dev, graph):
    for tid, t in enumerate(graph["tables"]):
        ctx.load_shares(tid, [torch.from_numpy(x.view(np.int32)).to(dev) for x in t["shares"]], t["bits"])
    return {tid: t["values"].shape[1] for tid, t in enumerate(graph["tables"])}


def _timed_graph(torch, ctx, plan, stream, warmup, steps):
    """Launch a plan `warmup` times, capture one launch in a CUDA graph and time `steps` replays,
    each after an L2 flush."""
    for _ in range(warmup):
        ctx.plan_launch(plan, stream)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ctx.plan_launch(plan, torch.cuda.current_stream())
    torch.cuda.synchronize()
    flush = L2Flush(torch, torch.device("cuda", torch.cuda.current_device()))
    evs = []
    for _ in range(steps):
        # queued without waiting: the flush before each replay keeps the GPU busy while the host
        # submits the replay, so the events time the device's work and not the submission
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        evs.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def sampled_parity(torch, graph, queries, outs, k_elems=4096, seed=21) -> bool:
    """Every group of the given queries: the three output share sets, read back at k_elems random
    elements plus the first and the last, reconstruct to the plaintext AND of the group's
    predicates (Def. 2) at those elements."""
    g = W.rng(seed)
    ok = True
    for q, out in zip(queries, outs):
        groups = {}
        for p in q["preds"]:
            groups.setdefault(p["group"], []).append(p)
        for grp, gp in groups.items():
            vals = graph["tables"][gp[0]["table"]]["values"]
            n = vals.shape[1]
            idx = np.unique(np.concatenate([g.integers(0, n, min(k_elems, n)), [0, n - 1]]))
            it = torch.from_numpy(idx.astype(np.int64)).to(out[grp][0].device)
            rec = sum(o.index_select(0, it).cpu().numpy().view(np.uint32).astype(np.uint64) for o in out[grp])
            ok &= bool(np.array_equal(rec & 0xFFFFFFFF, plain_and(gp, vals[:, idx])))
    return ok


def oracle_query_leg(graph, toks_o, preds, seconds: float, what: str, seed: int = 31) -> dict:
    """The oracle as it stands, on all host cores, on random elements of every group of one query
    (the same number per group), sized to take about `seconds`; element-predicates/s."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    tabs = [(t["shares"], t["bits"]) for t in graph["tables"]]
    groups = {}
    for p in preds:
        groups.setdefault(p["group"], []).append(p)
    g = W.rng(seed)

    def run(m):
        units, t0 = 0, time.perf_counter()
        for grp, gp in groups.items():
            n = graph["tables"][gp[0]["table"]]["values"].shape[1]
            elems = g.integers(0, n, m)
            oracle.filter_group(toks_o, 1, PRF, tabs, grp, elems, threads=cores)
            units += m * len(gp)
        return units, time.perf_counter() - t0

    u, dt = run(2 * cores)
    m = max(2 * cores, int(2 * cores * seconds / max(dt, 1e-6)))
    u, dt = run(m)
    return {"value": u / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{m} random elements of each of the query's {len(groups)} groups ({what}), "
                      f"{dt:.1f} s on {cores} threads"}


def filter_workload_record(P, torch, name: str, graph, queries, sched, steps: int, warmup: int, plain_k: int,
                           cpu_seconds: float, no_cpu: bool, plain_reps: int = 1) -> dict:
    """One filter workload, timed on its own: the queries as one prepared batch (one persistent
    launch) captured in a CUDA graph and replayed, L2 flushed before every replay; the plain
    per-query path on the first plain_k queries beside the fused launch on the same queries;
    sampled reconstruction against plaintext; the oracle on a bounded sample of query 0."""
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    peaks = measured_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_lu = sm_count * LDS_LANES_PER_CLK * max_mhz / 1e3
    n_bits = graph["n_bits"]
    ctx = P.Context(0, prf_keys=PRF)
    ctx.set_schedule(*sched)
    table_n = _load_graph(ctx, torch, dev, graph)
    toks = [P.keygen(q["preds"], n_bits, struct_seed(i)) for i, q in enumerate(queries)]
    outs = [query_outs(torch, dev, q["preds"], table_n) for q in queries]
    qids = list(range(1, len(queries) + 1))
    units = sum(query_units(q["preds"], table_n) for q in queries)
    aes = sum(query_aes(q["preds"], table_n, n_bits) for q in queries)
    lookups = sum(query_lookups(q["preds"], table_n, n_bits) for q in queries)
    # the plain per-query path on the first plain_k queries, beside the fused launch of the same
    # queries; those fused launches also warm the kernel up before the timed replays
    plain = None
    if plain_k:
        k = min(plain_k, len(queries))
        sub = list(range(k))
        plan = ctx.plan_create([qids[i] for i in sub], [toks[i] for i in sub], [outs[i] for i in sub])
        fms = _timed_graph(torch, ctx, plan, stream, 1, 2)
        ctx.plan_destroy(plan)
        l0 = ctx.launch_count()
        ps = time_plain(ctx, [toks[i] for i in sub], [outs[i] for i in sub], stream, reps=plain_reps)
        plain_launches = (ctx.launch_count() - l0) // plain_reps
        u = sum(query_units(queries[i]["preds"], table_n) for i in sub)
        pl = sum(query_lookups(queries[i]["preds"], table_n, n_bits) for i in sub)
        plain = {"queries": k, "value": u / ps, "unit": UNIT, "ms": ps * 1e3, "gpu_launches": plain_launches,
                 "fused_value_same_queries": u / (np.mean(fms) / 1e3), "fused_speedup": ps / (np.mean(fms) / 1e3),
                 "frac_of_lookup_ceiling": pl / ps / 1e9 / peak_lu}
    plan = ctx.plan_create(qids, toks, outs)
    shape = ctx.plan_describe(plan)
    sampler = ClockSampler(gpu_index_of(0))
    sampler.start()
    ms = _timed_graph(torch, ctx, plan, stream, warmup, steps)
    clocks = sampler.stop()
    ctx.plan_destroy(plan)
    step_s = float(np.mean(ms)) / 1e3
    k_check = min(8, len(queries))
    rec = {"metric": METRIC, "value": units / step_s, "unit": UNIT, "ms_per_step": step_s * 1e3,
           "steps": steps, "warmup": warmup, "gpu_launches": steps,
           "config": {"workload": name, "queries": len(queries), "element_predicates_per_step": units,
                      "aes_blocks_per_step": aes, "tables": {str(k): v for k, v in table_n.items()},
                      "n_bits": n_bits, "l2": "flushed between timed steps",
                      "launch": f"one persistent {shape['kernel']} launch ({shape['grid']} CTAs x "
                                f"{shape['threads']} threads, {shape['items']} tiles of up to {shape['tile']} "
                                "elements) replayed from a CUDA graph",
                      "warmup_launches": f"{warmup} of this plan" + (
                          f", after 3 of the first {plain['queries']} queries' plan (same kernel)" if plain else ""),
                      "reconstructs_to_plaintext_sampled": sampled_parity(torch, graph, queries[:k_check],
                                                                          outs[:k_check]),
                      "parity_queries_checked": k_check},
           "roofline": lookup_roofline(lookups, step_s, peak_lu, aes),
           "clocks": clocks}
    rec["roofline"]["kernel"] = shape["kernel"]
    if plain:
        rec["plain_path"] = plain
    ctx.close()
    del outs
    if not no_cpu:
        import oracle
        toks_o = oracle.keygen(queries[0]["preds"], n_bits, struct_seed(0))
        rec["cpu_baseline"] = oracle_query_leg(graph, toks_o, queries[0]["preds"], cpu_seconds, "query 0")
    return rec


def record_tiny(P, torch, args, sched) -> dict:
    """1,000 vertices / 4,000 edges, 3-vertex path query, one equality + one range predicate, n = 16."""
    wl = W.tiny_path(seed=1)
    graph = {"tables": wl["tables"], "n_bits": 16}
    # a step is ~0.06 ms: 3,000 timed replays keep the clock sampler (200 ms period) in the region
    return filter_workload_record(P, torch, wl["name"], graph, [{"preds": wl["preds"]}], sched,
                                  steps=args.sub_steps or 3000, warmup=3, plain_k=1, cpu_seconds=4.0,
                                  no_cpu=args.no_cpu_baseline, plain_reps=5)


def record_edges(P, torch, args, sched) -> dict:
    """Triangle + pendant (4 vertices, 4 edges, 6 mixed predicates) on a 1M-vertex / 10M-edge graph."""
    graph = W.edge_graph(1_000_000, 10_000_000, 2, 2, seed=3)
    return filter_workload_record(P, torch, "triangle_pendant_1Mv_10Me_6pred_n32", graph,
                                  [W.triangle_pendant(graph, seed=3)], sched, steps=args.sub_steps or 3, warmup=1,
                                  plain_k=1, cpu_seconds=4.0, no_cpu=args.no_cpu_baseline)


def record_batch(P, torch, args, sched) -> dict:
    """256 queries (2-8 vertices, 1-6 predicates) on the 1M / 10M graph with 4 vertex attributes,
    one persistent launch replayed from a CUDA graph; plain path on the first 8 queries."""
    graph = W.edge_graph(1_000_000, 10_000_000, 4, 2, seed=4)
    return filter_workload_record(P, torch, "query_mix_256q_1Mv_10Me_n32", graph, W.query_mix(graph, 256, seed=4),
                                  sched, steps=args.sub_steps or 1, warmup=0, plain_k=8, cpu_seconds=4.0,
                                  no_cpu=args.no_cpu_baseline)


def record_serve(P, torch, args, sched) -> dict:
    """The serving loop on a 4M-vertex / 40M-edge graph resident in HBM: Poisson arrivals of mixed
    queries at 50, 200 and 1000 queries/s (args.serve_overload_queries arrivals each) and at half
    the estimated capacity (args.serve_queries arrivals); the plain path serves the first
    args.plain_queries arrivals of each rate as a FIFO at the same arrival times.  Above capacity
    the queue only grows, so there the completed rate is the figure and the latencies say how
    long the arrivals took to drain; the rate below capacity gives the steady-state p50/p99."""
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    peaks = measured_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_lu = sm_count * LDS_LANES_PER_CLK * float(peaks.get("sm_max_mhz", 2070.0)) / 1e3
    peak_aes = peak_lu / LOOKUPS_PER_AES
    graph = W.edge_graph(4_000_000, 40_000_000, 4, 2, seed=5)
    ctx = P.Context(0, prf_keys=PRF)
    ctx.set_schedule(*sched)
    table_n = _load_graph(ctx, torch, dev, graph)
    n_over, n_cal = args.serve_overload_queries, args.serve_queries
    queries = W.query_mix(graph, max(n_over, n_cal), seed=5)
    toks = [P.keygen(q["preds"], 32, struct_seed(i)) for i, q in enumerate(queries)]
    svc = [query_aes(q["preds"], table_n) / (peak_aes * 0.95e9) for q in queries]
    capacity = 1.0 / float(np.mean(svc))
    rates = [(50.0, n_over), (200.0, n_over), (1000.0, n_over), (0.5 * capacity, n_cal)]
    runs = []
    g = W.rng(55)
    sampler = ClockSampler(gpu_index_of(0))
    sampler.start()
    l0 = ctx.launch_count()
    sat_units = sat_lookups = sat_aes = 0.0
    for ri, (rate, n_arr) in enumerate(rates):
        units = sum(query_units(q["preds"], table_n) for q in queries[:n_arr])
        lookups = sum(query_lookups(q["preds"], table_n) for q in queries[:n_arr])
        if ri < 3:
            sat_units += units
            sat_lookups += lookups
            sat_aes += sum(query_aes(q["preds"], table_n) for q in queries[:n_arr])
        arrivals = np.cumsum(g.exponential(1.0 / rate, n_arr))
        arrivals -= arrivals[0]
        lat, tot, rej = serve_latency(ctx, toks[:n_arr], arrivals, P)
        run = {"rate_qps": rate, "queries": n_arr, "completed_qps": n_arr / tot, "wall_s": tot,
               "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "max_ms": float(np.max(lat) * 1e3),
               "rejected": rej, "element_predicates_per_s": units / tot,
               "frac_of_lookup_ceiling": lookups / tot / 1e9 / peak_lu}
        if args.plain_queries:
            k = min(args.plain_queries, n_arr)
            pouts = [query_outs(torch, dev, queries[i]["preds"], table_n) for i in range(k)]
            plat, ptot = plain_latency(ctx, toks[:k], pouts, arrivals[:k], stream)
            del pouts
            run.update({"plain_queries": k, "plain_p50_ms": pct(plat, 50), "plain_p99_ms": pct(plat, 99),
                        "fused_p50_ms_same_queries": pct(lat[:k], 50),
                        "fused_p99_ms_same_queries": pct(lat[:k], 99)})
        runs.append(run)
    launches = ctx.launch_count() - l0
    clocks = sampler.stop()
    ctx.close()
    sat = runs[:3]
    sat_s = sum(r["wall_s"] for r in sat)
    rec = {"metric": METRIC + " and query p50/p99 latency", "value": sat_units / sat_s, "unit": UNIT,
           "ms_per_query": sat_s / (3 * n_over) * 1e3, "steps": 3 * n_over, "warmup": 0,
           "gpu_launches": launches,
           "config": {"workload": "serve_4Mv_40Me_mixed_queries_n32", "tables": {str(k): v for k, v in table_n.items()},
                      "queries": "2-8 vertices, 1-6 predicates (uniform)",
                      "arrivals_per_rate": {"overloaded": n_over, "half_capacity": n_cal},
                      "estimated_capacity_qps": capacity,
                      "value": "element-predicates completed per second over the three overloaded rates "
                               "(50, 200, 1000 q/s)",
                      "launches": "the serving loop's fused batches on two streams (continuous batching); "
                                  "plain path FIFO on the same arrival prefix"},
           "roofline": lookup_roofline(sat_lookups, sat_s, peak_lu, sat_aes),
           "serving": runs, "clocks": clocks}
    if not args.no_cpu_baseline:
        import oracle
        toks_o = oracle.keygen(queries[0]["preds"], 32, struct_seed(0))
        rec["cpu_baseline"] = oracle_query_leg(graph, toks_o, queries[0]["preds"], 4.0, "query 0 of the mix")
    return rec


def record_onehot(P, torch, args, sched, ctx=None, steps=None, warmup=None) -> dict:
    """The paper's secEval as written (one-hot mode): one 16-bit attribute of 107,614 vertices
    (the size of the paper's graph) as binary-RSS one-hot vectors of 2^16 positions (2.64 GB
    resident), four predicates on that column in three AND-groups, one filter_onehot call per
    step with the L2 flushed before it."""
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    own = ctx is None
    if own:
        ctx = P.Context(0, prf_keys=PRF)
    steps = steps or args.sub_steps or 1000
    warmup = max(3, warmup or 3)
    n_v, n = 107_614, 16
    g = W.rng(6)
    vals = W.uniform_attrs(g, 1, n_v, n)
    tab = W.onehot_table(vals, n, g)
    ctx.load_onehot(0, [torch.from_numpy(x.view(np.int32)).to(dev) for x in tab["shares"]], n)
    del tab
    v0, v1 = int(vals[0, 11]), int(vals[0, 22])
    preds = [W.eq_pred(0, 0, 0, v0), W.range_pred(0, 0, 1, v1 // 2, min((1 << n) - 1, v1 + 9000)),
             W.eq_pred(0, 0, 2, v1), W.range_pred(0, 0, 2, v1 // 3, (1 << n) - 1)]
    toks = P.keygen_onehot(preds, n, KEY_SEED)
    words_out = (n_v + 31) // 32
    outs = [[torch.empty(words_out, dtype=torch.int32, device=dev) for _ in range(3)] for _ in range(3)]
    for _ in range(warmup):
        ctx.filter_onehot(1, toks, outs, stream)
    ctx.sync(stream)
    flush = L2Flush(torch, dev, stream)
    l0 = ctx.launch_count()
    sampler = ClockSampler(gpu_index_of(0))
    sampler.start()
    ms = []
    for k in range(steps):
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.filter_onehot(2 + k, toks, outs, stream)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    clocks = sampler.stop()
    launches = (ctx.launch_count() - l0) // steps
    ctx.sync(stream)
    # the last step's bits reconstruct to the plaintext predicates (every element)
    got = [np.stack([np.unpackbits(t.cpu().numpy().view(np.uint8), bitorder="little")[:n_v] for t in outs[gr]])
           for gr in range(3)]
    parity = all(np.array_equal((got[gr][0] ^ got[gr][1] ^ got[gr][2]).astype(np.uint64),
                                plain_and([q for q in preds if q["group"] == gr], vals))
                 for gr in range(3))
    step_s = float(np.mean(ms)) / 1e3
    units = len(preds) * n_v
    row_bytes = 3 * ((1 << n) // 32) * 4                   # the three share rows of one element
    columns = len({(p["table"], p["attr"]) for p in preds})
    # every share row of each column the query reads, once, plus the packed outputs
    algo_bytes = columns * n_v * row_bytes + 3 * 3 * words_out * 4
    peak_bw = float(measured_peaks().get("hbm_gbs", 6800.0))
    rec = {"metric": METRIC, "unit": UNIT, "value": units / step_s, "ms_per_step": step_s * 1e3, "steps": steps,
           "warmup": warmup, "gpu_launches": launches,
           "config": {"l2": "flushed between timed steps", "workload": "onehot_107614v_n16_4pred", "elements": n_v,
                      "one_hot_bits": 1 << n, "groups": "EQ | RANGE | EQ AND RANGE",
                      "element_predicates_per_step": units, "share_row_bytes_per_element": row_bytes,
                      "columns_read": columns, "reconstructs_to_plaintext": parity},
           "roofline": {"bound": "hbm", "achieved": algo_bytes / step_s / 1e9, "peak": peak_bw,
                        "unit": "GB/s", "frac": algo_bytes / step_s / 1e9 / peak_bw,
                        "what": "whole step (EvalAll + dot-product + fold launches) against the share "
                                "rows of each column read (once for all predicates on it) and the packed "
                                "outputs"},
           "clocks": clocks}
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        m = 4096
        sub = W.onehot_table(vals[:, :m], n, W.rng(16))["shares"]
        # group 0 (one equality predicate): its EvalAll over the 2^16 positions, then m vertices
        rec["cpu_baseline"] = oracle_leg(
            lambda k: [oracle.filter_onehot(toks, 1, PRF, [(sub, n)], 0, np.arange(m)) for _ in range(k)],
            m, UNIT, 1, f"oracle one-hot secEval of group 0 (1 predicate) on {m} vertices", target_s=4.0)
    del outs, flush
    if own:
        ctx.close()
    return rec


WORKLOAD_RECORDS = {"tiny": record_tiny, "edges": record_edges, "batch": record_batch, "serve": record_serve,
                    "onehot": record_onehot}


def workload_line(args) -> dict:
    """The other configurations, one JSON line each (not the headline line):
    tiny   -- 1,000-vertex / 4,000-edge path query, n = 16 (parity-sized);
    edges  -- 1,000,000 vertices / 10,000,000 edges, triangle + pendant, 6 predicates;
    batch  -- 256 queries (2-8 vertices, 1-6 predicates) on that graph in one persistent
              launch replayed from a CUDA graph, against the plain path on the first 8;
    serve  -- 4,000,000 vertices / 40,000,000 edges resident, Poisson arrivals at 50, 200 and
              1000 queries/s plus one rate at half the measured capacity."""
    import torch
    import paper_2209_03526_gb300 as P
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = P.Context(0, prf_keys=PRF)
    if args.workload in ("fresh", "keygen", "fetch", "onehot", "shuffle", "aes-layouts", "wp-sweep"):
        sched = ()                       # these modes do not launch k_filter
    else:
        sched = tuple(int(v) for v in args.schedule.split(",")) if args.schedule else ctx.autotune()
        if args.schedule:
            ctx.set_schedule(*sched)
    peaks = measured_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_lu = sm_count * LDS_LANES_PER_CLK * float(peaks.get("sm_max_mhz", 2070.0)) / 1e3
    peak_aes = peak_lu / LOOKUPS_PER_AES
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "u32",
            "data": "synthetic", "workload_mode": args.workload, "schedule": list(sched)}

    if args.workload == "fetch":
        # secFetch case I after a filter: 1,048,576 vertices, 4 uint32 attributes, the filter
        # matching one vertex; the fetch of its index and 4 attributes is timed alone
        n_v = N_VERTICES
        g = W.rng(8)
        vals = W.uniform_attrs(g, 4, n_v, 32)
        tab = W.table(vals, 32, g)
        ctx.load_shares(0, [torch.from_numpy(x.view(np.int32)).to(dev) for x in tab["shares"]], 32)
        target = int(g.integers(0, n_v))
        preds = [W.eq_pred(0, 0, 0, int(vals[0, target]))]
        toks = P.keygen(preds, 32, KEY_SEED)
        outs = [[torch.empty(n_v, dtype=torch.int32, device=dev) for _ in range(3)]]
        ctx.filter_and_combine(1, toks, outs, stream)
        res = torch.empty(3 * 5, dtype=torch.int32, device=dev)
        for _ in range(max(1, args.warmup)):
            ctx.fetch_unique(1, 0, 0, outs[0], [0, 1, 2, 3], res, stream)
        ctx.sync(stream)
        flush = L2Flush(torch, dev, stream)
        call_ms = []                               # the call as a host program makes it
        for k in range(args.steps):
            flush()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.fetch_unique(1, 0, 0, outs[0], [0, 1, 2, 3], res, stream)
            b.record(stream)
            b.synchronize()
            call_ms.append(a.elapsed_time(b))
        # the device's time: the call (output clear + k_fetch) captured once in a CUDA graph
        g_fetch = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_fetch):
            ctx.fetch_unique(1, 0, 0, outs[0], [0, 1, 2, 3], res, torch.cuda.current_stream())
        torch.cuda.synchronize()
        flush_cur = L2Flush(torch, dev)
        evs = []
        for k in range(args.steps):
            # queued without waiting: the flush keeps the GPU busy while the replay is submitted
            flush_cur()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            g_fetch.replay()
            b.record()
            evs.append((a, b))
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in evs]
        rec = (res.cpu().numpy().view(np.uint32).reshape(3, 5).astype(np.uint64).sum(axis=0)) & 0xFFFFFFFF
        ok = int(rec[0]) == target and [int(v) for v in rec[1:]] == [int(vals[a, target]) for a in range(4)]
        step_s = float(np.mean(ms)) / 1e3
        algo_bytes = 12 * n_v * (1 + 4)       # the three result share sets + 4 attributes' share sets
        peak_bw = float(peaks.get("hbm_gbs", 6800.0))
        line.update({"value": n_v / step_s, "unit": "candidates/s", "metric": "secFetch case I candidates/s",
                     "ms_per_step": step_s * 1e3, "steps": args.steps, "warmup": args.warmup,
                     "config": {"workload": "fetch_unique_1048576v_4attr", "attributes_fetched": 4,
                                "reconstructs_to_the_match": ok, "l2": "flushed between timed steps",
                                "launch": "k_fetch_clear + k_fetch (its programmatic dependent), replayed from a "
                                          "CUDA graph, replays queued behind the L2 flush",
                                "direct_call_ms": float(np.mean(call_ms))},
                     "roofline": {"bound": "hbm", "achieved": algo_bytes / step_s / 1e9, "peak": peak_bw,
                                  "unit": "GB/s", "frac": algo_bytes / step_s / 1e9 / peak_bw}})
        if not args.no_cpu_baseline:
            import oracle
            xs = [o.cpu().numpy().view(np.uint32) for o in outs[0]]
            line["cpu_baseline"] = oracle_leg(
                lambda k: [oracle.fetch_unique(xs, [(tab["shares"], 32)], 0, [0, 1, 2, 3], 1, 0, PRF)
                           for _ in range(k)], n_v, "candidates/s", 1,
                f"oracle secFetch case I over all {n_v} candidates, 4 attributes (numpy)")
        ctx.close()
        return line

    if args.workload == "fresh":
        # the headline workload (1,048,576 vertices, 4 equality + 4 range predicates, n = 32)
        # with a fresh mask and key triple per element and predicate: the client's GPU keygen
        # and the servers' filter on the device-resident tokens, each timed alone
        n_v = args.elems or N_VERTICES
        wl = W.bulk_vertex_filter(n_vertices=n_v, seed=2)
        preds = wl["preds"]
        ctx.load_shares(0, [torch.from_numpy(x.view(np.int32)).to(dev) for x in wl["tables"][0]["shares"]], 32)
        L = P.fresh_token_size(preds, 32, [n_v])
        toks = [torch.empty(L, dtype=torch.uint8, device=dev) for _ in range(3)]
        outs = [[torch.empty(n_v, dtype=torch.int32, device=dev) for _ in range(3)]]

        flush = L2Flush(torch, dev, stream)

        def timed(fn, reps):
            ms = []
            for k in range(reps):
                flush()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn(k)
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            return float(np.mean(ms)) / 1e3

        for _ in range(max(1, args.warmup)):
            ctx.keygen_fresh(preds, 32, [n_v], KEY_SEED, toks, stream)
        gen_s = timed(lambda k: ctx.keygen_fresh(preds, 32, [n_v], KEY_SEED, toks, stream), args.steps)
        for _ in range(max(1, args.warmup)):
            ctx.filter_fresh(1, toks, outs, stream)
        ctx.sync(stream)
        step_s = timed(lambda k: ctx.filter_fresh(2 + k, toks, outs, stream), args.steps)
        ctx.sync(stream)
        rec = (sum(o.cpu().numpy().view(np.uint32).astype(np.uint64) for o in outs[0]) & 0xFFFFFFFF)
        ok = bool(np.array_equal(rec, plain_and(preds, wl["tables"][0]["values"])))
        units = len(preds) * n_v
        lookups = lookups_per_element(preds) * n_v
        key_bytes = 3 * L                              # every token byte is read once per step
        pairs = n_v * sum(3 if p["kind"] == W.PRED_EQ else 6 for p in preds)
        peak_bw = float(peaks.get("hbm_gbs", 6800.0))
        line.update({"value": units / step_s, "ms_per_step": step_s * 1e3, "steps": args.steps,
                     "warmup": args.warmup,
                     "config": {"l2": "flushed between timed steps", "workload": f"fresh_keys_bulk_vertex_filter_{n_v}v_4attr_8pred_n32",
                                "token_bytes_per_server": L, "element_predicates_per_step": units,
                                "reconstructs_to_plaintext": ok,
                                "launch": "one k_filter_fresh launch (servers); one k_keygen_fresh launch (client)"},
                     "roofline": {"bound": "lds", "pipe": LDS_PIPE, "achieved": lookups / step_s / 1e9, "peak": peak_lu,
                                  "unit": "Glookup/s", "frac": lookups / step_s / 1e9 / peak_lu,
                                  "token_GB_per_s": key_bytes / step_s / 1e9,
                                  "token_frac_of_hbm": key_bytes / step_s / 1e9 / peak_bw},
                     "client_keygen": {"ms": gen_s * 1e3, "key_pairs_per_s": pairs / gen_s,
                                       "token_GB_per_s": key_bytes / gen_s / 1e9}})
        if not args.no_cpu_baseline:
            import oracle
            oracle.build()
            cores = os.cpu_count() or 1
            m = 4 * cores                     # a slice of the table: its first m vertices
            sub = [s_[:, :m].copy() for s_ in wl["tables"][0]["shares"]]
            otoks = oracle.keygen_fresh(preds, 32, [m], KEY_SEED)
            line["cpu_baseline"] = oracle_leg(
                lambda k: [oracle.filter_fresh(otoks, 1, PRF, [(sub, 32)], 0, np.arange(m), threads=cores)
                           for _ in range(k)],
                m * len(preds), UNIT, cores,
                f"servers' filter on the oracle's fresh tokens for {m} vertices of the table, all 8 predicates")
        ctx.close()
        return line

    if args.workload == "shuffle":
        # secShuffle of 1,048,576 records of 6 words (x, id and 4 attributes: the records of
        # secFetch case II on the bulk table) over additive shares, then secFetch case II on
        # that table after a filter matching about 1 % of the vertices
        n_v, width = N_VERTICES, 6
        g = W.rng(13)
        ins = [torch.from_numpy(g.integers(0, 1 << 32, (n_v, width), dtype=np.uint64).astype(np.uint32)
                                .view(np.int32)).to(dev) for _ in range(3)]
        outs = [torch.empty_like(ins[0]) for _ in range(3)]
        seeds = bytes(range(48))
        for _ in range(max(1, args.warmup)):
            ctx.shuffle(ins, seeds, outs, 0, stream)
        ctx.sync(stream)
        flush = L2Flush(torch, dev, stream)
        ms = []
        for k in range(args.steps):
            flush()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.shuffle(ins, seeds, outs, 0, stream)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        shuf_s = float(np.mean(ms)) / 1e3
        q = (width + 3) // 4
        # per row 8 q mask blocks of full AES (T12, T31 by CS1; T12, T23, R2 by CS2; T31, T23,
        # R1 by CS3); plus each permutation's round table, 4 x 2^h output-word-0 AES (h = 10)
        half = max(1, ((n_v - 1).bit_length() + 1) // 2)
        lookups = n_v * 8 * q * LOOKUPS_PER_AES + 12 * (1 << half) * LOOKUPS_PER_AES_W0
        # fetch case II after a filter on the bulk table
        wl = W.bulk_vertex_filter(n_vertices=n_v, seed=2)
        vals = wl["tables"][0]["values"]
        ctx.load_shares(0, [torch.from_numpy(x.view(np.int32)).to(dev) for x in wl["tables"][0]["shares"]], 32)
        thr = int(np.quantile(vals[1], 0.01))
        toks = P.keygen([W.range_pred(0, 1, 0, 0, thr)], 32, KEY_SEED)
        x = [torch.empty(n_v, dtype=torch.int32, device=dev) for _ in range(3)]
        ctx.filter_and_combine(1, toks, [x], stream)
        fouts = [torch.empty((n_v, 5), dtype=torch.int32, device=dev) for _ in range(3)]
        ctx.fetch_multi(0, x, [0, 1, 2, 3], seeds, fouts, stream)
        fms = []
        for k in range(args.steps):
            t0 = time.perf_counter()
            m = ctx.fetch_multi(0, x, [0, 1, 2, 3], seeds, fouts, stream)
            fms.append(time.perf_counter() - t0)
        rec = sum(f[:m, 0].cpu().numpy().view(np.uint32).astype(np.uint64) for f in fouts) & 0xFFFFFFFF
        ok = sorted(rec.tolist()) == np.flatnonzero(vals[1] <= thr).tolist()
        line.update({"metric": "secShuffle records/s", "unit": "records/s", "value": n_v / shuf_s,
                     "ms_per_step": shuf_s * 1e3, "steps": args.steps, "warmup": args.warmup,
                     "config": {"l2": "flushed between timed steps", "workload": "shuffle_1048576x6_add", "records": n_v, "words_per_record": width,
                                "launch": "k_feistel_tab + k_perms + one kernel per server (k_shuf_cs1..3)"},
                     "roofline": {"bound": "lds", "pipe": LDS_PIPE, "achieved": lookups / shuf_s / 1e9, "peak": peak_lu,
                                  "unit": "Glookup/s", "frac": lookups / shuf_s / 1e9 / peak_lu},
                     "fetch_case_ii": {"candidates": n_v, "matches": int(m), "ms_host_clock": float(np.mean(fms)) * 1e3,
                                       "candidates_per_s": n_v / float(np.mean(fms)),
                                       "returns_the_matches": bool(ok)}})
        if not args.no_cpu_baseline:
            import oracle
            oracle.build()
            m = 1 << 13
            gs = W.rng(15)
            osh = [gs.integers(0, 1 << 32, (m, width), dtype=np.uint64).astype(np.uint32) for _ in range(3)]
            line["cpu_baseline"] = oracle_leg(lambda k: [oracle.shuffle(osh, seeds, 0) for _ in range(k)], m,
                                              "records/s", 1, f"oracle secShuffle of {m} records x {width} words")
        ctx.close()
        return line

    if args.workload == "keygen":
        # batched Gen on the device: 1,048,576 DPF pairs and 1,048,576 DCF pairs with n = 32
        # (one fresh pair per element of a 2^20-vertex column, the masked approach's per-value
        # keys), each timed alone; plus the host genToken time and size of Table 1's queries
        m, n = N_VERTICES, 32
        g = W.rng(12)
        alpha = torch.from_numpy(g.integers(0, 1 << 32, m, dtype=np.uint64).astype(np.uint32).view(np.int32)).to(dev)
        beta = torch.from_numpy(g.integers(0, 1 << 32, m, dtype=np.uint64).astype(np.uint32).view(np.int32)).to(dev)
        kinds = {}
        total_s = total_lu = total_pairs = 0.0
        for name, kind in (("dpf", P.KEY_DPF), ("dcf", P.KEY_DCF)):
            L = 28 + n * (20 if kind == P.KEY_DPF else 24)
            out = torch.empty(2 * m * L, dtype=torch.uint8, device=dev)
            for _ in range(max(1, args.warmup)):
                ctx.keygen_device(kind, n, alpha, beta, KEY_SEED, out, stream)
            flush = L2Flush(torch, dev, stream)
            ms = []
            for k in range(args.steps):
                flush()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctx.keygen_device(kind, n, alpha, beta, KEY_SEED, out, stream)
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            ctx.sync(stream)
            s_ = float(np.mean(ms)) / 1e3
            full, w0 = keygen_blocks_per_pair(kind == P.KEY_DCF, n)
            lu = m * (full * LOOKUPS_PER_AES + w0 * LOOKUPS_PER_AES_W0)
            kinds[name] = {"pairs_per_s": m / s_, "ms": s_ * 1e3, "key_bytes": L,
                           "key_GB_per_s": 2 * m * L / s_ / 1e9, "glookup_per_s": lu / s_ / 1e9}
            total_s += s_
            total_lu += lu
            total_pairs += m
            del out
        table1 = {}
        for sym, mk in (("=", lambda v, i: W.eq_pred(0, 0, i, v)),
                        ("<<", lambda v, i: W.range_pred(0, 0, i, v, v + 1000))):
            for q in (2, 4, 8):
                preds = [mk(1000 * (i + 1), i) for i in range(q)]
                reps, t0 = 20, time.perf_counter()
                for _ in range(reps):
                    tk = P.keygen(preds, 32, KEY_SEED)
                dt = (time.perf_counter() - t0) / reps
                table1[f"{sym} |q|={q}"] = {"host_ms": dt * 1e3, "token_MB": sum(len(t) for t in tk) / 1e6}
        line.update({"metric": "FSS key pairs generated/s (n = 32)", "unit": "key-pairs/s",
                     "value": total_pairs / total_s, "ms_per_step": total_s * 1e3, "steps": args.steps,
                     "warmup": args.warmup,
                     "config": {"l2": "flushed between timed steps", "workload": "keygen_1048576_dpf_1048576_dcf_n32", "pairs_per_kind": m,
                                "launch": "one k_keygen launch per kind"},
                     "kinds": kinds,
                     "roofline": {"bound": "lds", "pipe": LDS_PIPE, "achieved": total_lu / total_s / 1e9, "peak": peak_lu,
                                  "unit": "Glookup/s", "frac": total_lu / total_s / 1e9 / peak_lu},
                     "table1_host_gentoken": table1})
        if not args.no_cpu_baseline:
            import oracle
            oracle.build()
            ga = W.rng(14)
            al = [int(v) for v in ga.integers(0, 1 << 32, 64, dtype=np.uint64)]

            def gen_pairs(k):
                for r in range(k):
                    for i, a in enumerate(al):
                        oracle.dpf_gen(32, a, a ^ 0x5A5A, KEY_SEED, SEED_B)
                        oracle.dcf_gen(32, a, a ^ 0x5A5A, KEY_SEED, SEED_B)

            line["cpu_baseline"] = oracle_leg(gen_pairs, 2 * len(al), "key-pairs/s", 1,
                                              "oracle DPF and DCF Gen at n = 32, 64 pairs of each, one thread")
        ctx.close()
        return line

    if args.workload == "onehot":
        line.update(record_onehot(P, torch, args, sched, ctx=ctx, steps=args.steps, warmup=args.warmup))
        ctx.close()
        return line

    if args.workload == "aes-layouts":
        # the autotuner's AES-layout dimension: the PRG on 2^26 counter blocks in both layouts
        runs = [ctx.autotune_aes_layout() for _ in range(max(1, args.steps))]
        mhz = float(peaks.get("sm_max_mhz", 2070.0))
        tt = statistics.median(r[1] for r in runs)
        bs = statistics.median(r[2] for r in runs)
        line.update({"metric": "fixed-key PRG blocks/s by AES layout", "unit": "blocks/s", "value": max(tt, bs),
                     "steps": len(runs), "warmup": 1,
                     "config": {"workload": "prg_2pow26_counter_blocks_K_L", "blocks_per_timing": 1 << 26,
                                "chosen_layout": "bitsliced" if runs[-1][0] == P.AES_BITSLICED else "T-table"},
                     "ttable": {"blocks_per_s": tt, "blocks_per_clk_per_sm": tt / (sm_count * mhz * 1e6)},
                     "bitsliced": {"blocks_per_s": bs, "blocks_per_clk_per_sm": bs / (sm_count * mhz * 1e6)},
                     "roofline": {"bound": "lds", "achieved": tt * LOOKUPS_PER_AES / 1e9, "peak": peak_lu,
                                  "unit": "Glookup/s", "frac": tt * LOOKUPS_PER_AES / 1e9 / peak_lu,
                                  "what": "the T-table layout against the shared-memory lookup ceiling"}})
        ctx.close()
        return line

    if args.workload == "wp-sweep":
        # the walk-parallel kernel's item time by tile width: one predicate of each kind at n = 16
        # and 32 on a table of 152 x w (one item per SM) or 304 x w (two) elements, tile forced
        ctx.set_walk_parallel((1 << 64) - 1)
        rows = []
        for n in (16, 32):
            for kind in ("eq", "range"):
                for waves in (1, 2):
                    for w in (1, 4, 8, 12, 16, 20, 24, 28, 32, 36, 40):
                        N = sm_count * w * waves
                        g = W.rng(w)
                        tab = W.table(W.uniform_attrs(g, 1, N, n), n, g)
                        ctx.load_shares(0, [torch.from_numpy(x.view(np.int32)).to(dev) for x in tab["shares"]], n)
                        pred = W.eq_pred(0, 0, 0, 5) if kind == "eq" else W.range_pred(0, 0, 0, 7, ((1 << n) - 1) // 2)
                        toks = P.keygen([pred], n, KEY_SEED)
                        outs = [[torch.empty(N, dtype=torch.int32, device=dev) for _ in range(3)]]
                        ctx.set_walk_parallel_tile(w)
                        plan = ctx.plan_create([1], [toks], [outs])
                        ms = _timed_graph(torch, ctx, plan, stream, 3, max(5, args.steps))
                        ctx.plan_destroy(plan)
                        rows.append({"n": n, "kind": kind, "items_per_sm": waves, "tile": w,
                                     "us": float(np.median(ms)) * 1e3})
        wl = W.tiny_path(seed=1)
        for tid, t in enumerate(wl["tables"]):
            ctx.load_shares(tid, [torch.from_numpy(x.view(np.int32)).to(dev) for x in t["shares"]], 16)
        toks = P.keygen(wl["preds"], 16, KEY_SEED)
        outs = [[torch.empty(t["values"].shape[1], dtype=torch.int32, device=dev) for _ in range(3)]
                for t in wl["tables"]]
        tiny = []
        for w in [0] + list(range(20, 41, 2)):
            ctx.set_walk_parallel_tile(w)
            plan = ctx.plan_create([1], [toks], [outs])
            shape = ctx.plan_describe(plan)
            ms = _timed_graph(torch, ctx, plan, stream, 3, max(50, args.steps))
            ctx.plan_destroy(plan)
            tiny.append({"forced_tile": w, "tile": shape["tile"], "items": shape["items"],
                         "us": float(np.median(ms)) * 1e3})
        line.update({"metric": "walk-parallel item time", "unit": "us", "higher_is_better": False,
                     "config": {"workload": "walk_parallel_tile_sweep"}, "sweep": rows, "tiny_path_by_tile": tiny})
        ctx.close()
        return line

    if args.workload in WORKLOAD_RECORDS:
        ctx.close()
        args.sub_steps = args.sub_steps or args.steps
        line.update(WORKLOAD_RECORDS[args.workload](P, torch, args, sched))
        return line
    ctx.close()
    raise ValueError(f"unknown workload {args.workload}")


def run_workload(args):
    print(json.dumps(workload_line(args)), flush=True)
    return 0


def mode_record(mode: str, steps: int):
    """A default-line record of one of the single-operation modes (fetch, shuffle, keygen): the
    mode's own measurement, its clocks sampled over the whole record (setup included)."""
    def rec(P, torch, args, sched) -> dict:
        a = argparse.Namespace(**vars(args))
        a.workload, a.steps, a.warmup, a.schedule = mode, args.sub_steps or steps, 3, ""
        sampler = ClockSampler(gpu_index_of(0))
        sampler.start()
        line = workload_line(a)
        line["clocks"] = dict(sampler.stop(), over="the whole record, setup included")
        for k in ("n_gpus", "higher_is_better", "dtype", "data", "workload_mode", "schedule"):
            line.pop(k, None)
        return line
    return rec


WORKLOAD_RECORDS.update({"fetch": mode_record("fetch", 200), "shuffle": mode_record("shuffle", 20),
                         "keygen": mode_record("keygen", 5), "fresh": mode_record("fresh", 3)})


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-compare", action="store_true",
                    help="the headline step only: skip the plain-path and latency comparisons and the other "
                         "workloads' records")
    ap.add_argument("--workloads", default="tiny,edges,batch,serve,onehot,fetch,shuffle,keygen,fresh",
                    help="records of the other workloads in the default line (comma list of tiny, edges, batch, "
                         "serve, onehot, fetch, shuffle, keygen, fresh; empty for none)")
    ap.add_argument("--sub-steps", type=int, default=0, help="timed replays per workload record (0: its default)")
    ap.add_argument("--latency-queries", type=int, default=200, help="Poisson arrivals of the headline latency leg")
    ap.add_argument("--latency-plain", type=int, default=100,
                    help="arrivals of the latency leg that the plain path also serves (a prefix)")
    ap.add_argument("--serve-queries", type=int, default=96,
                    help="arrivals of the serving record's rate at half its capacity")
    ap.add_argument("--serve-overload-queries", type=int, default=32,
                    help="arrivals of each of the serving record's overloaded rates (50, 200, 1000 q/s)")
    ap.add_argument("--plain-queries", type=int, default=6,
                    help="plain-path arrivals per rate of the serving record (a prefix)")
    ap.add_argument("--workload", choices=["bulk", "tiny", "edges", "batch", "serve", "onehot", "fetch", "keygen", "fresh",
                                           "shuffle", "aes-layouts", "wp-sweep"],
                    default="bulk",
                    help="bulk (default, the headline line); the others print their own line")
    ap.add_argument("--elems", type=int, default=0, help="--workload fresh: vertices (default 1,048,576)")
    ap.add_argument("--schedule", default="", help="threads,elems_per_thread (skips the autotuner)")
    ap.add_argument("--profile-case", action="store_true",
                    help="one small fused launch for ncu: 4,194,304 elements, 1 attribute, 1 equality + 1 range "
                         "predicate, after one warm-up launch")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "bulk":
        return run_workload(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
