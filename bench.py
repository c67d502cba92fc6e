#!/usr/bin/env python
"""Benchmark of the FM-index search path on GB300 (one JSON line on rank 0).

Main line (the step): one batched inexact search (D lower bound, persistent search kernel,
canonical interval sets) of 10,000,000 reads of 50-250 bp (1% substitutions, 0.05% single-base
indels, drawn from both strands) against a 2,000,000,000-base repeat-structured reference,
z = 2 differences with at most 1 gap, each read searched on both strands.  Metric: reads/s.
Beside it, in the same line:
  * the plain per-read kernel on the same batch (bit-exact comparison of the two);
  * best_hits: the same batch with per-interval minimum costs, keeping each query's best;
  * end_restricted: the same batch with indel columns kept 5 read symbols from either end;
  * e2e: the same batch end to end through the C ABI with host buffers (fm_server_submit /
    fm_server_poll: reads copied from host memory, interval sets read back to host memory),
    and beside it the device-pointer call with torch copies of the reads in and the interval
    sets out;
  * serving: mixed-mode requests on the resident index, offline and under Poisson arrivals;
  * locate: SA positions of 2^24 random rows (Eq. 4-5);
  * occ8: the Occ micro-benchmark, 2^28 eight-Occ queries on a 2 Gbp i.i.d. 41% GC index
    (half in one checkpoint block, half at a geometric gap of mean 1000), against the
    random-gather roofline;
  * exact: plain exact search of 10,000 32 bp reads on a 1 Mbp uniform reference;
  * both_strands_256mbp: two queries per read on R against one on R . revcomp(R);
  * inexact_64mbp: 10^6 100 bp reads, z = 2 mismatches, on a 64 Mbp repeat reference;
  * cpu_baseline: the CPU oracle on a bounded sample of the main workload.
With --impl reference the CPU oracle itself is timed on a bounded sample per step.
Launch: python bench.py [--gpus N --steps K --warmup W]; under torchrun one replica per GPU,
each with its own read batch (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("reads/s at z<=2 (batched vs plain kernel, bit-exact); 8-Occ Gq/s vs gather "
          "roofline")
SEED_EXACT, SEED_OCC, SEED_SEARCH = 1811061271, 1811061272, 1811061274
# bytes of one checkpoint block per interval (fm_info reports the same)
BLOCK_BYTES = {32: 32, 64: 32, 128: 64, 256: 96}
# DRAM bytes (read + write) per launch of the current search kernel from one ncu capture,
# keyed by (interval, reference bp, reads, canonical enumeration on, interval-table depth, pair
# steps on) and reported only when the run matches that configuration.  An entry is removed
# when the kernel changes and added back from a fresh capture.
TRAFFIC_NCU = {(64, 2_000_000_000, 10_000_000, True, 14, True): 2.663352970752e12 + 5.28495616e8,
               (32, 2_000_000_000, 10_000_000, True, 14, True): 2.687482436864e12 + 5.27048960e8}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--ref-n", type=int, default=2_000_000_000)
    ap.add_argument("--reads", type=int, default=10_000_000)
    ap.add_argument("--occ-n", type=int, default=2_000_000_000)
    ap.add_argument("--occ-queries", type=int, default=1 << 28)
    ap.add_argument("--interval", type=int, default=64)
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--skip-occ8", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-best", action="store_true")
    ap.add_argument("--skip-both", action="store_true")
    ap.add_argument("--skip-end", action="store_true")
    ap.add_argument("--end-skip", type=int, default=5,
                    help="end restriction of the end_restricted line: indel columns only with at "
                         "least this many read symbols on each side")
    ap.add_argument("--skip-cfg3", action="store_true")
    ap.add_argument("--skip-serving", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=4.0)
    ap.add_argument("--autotune", type=int, default=1, help="1: tune interval/occupancy/chunk")
    ap.add_argument("--canonical", type=int, default=1, choices=[1, 2],
                    help="1: enumerate canonical alignments (same interval sets, fewer nodes); "
                         "2: every call of Listing 2")
    ap.add_argument("--pair-steps", type=int, default=None, choices=[1, 2],
                    help="1: exact continuations two symbols per step (pair table); 2: one "
                         "(default: the autotuner's choice, else 1)")
    ap.add_argument("--kmer-depth", type=int, default=None,
                    help="interval tables of short strings: 1..14 levels, 254 automatic "
                         "(floor(log4(n+1)) - 2), 255 none (default: the autotuner's choice, "
                         "else automatic)")
    ap.add_argument("--refill", type=int, default=0,
                    help="persistent kernel: take queries below this pool level (0: library)")
    ap.add_argument("--chain2-min", type=int, default=0,
                    help="persistent kernel: step second exact chains when this many lanes hold "
                         "one (0: library default)")
    ap.add_argument("--tune-reads", type=int, default=1_000_000)
    ap.add_argument("--tune-cache", default=None, help="JSON cache of tuning results")
    ap.add_argument("--cpu-sample-reads", type=int, default=200_000)
    ap.add_argument("--cpu-sample-ref", type=int, default=32_000_000)
    ap.add_argument("--log", default=None, help="also append the JSON line to this file")
    ap.add_argument("--gather-sweep", action="store_true",
                    help="only print the random-gather ceiling for 32/64/128-byte granules "
                         "over 128 MB..8 GB buffers (one JSON line per point)")
    return ap.parse_args()


# ---------------------------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------------------------

def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup(args):
    from paper_1811_06127_gb300 import replicas
    return replicas.env_rank()


# ---------------------------------------------------------------------------------------------
# reference arm / CPU baseline: the oracle as it stands
# ---------------------------------------------------------------------------------------------

def oracle_sample(args, nreads, seed_off=0):
    import oracle
    from paper_1811_06127_gb300 import synth
    R = synth.repeat_text(SEED_SEARCH, args.cpu_sample_ref)
    ix = oracle.Index(R, "sais")
    reads = synth.sample_reads(SEED_SEARCH + 7 + seed_off, R, nreads, 50, 250, sub_rate=0.01,
                               indel_rate=0.0005, both_strands=True)
    return ix, reads


def cpu_baseline(args):
    import oracle
    ix, reads = oracle_sample(args, args.cpu_sample_reads)
    thr = oracle.default_threads()
    t0 = time.perf_counter()
    res = ix.inexact(reads.codes, reads.offs, 2, 1, strands=2, threads=thr)
    dt = time.perf_counter() - t0
    return {"value": len(reads) / dt, "unit": "reads/s", "cores": thr, "kind": "oracle",
            "sample": (f"{len(reads)} reads of the same read model (50-250 bp, 1% subst, 0.05% "
                       f"indel, both strands, z=2, 1 gap) against a {args.cpu_sample_ref} bp "
                       "reference from the same repeat generator; the oracle's own index of the "
                       "2 Gbp reference is not built (its SA-IS takes over ten minutes); index "
                       "build not timed"),
            "seconds": dt, "nodes_per_read": float(res["nodes"].sum()) / len(reads)}


def cpu_configs(args):
    """The oracle timed on bounded samples of the other configurations, on one host thread and
    on all of them (index builds not timed): exact search and fm_occ8-style queries of
    config 1, the occ8 query mix of config 2 on a 32 Mbp reference of the same generator (the
    oracle's index of 2 Gbp takes over ten minutes), config 3's read model, and a one-thread
    sample of the main read model."""
    import oracle
    from paper_1811_06127_gb300 import synth
    thr = oracle.default_threads()
    out = {"cores": thr}

    def timed(fn, n, unit, sample):
        res = {"sample": sample, "unit": unit}
        for name, t in (("one_thread", 1), ("all_cores", thr)):
            t0 = time.perf_counter()
            fn(t, n[name])
            res[name] = n[name] / (time.perf_counter() - t0)
        return res

    R1 = synth.uniform_text(SEED_EXACT, 1_000_000)
    ix1 = oracle.Index(R1, "sais")
    rd1 = synth.exact_reads(SEED_EXACT, R1, 10_000, 32)
    k1, l1 = synth.occ_queries_uniform(SEED_EXACT, R1.size, 1_000_000)
    out["cfg1_exact"] = timed(lambda t, n: ix1.exact(rd1.codes, rd1.offs, threads=t),
                              {"one_thread": 10_000, "all_cores": 10_000}, "reads/s",
                              "config 1 in full: 10,000 reads of 32 bp on 1 Mbp")
    out["cfg1_occ8"] = timed(lambda t, n: ix1.occ8(k1[:n], l1[:n], threads=t),
                             {"one_thread": 1_000_000, "all_cores": 1_000_000}, "8-Occ/s",
                             "config 1 in full: 10^6 queries on 1 Mbp")
    R2 = synth.gc_text(SEED_OCC, 32_000_000, 0.41)
    ix2 = oracle.Index(R2, "sais")
    k2, l2 = synth.occ_queries_mixed(SEED_OCC, R2.size, 1 << 22, 64)
    out["cfg2_occ8"] = timed(lambda t, n: ix2.occ8(k2[:n], l2[:n], threads=t),
                             {"one_thread": 1 << 20, "all_cores": 1 << 22}, "8-Occ/s",
                             "config 2's query mix on a 32 Mbp 41% GC reference: 2^20 queries "
                             "(1 thread), 2^22 (all cores)")
    del ix2, R2
    R3 = synth.repeat_text(1811061273, 64_000_000)
    ix3 = oracle.Index(R3, "sais")
    rd3 = synth.sample_reads(1811061273, R3, 40_000, 100, 100, sub_rate=0.005,
                             both_strands=True, random_frac=0.05)

    def cfg3(t, n):
        sub = rd3.subset(np.arange(n))
        ix3.inexact(sub.codes, sub.offs, 2, 0, strands=2, threads=t)
    out["cfg3_inexact"] = timed(cfg3, {"one_thread": 2_000, "all_cores": 40_000}, "reads/s",
                                "config 3 in full size (64 Mbp), 2,000 reads (1 thread) and "
                                "40,000 (all cores) of its 10^6")
    del ix3, R3
    ix4, rd4 = oracle_sample(args, 4_000, seed_off=1)
    t0 = time.perf_counter()
    ix4.inexact(rd4.codes, rd4.offs, 2, 1, strands=2, threads=1)
    out["cfg4_inexact_one_thread"] = {"value": len(rd4) / (time.perf_counter() - t0),
                                      "unit": "reads/s",
                                      "sample": f"4,000 reads of the main read model on the "
                                                f"{args.cpu_sample_ref} bp sample reference"}
    return out


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    import oracle
    n_step = max(2000, args.cpu_sample_reads // 10)
    ix, reads = oracle_sample(args, n_step * (args.warmup + args.steps))
    thr = oracle.default_threads()
    times = []
    for s in range(args.warmup + args.steps):
        sub = reads.subset(np.arange(s * n_step, (s + 1) * n_step))
        t0 = time.perf_counter()
        ix.inexact(sub.codes, sub.offs, 2, 1, strands=2, threads=thr)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = n_step * args.steps / total
    line = {"metric": METRIC, "value": value, "unit": "reads/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8/u32 (integer)",
            "data": "synthetic",
            "config": {"workload": "inexact search z=2 (1 gap), 50-250 bp reads, both strands, "
                                   f"oracle sample on a {args.cpu_sample_ref} bp reference",
                       "reads_per_step": n_step},
            "cpu_baseline": {"value": value, "unit": "reads/s", "cores": thr, "kind": "oracle",
                             "sample": f"{n_step} reads per step against a {args.cpu_sample_ref}"
                                       " bp reference from the same generator"},
            "e2e": {"value": value, "unit": "reads/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    from paper_1811_06127_gb300 import fmocc, synth

    if args.gather_sweep:
        return gather_sweep(torch, fmocc)
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    fmocc.load_library()
    dev = torch.device("cuda", local)
    hbm_peak, peak_kind = peaks()
    notes = {}

    from paper_1811_06127_gb300 import replicas

    def barrier():
        torch.cuda.synchronize()
        replicas.barrier()

    max_over_ranks = replicas.max_over_ranks

    # the flush writes at least twice the L2 size read from the device (129 MB on GB300)
    l2_bytes = int(getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 0) or 0)
    flush_bytes = max(256 << 20, 2 * l2_bytes)
    l2_flush = torch.empty(flush_bytes, dtype=torch.uint8, device=dev)

    def flush():
        l2_flush.add_(1)

    # ---- main workload: index and reads -------------------------------------------------
    t0 = time.time()
    R = synth.repeat_text(SEED_SEARCH, args.ref_n)
    notes["ref_gen_s"] = time.time() - t0
    t0 = time.time()
    reads = synth.sample_reads(replicas.shard_seed(SEED_SEARCH, rank), R, args.reads, 50, 250, sub_rate=0.01,
                               indel_rate=0.0005, both_strands=True)
    notes["reads_gen_s"] = time.time() - t0
    tuned = None
    if args.autotune:
        from paper_1811_06127_gb300 import autotune
        tuned = autotune.autotune(R, reads, 2, 1, strands=2, device=local,
                                  workload={"reads": "50-250 bp, 1% subst, 0.05% indel"},
                                  sample_reads=args.tune_reads, cache_path=args.tune_cache)
        args.interval = tuned["interval"]
    t0 = time.time()
    h = fmocc.fm_build(R, interval=args.interval, device=local)
    torch.cuda.synchronize()
    notes["build_s"] = time.time() - t0
    if tuned:
        autotune.apply(h, tuned)
    fmocc.fm_set_tuning(h, canonical=args.canonical,
                        kmer_depth=args.kmer_depth if args.kmer_depth is not None else 0,
                        pair_steps=args.pair_steps if args.pair_steps is not None else 0,
                        refill=args.refill, chain2_min=args.chain2_min)
    tun = fmocc.fm_get_tuning(h)
    kdepth = tun["kmer_depth"]
    kdepth = 0 if kdepth == fmocc.KMER_OFF else kdepth
    args.pair_steps = tun["pair_steps"]
    del R
    codes_h = torch.from_numpy(reads.codes).pin_memory()
    offs_h = torch.from_numpy(reads.offs.view(np.int32)).pin_memory()
    codes = codes_h.to(dev)
    offs = offs_h.to(dev)
    nq = 2 * args.reads
    counts = torch.empty(nq, dtype=torch.int32, device=dev)
    offsets = torch.empty(nq + 1, dtype=torch.int64, device=dev)
    stats = torch.zeros(4, dtype=torch.int64, device=dev)
    prof = fmocc.fm_profile()

    def search(kernel, pairs_buf, st=None):
        return fmocc.fm_inexact(h, codes, offs, 2, 1, strands=2, kernel=kernel, stats=st,
                                counts=counts, offsets=offsets, pairs=pairs_buf, profile=prof)

    # size the pairs buffer with one untimed call
    c0, o0, p0 = search("persistent", None)
    pairs_cap = int(p0.shape[0]) + 1024
    pairs = torch.empty((pairs_cap, 2), dtype=torch.int32, device=dev)
    ref_pairs = p0.clone()
    ref_offsets = o0.clone()

    # warm-up, then K timed steps (events per step on the launching stream, L2 flushed between)
    for _ in range(args.warmup):
        search("persistent", pairs)
    barrier()
    stats.zero_()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clk = Clocks(local)
    clk.start()
    search_ms, launches = [], 0
    for s in range(args.steps):
        flush()
        ev[s][0].record()
        _, o1, p1 = search("persistent", pairs, stats)
        ev[s][1].record()
        search_ms.append(prof.ms_search)
        launches += prof.launches
    barrier()
    clocks = clk.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = max_over_ranks(sum(step_ms) / 1000.0)
    st = stats.cpu().numpy()
    nodes_per_step = st[0] / args.steps
    blocks_per_step = st[1] / args.steps
    tables_per_step = st[3] / args.steps   # 32-byte interval-table sectors
    bbytes = BLOCK_BYTES[args.interval]
    value = args.reads * args.steps * world / total_s
    # dominant kernel: the persistent search kernel, its own event-timed duration per launch
    k_ms = float(np.mean(search_ms))
    alg_bytes = blocks_per_step * bbytes + tables_per_step * 32
    achieved = alg_bytes / (k_ms / 1000.0) / 1e9
    same = bool(torch.equal(p1, ref_pairs) and torch.equal(o1, ref_offsets))

    # step fill of the persistent kernel: one more (untimed) search with its counters on
    fprof = fmocc.fm_profile()
    fprof.fill_counters = 1
    search("persistent", pairs)
    fmocc.fm_inexact(h, codes, offs, 2, 1, strands=2, counts=counts, offsets=offsets, pairs=pairs,
                     profile=fprof)
    fd = fprof.as_dict()
    fill = {"exact_steps": fd["exact_steps"], "general_steps": fd["general_steps"],
            "lanes_per_exact_step": (fd["exact_lanes"] + fd["exact_lanes2"]) / max(fd["exact_steps"], 1),
            "first_chain_lanes_per_exact_step": fd["exact_lanes"] / max(fd["exact_steps"], 1),
            "lanes_per_general_step": fd["general_lanes"] / max(fd["general_steps"], 1),
            "queries_per_admission": fd["admitted"] / max(fd["admissions"], 1),
            "exact_steps_with_parked_second_chains": fd["parked"],
            "note": "exact steps run up to two chains per lane (64 per warp step); general "
                    "steps up to 32 nodes"}

    # ---- plain per-read kernel on the same batch ----------------------------------------
    plain = None
    if not args.skip_plain:
        search("plain", pairs)
        barrier()
        pms = []
        for _ in range(args.plain_steps):
            flush()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            _, op, pp = search("plain", pairs)
            b.record()
            torch.cuda.synchronize()
            pms.append(a.elapsed_time(b))
        same_plain = bool(torch.equal(pp, ref_pairs) and torch.equal(op, ref_offsets))
        ptot = max_over_ranks(sum(pms) / 1000.0)
        plain = {"value": args.reads * len(pms) * world / ptot, "unit": "reads/s",
                 "ms_per_step": 1000 * ptot / len(pms), "steps": len(pms),
                 "kernel_ms": prof.ms_search, "bit_exact_vs_persistent": same_plain}

    # ---- minimum-cost annotation and best hits on the same batch -------------------------
    best = None
    if not args.skip_best:
        costs_buf = torch.empty(pairs_cap, dtype=torch.uint8, device=dev)
        best_pairs = torch.empty((pairs_cap, 2), dtype=torch.int32, device=dev)

        def search_best():
            return fmocc.fm_inexact(h, codes, offs, 2, 1, strands=2, counts=counts,
                                    offsets=offsets, pairs=best_pairs, costs=costs_buf,
                                    best=True, profile=prof)
        search_best()
        barrier()
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        _, ob, pb, cb = search_best()
        b.record()
        torch.cuda.synchronize()
        bms = max_over_ranks(a.elapsed_time(b) / 1000.0)
        cvals = cb.cpu().numpy()
        best = {"value": args.reads * world / bms, "unit": "reads/s", "ms_per_step": 1000 * bms,
                "steps": 1, "what": "every query's minimum-cost intervals with their costs "
                                    "(eager path: search, grouping, per-interval minimum cost, "
                                    "best-hit compaction)",
                "best_intervals": int(ob[-1].item()),
                "all_intervals": int(ref_offsets[-1].item()),
                "cost_histogram": np.bincount(cvals, minlength=3).tolist()}

    # ---- end restriction on indel columns, same batch --------------------------------------
    endr = None
    if not args.skip_end:
        end_pairs = torch.empty((pairs_cap, 2), dtype=torch.int32, device=dev)
        est = torch.zeros(4, dtype=torch.int64, device=dev)

        def search_end(st=None):
            return fmocc.fm_inexact(h, codes, offs, 2, 1, strands=2, counts=counts,
                                    offsets=offsets, pairs=end_pairs, end_skip=args.end_skip,
                                    stats=st, profile=prof)
        search_end()
        barrier()
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        _, oe, _ = search_end(est)
        b.record()
        torch.cuda.synchronize()
        ems = max_over_ranks(a.elapsed_time(b) / 1000.0)
        endr = {"value": args.reads * world / ems, "unit": "reads/s", "ms_per_step": 1000 * ems,
                "steps": 1, "end_skip": args.end_skip, "kernel_ms": prof.ms_search,
                "what": "indel columns only where at least end_skip read symbols lie on each "
                        "side; every alignment of Listing 2 is enumerated (the canonical "
                        "rewrites move indels across that boundary)",
                "intervals": int(oe[-1].item()), "all_intervals": int(ref_offsets[-1].item()),
                "nodes": int(est[0].item()), "nodes_unrestricted": int(nodes_per_step)}
        del end_pairs

    # ---- e2e through the C ABI with host buffers ----------------------------------------
    e2e = None
    if not args.skip_e2e:
        counts_h = torch.empty(nq, dtype=torch.int32).pin_memory()
        offsets_h = torch.empty(nq + 1, dtype=torch.int64).pin_memory()
        pairs_h = torch.empty((pairs_cap, 2), dtype=torch.int32).pin_memory()
        d2h = 0
        barrier()
        t0 = time.perf_counter()
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record()
        for _ in range(args.steps):
            codes.copy_(codes_h, non_blocking=True)
            offs.copy_(offs_h, non_blocking=True)
            c2, o2, p2 = search("persistent", pairs)
            counts_h.copy_(c2, non_blocking=True)
            offsets_h.copy_(o2, non_blocking=True)
            npairs = p2.shape[0]
            pairs_h[:npairs].copy_(p2, non_blocking=True)
            d2h = counts_h.numel() * 4 + offsets_h.numel() * 8 + npairs * 8
        eb.record()
        torch.cuda.synchronize()
        e_s = max_over_ranks(ea.elapsed_time(eb) / 1000.0)
        e2e = {"value": args.reads * args.steps * world / e_s, "unit": "reads/s",
               "h2d_bytes_per_step": codes_h.numel() + offs_h.numel() * 4,
               "d2h_bytes_per_step": int(d2h), "wall_s": time.perf_counter() - t0}
    serving = None if args.skip_serving else bench_serving(args, fmocc, h, reads)
    e2e_abi = None if args.skip_e2e else bench_e2e_serving_abi(args, fmocc, h, reads, world)
    ceil_main = gather_ceiling(torch, fmocc, dev, fmocc.fm_info(h)["n_blocks"] * bbytes, flush)
    locate = bench_locate(args, torch, fmocc, h, dev, flush)
    h.close()
    del codes, offs, pairs

    # ---- Occ micro-benchmark -----------------------------------------------------------
    occ8 = None
    if not args.skip_occ8:
        occ8 = bench_occ8(args, torch, fmocc, synth, dev, hbm_peak, peak_kind, flush, barrier,
                          max_over_ranks, world)
    exact = bench_exact(args, torch, fmocc, synth, dev, flush, barrier)
    both = None if args.skip_both else bench_both_strands(args, torch, fmocc, synth, dev, flush,
                                                          barrier)
    cfg3 = None if args.skip_cfg3 else bench_cfg3(args, torch, fmocc, synth, dev, flush, barrier,
                                                   hbm_peak)

    cpu = cpu_cfg = None
    if not args.skip_cpu and rank == 0 and world == 1:
        cpu = cpu_baseline(args)
        cpu_cfg = cpu_configs(args)

    traffic_key = (args.interval, args.ref_n, args.reads, args.canonical == 1, kdepth,
                   args.pair_steps == 1)
    line = {
        "metric": METRIC, "value": value, "unit": "reads/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8/u32 (integer)",
        "data": "synthetic (seeded genome-shaped reference and reads; no dataset)",
        "config": {"workload": ("batched uneven inexact search: 2 Gbp repeat-structured reference "
                                "(41% GC, 20% copies of 500 families), 10M reads 50-250 bp, 1% "
                                "subst + 0.05% indel, z=2 with <=1 gap, both strands, persistent "
                                "kernel"),
                   "enumeration": ("canonical alignments (the interval sets of Listing 2)"
                                   if args.canonical == 1 else "every call of Listing 2"),
                   "pair_steps": args.pair_steps == 1,
                   "interval_tables": (f"strings of length <= {kdepth} expanded from tables "
                                       f"({(2 << (2 * kdepth)) * 8 / 1e6:.0f} MB)"
                                       if kdepth else "none"),
                   "reference_bp": args.ref_n, "reads_per_step": args.reads,
                   "queries_per_step": nq, "interval": args.interval,
                   "tuning": ({k: tuned.get(k) for k in ("interval", "warps_per_block",
                                                          "blocks_per_sm", "chunk", "kmer_depth",
                                                          "pair_steps", "trials", "tune_seconds",
                                                          "cached")} if tuned else None),
                   "scheduler": {k: tun[k] for k in ("warps_per_block", "blocks_per_sm", "chunk",
                                                     "refill", "chain2_min", "kmer_depth",
                                                     "pair_steps")},
                   "parallelism": f"replicas x{world} (read sharding)",
                   "l2": (f"flushed between timed steps ({flush_bytes >> 20} MB write; L2 "
                          f"{l2_bytes >> 20} MB read from the device); index 2x1 GB > L2")},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak,
                     "traffic": TRAFFIC_NCU.get(traffic_key),
                     "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                        "full-size launch of the current kernel, "
                                        "profiles/k_inexact_persistent_2gbp_10m_reads_dram.md"
                                        if traffic_key in TRAFFIC_NCU else
                                        "no capture of this configuration (interval, size, "
                                        "tables, pair steps)"),
                     "kernel": "k_inexact_persistent", "kernel_ms": k_ms,
                     # the captured DRAM bytes over this run's kernel time, and that rate over
                     # the copy peak (random reads move whole DRAM lines: traffic > algorithmic)
                     "traffic_gb_s": (TRAFFIC_NCU[traffic_key] / (k_ms / 1000) / 1e9
                                      if traffic_key in TRAFFIC_NCU else None),
                     "traffic_frac": (TRAFFIC_NCU[traffic_key] / (k_ms / 1000) / 1e9 / hbm_peak
                                      if traffic_key in TRAFFIC_NCU else None),
                     "gather_ceiling": ceil_main,
                     # every 32-byte unit the kernel gathers (checkpoint blocks and table or pair
                     # sectors) per second, over the live random 32-byte gather ceiling; above 1
                     # where shallow table sectors hit in L2
                     "gathers_per_s_over_gather_ceiling": (
                         (blocks_per_step * bbytes / 32 + tables_per_step) / (k_ms / 1000) / 1e9
                         / ceil_main["g_gathers_s"]),
                     "checkpoint_blocks_per_s_over_gather_ceiling": (
                         blocks_per_step / (k_ms / 1000) / 1e9 / ceil_main["g_gathers_s"]),
                     "algorithmic_bytes": alg_bytes, "peak_kind": peak_kind,
                     "per_unit": f"{bbytes} B per checkpoint block read and 32 B per "
                                 f"interval-table sector or pair record read; "
                                 f"{blocks_per_step / max(nodes_per_step, 1):.3f} blocks and "
                                 f"{tables_per_step / max(nodes_per_step, 1):.3f} table sectors "
                                 f"per node, {nodes_per_step / nq:.1f} nodes per query"},
        "gpu_launches": launches,
        "clocks": clocks,
        "search": {"nodes_per_step": nodes_per_step, "blocks_per_step": blocks_per_step,
                   "table_sectors_per_step": tables_per_step,
                   "intervals_per_step": int(ref_offsets[-1].item()),
                   "bit_exact_repeat": same, "step_ms": step_ms, "fill": fill,
                   "profile_last": prof.as_dict()},
        "plain": plain,
        "best_hits": best,
        "end_restricted": endr,
        # end to end through the C ABI with host buffers (the serving calls); the device-pointer
        # call with torch copies of the same batch beside it
        "e2e": e2e_abi,
        "e2e_device_api_with_copies": e2e,
        "occ8": occ8,
        "exact": exact,
        "inexact_64mbp": cfg3,
        "both_strands_256mbp": both,
        "serving": serving,
        "locate": locate,
        "cpu_baseline": cpu,
        "cpu_baseline_configs": cpu_cfg,
        "setup": notes,
    }
    if rank == 0:
        s = json.dumps(line)
        print(s, flush=True)
        if args.log:
            with open(args.log, "a") as f:
                f.write(s + "\n")
    if dist is not None:
        dist.destroy_process_group()
    return 0


def gather_sweep(torch, fmocc):
    """Random-gather throughput by granule and footprint (fm_probe_gather)."""
    dev = torch.device("cuda", 0)
    fmocc.load_library()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    big = torch.empty(8 << 30, dtype=torch.uint8, device=dev)
    threads = torch.cuda.get_device_properties(dev).multi_processor_count * 2048
    for size in (128 << 20, 512 << 20, 1 << 30, 2 << 30, 8 << 30):
      buf = big[:size]
      for inflight in (1, 4, 8):
        for g in (32, 64, 128) if inflight < 8 else (32, 64):
            per = 64 if g == 32 else 32
            sink = torch.empty(threads, dtype=torch.int32, device=dev)
            for _ in range(3):
                fmocc.fm_probe_gather(buf, g, threads, per, 7, sink, inflight=inflight)
            ms = []
            for r in range(5):
                flush.add_(1)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fmocc.fm_probe_gather(buf, g, threads, per, 100 + r, sink, inflight=inflight)
                b.record()
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            t = float(np.median(ms)) / 1e3
            n = threads * per
            print(json.dumps({"footprint_MB": size >> 20, "granule": g, "inflight": inflight,
                              "ms": t * 1e3,
                              "G_gathers_s": n / t / 1e9, "useful_GB_s": n * g / t / 1e9}),
                  flush=True)
    return 0


def gather_ceiling(torch, fmocc, dev, footprint, flush):
    """Empirical random-gather ceiling: fm_probe_gather reads random 32-byte sectors of a
    device buffer as large as the index (all SMs, full occupancy, 4 loads in flight per
    thread); median of 5 launches."""
    footprint = max(int(footprint) // 32 * 32, 1 << 20)
    buf = torch.empty(footprint, dtype=torch.uint8, device=dev)
    threads = torch.cuda.get_device_properties(dev).multi_processor_count * 2048
    per = 64
    sink = torch.empty(threads, dtype=torch.int32, device=dev)
    for _ in range(3):
        fmocc.fm_probe_gather(buf, 32, threads, per, 7, sink)
    ms = []
    for r in range(5):
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fmocc.fm_probe_gather(buf, 32, threads, per, 100 + r, sink)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = float(np.median(ms)) / 1000
    del buf
    return {"g_gathers_s": threads * per / t / 1e9, "granule_bytes": 32,
            "useful_gb_s": threads * per * 32 / t / 1e9, "footprint_bytes": footprint}


def bench_occ8(args, torch, fmocc, synth, dev, hbm_peak, peak_kind, flush, barrier,
               max_over_ranks, world):
    """Config 2 at the main checkpoint interval, and beside it at the other intervals of
    {64, 128, 256} (each with its own index and the query mix drawn for its block size)."""
    R = synth.gc_text(SEED_OCC, args.occ_n, 0.41)
    main = occ8_at(args, args.interval, R, torch, fmocc, synth, dev, hbm_peak, peak_kind, flush,
                   barrier, max_over_ranks, world)
    main["other_intervals"] = [
        occ8_at(args, I, R, torch, fmocc, synth, dev, hbm_peak, peak_kind, flush, barrier,
                max_over_ranks, world) for I in (64, 128, 256) if I != args.interval]
    return main


def occ8_at(args, I, R, torch, fmocc, synth, dev, hbm_peak, peak_kind, flush, barrier,
            max_over_ranks, world):
    t0 = time.time()
    h = fmocc.fm_build(R, interval=I, device=dev.index, forward_only=True)
    n = args.occ_n
    k, l = synth.occ_queries_mixed(SEED_OCC, n, args.occ_queries, I)
    same = (k // I) == ((l.astype(np.int64) + 1) // I)
    blocks = float(np.where(same, 1, 2).sum())
    kd = torch.from_numpy(k.view(np.int32)).to(dev)
    ld = torch.from_numpy(l.view(np.int32)).to(dev)
    del k, l
    out = torch.empty((args.occ_queries, 8), dtype=torch.int32, device=dev)
    setup_s = time.time() - t0
    for _ in range(3):
        fmocc.fm_occ8(h, kd, ld, out)
    barrier()
    ms = []
    for _ in range(max(args.steps, 3)):
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fmocc.fm_occ8(h, kd, ld, out)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = max_over_ranks(float(np.mean(ms)) / 1000.0)
    bb = BLOCK_BYTES[I]
    gather = blocks * bb
    ceil = gather_ceiling(torch, fmocc, dev, fmocc.fm_info(h)["n_blocks"] * bb, flush)
    io = args.occ_queries * 40.0
    h.close()
    return {"value": args.occ_queries * world / t / 1e9, "unit": "G 8-Occ/s",
            "config": {"reference_bp": n, "gc": 0.41, "queries": args.occ_queries,
                       "interval": I, "block_bytes": bb, "same_block_frac": float(same.mean())},
            "ms_per_launch": t * 1000,
            "roofline": {"bound": "hbm", "achieved": gather / t / 1e9, "peak": hbm_peak,
                         "unit": "GB/s", "frac": gather / t / 1e9 / hbm_peak,
                         "peak_kind": peak_kind,
                         "gather_roofline_gq_s": hbm_peak * 1e9 / (gather / args.occ_queries) / 1e9,
                         "total_traffic_frac": (gather + io) / t / 1e9 / hbm_peak,
                         "blocks_per_query": blocks / args.occ_queries,
                         "gather_ceiling": ceil,
                         "frac_of_gather_ceiling": blocks / t / 1e9 / ceil["g_gathers_s"]},
            "setup_s": setup_s}


def bench_locate(args, torch, fmocc, h, dev, flush):
    """Locate (Eq. 4-5) of 2^24 uniform random rows of the 2 Gbp index: SA samples every 32
    rows, one Psi^-1 step (one block gather) per walked row."""
    n = fmocc.fm_info(h)["n"]
    g = torch.Generator(device="cpu").manual_seed(1811061276)
    rows = torch.randint(0, n + 1, (1 << 24,), generator=g, dtype=torch.int64).to(torch.int32).to(dev)
    pos = torch.empty_like(rows)
    steps = torch.zeros(1, dtype=torch.int64, device=dev)
    for _ in range(2):
        fmocc.fm_locate(h, rows, pos)
    ms = []
    for _ in range(3):
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fmocc.fm_locate(h, rows, pos, steps=steps)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = float(np.median(ms)) / 1000
    st = int(steps.item()) / 3
    return {"rows": 1 << 24, "rows_per_s": (1 << 24) / t, "ms": t * 1000,
            "steps_per_row": st / (1 << 24), "steps_per_s": st / t}


def bench_e2e_serving_abi(args, fmocc, h, reads, world):
    """The main batch end to end through the host-buffer serving ABI: the 10^7 reads submitted
    from host memory as requests of the server's maximum batch (fm_server_submit copies them),
    searched by the server's workers (three batches in flight), and every result read back to host
    memory (fm_server_poll); timed from the first submission to the last result."""
    chunk = 262_144
    nr = len(reads)
    with fmocc.Server(h, max_batch_reads=chunk, strands=2) as srv:
        # one untimed request sizes the workers' buffers and scratch
        w = reads.subset(np.arange(min(chunk, nr)))
        srv.wait(srv.submit(w.codes, w.offs, 2, 1))
        t0 = time.perf_counter()
        tickets = []
        for a in range(0, nr, chunk):
            b = min(nr, a + chunk)
            offs = reads.offs[a:b + 1]
            tickets.append(srv.submit(reads.codes[offs[0]:offs[-1]], offs - offs[0], 2, 1))
        d2h = 0
        for t in tickets:
            r = srv.wait(t)
            d2h += r["counts"].nbytes + r["offsets"].nbytes + r["pairs"].nbytes
        dt = time.perf_counter() - t0
    return {"value": nr * world / dt, "unit": "reads/s", "seconds": dt,
            "h2d_bytes_per_step": int(reads.codes.nbytes + reads.offs.nbytes),
            "d2h_bytes_per_step": int(d2h),
            "what": f"fm_server_submit/poll with host buffers, {len(tickets)} requests of up to "
                    f"{chunk} reads, z=2 with 1 gap, both strands; host clock"}


def bench_serving(args, fmocc, h, reads):
    """Serving on the resident 2 Gbp index: requests of U[1, 4096] reads of the main read model,
    mode uniform over {exact, z=1, z=2 with one gap}, both strands.  First the offline rate
    (a backlog of requests submitted at once), then Poisson arrivals at 0.5x and 0.8x that rate
    for a few seconds each; latency = completion - submission (library steady clock)."""
    modes = [(0, 0), (1, 0), (2, 1)]
    rng = np.random.default_rng(1811061275)
    nr = len(reads)
    cursor = [0]

    def next_request():
        m = int(rng.integers(1, 4097))
        if cursor[0] + m > nr:
            cursor[0] = 0
        a = cursor[0]
        cursor[0] += m
        z, g = modes[int(rng.integers(0, 3))]
        offs = reads.offs[a:a + m + 1]
        return reads.codes[offs[0]:offs[-1]], offs - offs[0], z, g, m

    out = {"requests": "U[1,4096] reads of 50-250 bp, mode uniform over exact / z=1 / z=2+1 gap",
           "rates": []}
    with fmocc.Server(h, max_batch_reads=262144, strands=2) as srv:
        # offline: a backlog of requests
        reqs = [next_request() for _ in range(200)]
        t0 = time.perf_counter()
        tk = [srv.submit(c, o, z, g) for c, o, z, g, _ in reqs]
        res = [srv.wait(t) for t in tk]
        dt = time.perf_counter() - t0
        total = sum(r[4] for r in reqs)
        offline = total / dt
        out["offline_reads_per_s"] = offline
        out["offline_batches"] = srv.stats()["batches"]
        for load in (0.5, 0.8):
            lam = load * offline / 2048.5            # requests per second
            duration = args.serve_seconds
            arrivals = np.cumsum(rng.exponential(1.0 / lam, size=int(lam * duration * 1.5) + 10))
            arrivals = arrivals[arrivals < duration]
            reqs = [next_request() for _ in range(arrivals.size)]
            b0 = srv.stats()["batches"]
            start = time.perf_counter()
            tk = []
            for (c, o, z, g, _), at in zip(reqs, arrivals):
                delay = start + at - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                tk.append(srv.submit(c, o, z, g))
            res = [srv.wait(t) for t in tk]
            end = time.perf_counter()
            lat = np.array([(r["t_done_ns"] - r["t_submit_ns"]) / 1e6 for r in res])
            nreads = sum(r[4] for r in reqs)
            out["rates"].append({"load": load, "offered_reads_per_s": load * offline,
                                 "requests": len(reqs), "reads": nreads,
                                 "achieved_reads_per_s": nreads / (end - start),
                                 "p50_ms": float(np.percentile(lat, 50)),
                                 "p99_ms": float(np.percentile(lat, 99)),
                                 "batches": srv.stats()["batches"] - b0})
    return out


def bench_both_strands(args, torch, fmocc, synth, dev, flush, barrier):
    """Both strands two ways, 256 Mbp repeat reference, 10^6 reads of the main read model,
    z=2 with 1 gap: each read and its reverse complement as two queries on the index of R,
    against one query per read on the index of R . revcomp(R) (FM_BUILD_BOTH_STRANDS)."""
    R = synth.repeat_text(1811061276, 256_000_000)
    reads = synth.sample_reads(1811061276, R, 1_000_000, 50, 250, sub_rate=0.01,
                               indel_rate=0.0005, both_strands=True)
    codes, offs = fmocc.to_device_reads(reads, dev)
    out = {"reference_bp": R.size, "reads": len(reads)}
    for name, kw, strands in (("two_queries", {}, 2), ("one_query_both_strands_index",
                                                        {"both_strands": True}, 1)):
        h = fmocc.fm_build(R, interval=64, device=dev.index, **kw)
        stats = torch.zeros(4, dtype=torch.int64, device=dev)
        prof = fmocc.fm_profile()
        fmocc.fm_inexact(h, codes, offs, 2, 1, strands=strands)   # sizing, tables
        ms = []
        for rep in range(3):
            flush()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            _, o, _ = fmocc.fm_inexact(h, codes, offs, 2, 1, strands=strands, profile=prof,
                                       stats=stats if rep else None)
            b.record()
            torch.cuda.synchronize()
            if rep:
                ms.append(a.elapsed_time(b))
        st = stats.cpu().numpy() / len(ms)
        out[name] = {"reads_per_s": len(reads) / (np.mean(ms) / 1000), "ms_per_step": np.mean(ms),
                     "nodes": float(st[0]), "intervals": int(o[-1].item()),
                     "index_bytes": fmocc.fm_info(h)["bytes_device"]}
        h.close()
    return out


def bench_cfg3(args, torch, fmocc, synth, dev, flush, barrier, hbm_peak):
    """Inexact search on the 64 Mbp repeat reference: 10^6 reads of 100 bp (0.5% substitutions,
    5% random, both strands), z=2 mismatches only, D pruning, persistent kernel."""
    R = synth.repeat_text(1811061273, 64_000_000)
    reads = synth.sample_reads(1811061273, R, 1_000_000, 100, 100, sub_rate=0.005,
                               both_strands=True, random_frac=0.05)
    h = fmocc.fm_build(R, interval=64, device=dev.index)
    codes, offs = fmocc.to_device_reads(reads, dev)
    nq = 2 * len(reads)
    counts = torch.empty(nq, dtype=torch.int32, device=dev)
    offsets = torch.empty(nq + 1, dtype=torch.int64, device=dev)
    prof = fmocc.fm_profile()
    stats = torch.zeros(4, dtype=torch.int64, device=dev)
    _, _, p0 = fmocc.fm_inexact(h, codes, offs, 2, 0, strands=2, counts=counts, offsets=offsets)
    pairs = torch.empty((p0.shape[0] + 1024, 2), dtype=torch.int32, device=dev)
    for _ in range(3):
        fmocc.fm_inexact(h, codes, offs, 2, 0, strands=2, counts=counts, offsets=offsets,
                         pairs=pairs)
    barrier()
    ms, kms = [], []
    for _ in range(max(args.steps, 3)):
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fmocc.fm_inexact(h, codes, offs, 2, 0, strands=2, counts=counts, offsets=offsets,
                         pairs=pairs, stats=stats, profile=prof)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        kms.append(prof.ms_search)
    st = stats.cpu().numpy() / len(ms)
    h.close()
    t = float(np.mean(ms)) / 1000
    alg = st[1] * 32
    return {"config": "64 Mbp repeat reference, 1,000,000 x 100 bp reads (0.5% subst, 5% "
                      "random), both strands, z=2 mismatches only, I=64",
            "reads_per_s": len(reads) / t, "ms_per_step": t * 1000,
            "kernel_ms": float(np.mean(kms)), "nodes_per_read": float(st[0]) / len(reads),
            "roofline": {"bound": "hbm", "achieved": alg / (np.mean(kms) / 1000) / 1e9,
                         "peak": hbm_peak, "unit": "GB/s",
                         "frac": alg / (np.mean(kms) / 1000) / 1e9 / hbm_peak,
                         "note": "index 2 x 64 MB: mostly L2-resident"}}


def bench_exact(args, torch, fmocc, synth, dev, flush, barrier):
    R = synth.uniform_text(SEED_EXACT, 1_000_000)
    h = fmocc.fm_build(R, interval=args.interval, device=dev.index)
    reads = synth.exact_reads(SEED_EXACT, R, 10_000, 32)
    codes, offs = fmocc.to_device_reads(reads, dev)
    k1, l1 = synth.occ_queries_uniform(SEED_EXACT, R.size, 1_000_000)
    kd = torch.from_numpy(k1.view(np.int32)).to(dev)
    ld = torch.from_numpy(l1.view(np.int32)).to(dev)
    out = torch.empty((kd.numel(), 8), dtype=torch.int32, device=dev)
    for _ in range(3):
        fmocc.fm_exact(h, codes, offs)
        fmocc.fm_occ8(h, kd, ld, out)
    barrier()
    ms_e, ms_o = [], []
    for _ in range(max(args.steps, 3)):
        for fn, acc in ((lambda: fmocc.fm_exact(h, codes, offs), ms_e),
                        (lambda: fmocc.fm_occ8(h, kd, ld, out), ms_o)):
            flush()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            acc.append(a.elapsed_time(b))
    h.close()
    te, to = float(np.mean(ms_e)), float(np.mean(ms_o))
    return {"config": "1 Mbp uniform reference, 10,000 reads of 32 bp (90% copied), I=64; "
                      "1,000,000 fm_occ8 queries",
            "reads_per_s": 10_000 / (te / 1000), "ms_per_call": te,
            "occ8_gq_s": 1e6 / (to / 1000) / 1e9, "occ8_ms": to,
            "note": "index L2-resident (0.5 MB): latency-bound, no roofline claim"}


if __name__ == "__main__":
    sys.exit(main())
