"""Autotuner of the batched inexact search.

It picks, by timing the search kernel itself (CUDA events recorded by the library on the
launching stream, ``fm_profile.ms_search``) on a sample of the workload's reads:
  * stage 1: the checkpoint interval I (index layout), the warps per CTA and CTAs per SM of
    the persistent kernel (occupancy) and the number of queries a warp takes from the work
    queue at once (the frontier chunk), with the library's default tables;
  * stage 2, at the stage-1 choice: the depth of the interval tables of short strings
    (relative to the automatic depth floor(log4(n+1)) - 1) and whether exact continuations
    take two symbols per step over the pair table.
In this design every lane expands one node per step, whichever read it belongs to, so the
"lanes per read" of a read-per-lane design is not a knob here; the chunk plays its role.
Every knob changes speed and memory only, never results; ``points`` lists every configuration
the tuner can return, so that the parity tests can run each one.

The default sample is 10^6 reads: on a 2 Gbp index a 2 x 10^5-read sample runs the kernel for
about 11 ms, where the last warps' tail favours small CTAs (4 warps per CTA won there, and ran
2.5% slower than 8 on the full batch of 10^7 reads).

Results are cached as JSON keyed by the GPU name and the workload description, so a later
run with the same key skips the search.  Everything runs through the C ABI.
"""
from __future__ import annotations

import itertools
import json
import os
import time

import numpy as np
import torch

from . import fmocc

DEFAULT_SPACE = {
    "interval": (32, 64, 128),
    "warps_per_block": (4, 8),
    "blocks_per_sm": (2, 3, 32),     # 32: as many as fit (the library clamps to occupancy)
    "chunk": (8, 16, 32),
}
# stage 2: interval-table depth relative to the automatic one, and pair steps (1 on, 2 off)
TABLE_SPACE = {
    "kmer_offset": (-1, 0, 1),
    "pair_steps": (1, 2),
}


def auto_kmer_depth(n: int) -> int:
    """The library's automatic interval-table depth for a reference of n symbols:
    floor(log4(n+1)) - 1, at most 15 (0: no tables)."""
    lg = 0
    while 4 ** (lg + 1) <= n + 1:
        lg += 1
    return min(15, lg - 1) if lg > 1 else 0


def kmer_depth_of(n: int, offset: int) -> int:
    return max(1, min(15, auto_kmer_depth(n) + offset))


def points(n: int, space: dict | None = None, table_space: dict | None = None):
    """Every configuration the tuner can return for a reference of n symbols, as dicts of
    interval, warps_per_block, blocks_per_sm, chunk, kmer_depth and pair_steps (the stage-2
    knobs can be combined with any stage-1 point, since stage 1 may pick any of them)."""
    space = dict(DEFAULT_SPACE, **(space or {}))
    ts = dict(TABLE_SPACE, **(table_space or {}))
    depths = sorted({kmer_depth_of(n, o) for o in ts["kmer_offset"]})
    out = []
    for I, wpb, bps, chunk, kd, ps in itertools.product(
            space["interval"], space["warps_per_block"], space["blocks_per_sm"], space["chunk"],
            depths, ts["pair_steps"]):
        out.append({"interval": I, "warps_per_block": wpb, "blocks_per_sm": bps,
                    "chunk": chunk, "kmer_depth": kd, "pair_steps": ps})
    return out


def _key(workload: dict) -> str:
    name = torch.cuda.get_device_name()
    return name + "|" + json.dumps(workload, sort_keys=True)


def load_cache(path: str) -> dict:
    if path and os.path.exists(path):
        try:
            return json.load(open(path))
        except (OSError, ValueError):
            return {}
    return {}


def save_cache(path: str, cache: dict):
    if not path:
        return
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_search(h, codes, offs, z, max_gaps, strands, bufs, repeats=2):
    prof = fmocc.fm_profile()
    best = float("inf")
    for _ in range(repeats):
        fmocc.fm_inexact(h, codes, offs, z, max_gaps, strands=strands, kernel="persistent",
                         counts=bufs[0], offsets=bufs[1], pairs=bufs[2], profile=prof)
        best = min(best, prof.ms_search)
    return best


def autotune(ref_codes: np.ndarray, reads, z: int, max_gaps: int, strands: int = 2,
             workload: dict | None = None, space: dict | None = None,
             sample_reads: int = 1_000_000, cache_path: str | None = None, device: int = -1,
             log=None, table_space: dict | None = None) -> dict:
    """Return the best configuration {interval, warps_per_block, blocks_per_sm, chunk,
    kmer_depth, pair_steps, ms_search, ...} for searching ``reads`` (a synth.Reads batch) in
    ``ref_codes``."""
    space = dict(DEFAULT_SPACE, **(space or {}))
    ts = dict(TABLE_SPACE, **(table_space or {}))
    workload = dict(workload or {}, n=int(ref_codes.size), z=z, max_gaps=max_gaps,
                    strands=strands, sample=sample_reads, stages=2)
    key = _key(workload)
    cache = load_cache(cache_path)
    if key in cache:
        return dict(cache[key], cached=True)
    n = min(sample_reads, len(reads))
    sample = reads.subset(np.arange(n)) if n < len(reads) else reads
    codes, offs = fmocc.to_device_reads(sample)
    nq = n * strands
    bufs = (torch.empty(nq, dtype=torch.int32, device=codes.device),
            torch.empty(nq + 1, dtype=torch.int64, device=codes.device),
            torch.empty((8 * nq + 4096, 2), dtype=torch.int32, device=codes.device))
    n_ref = int(ref_codes.size)
    auto = auto_kmer_depth(n_ref)
    trials = []
    t0 = time.time()
    for interval in space["interval"]:
        h = fmocc.fm_build(ref_codes, interval=interval, device=device)
        try:
            for wpb, bps, chunk in itertools.product(space["warps_per_block"],
                                                     space["blocks_per_sm"], space["chunk"]):
                fmocc.fm_set_tuning(h, warps_per_block=wpb, blocks_per_sm=bps, chunk=chunk)
                _time_search(h, codes, offs, z, max_gaps, strands, bufs, repeats=1)  # warm
                ms = _time_search(h, codes, offs, z, max_gaps, strands, bufs)
                trials.append({"interval": interval, "warps_per_block": wpb,
                               "blocks_per_sm": bps, "chunk": chunk, "kmer_depth": auto,
                               "pair_steps": 1, "ms_search": ms})
                if log:
                    log(trials[-1])
        finally:
            h.close()
    best = pick(trials)
    # stage 2: tables at the stage-1 choice
    trials2 = []
    h = fmocc.fm_build(ref_codes, interval=best["interval"], device=device)
    try:
        fmocc.fm_set_tuning(h, warps_per_block=best["warps_per_block"],
                            blocks_per_sm=best["blocks_per_sm"], chunk=best["chunk"])
        for kd, ps in itertools.product(sorted({kmer_depth_of(n_ref, o)
                                                for o in ts["kmer_offset"]}), ts["pair_steps"]):
            fmocc.fm_set_tuning(h, kmer_depth=kd, pair_steps=ps)
            _time_search(h, codes, offs, z, max_gaps, strands, bufs, repeats=1)   # builds, warms
            ms = _time_search(h, codes, offs, z, max_gaps, strands, bufs)
            trials2.append(dict(best, kmer_depth=kd, pair_steps=ps, ms_search=ms))
            if log:
                log(trials2[-1])
    finally:
        h.close()
    best = pick_tables(trials2)
    result = dict(best, trials=len(trials) + len(trials2), tune_seconds=time.time() - t0,
                  sample_reads=n)
    cache[key] = result
    save_cache(cache_path, cache)
    return dict(result, cached=False)


def pick(trials, tolerance: float = 0.02) -> dict:
    """The fastest trial, except that among the trials within ``tolerance`` of it the one
    with the largest checkpoint interval (the smallest index in memory) wins, fastest first:
    intervals whose times differ by less than the run-to-run noise then tune to one stable
    configuration."""
    fastest = min(t["ms_search"] for t in trials)
    near = [t for t in trials if t["ms_search"] <= fastest * (1 + tolerance)]
    return min(near, key=lambda t: (-t["interval"], t["ms_search"]))


def pick_tables(trials, tolerance: float = 0.02) -> dict:
    """Stage 2: the fastest trial, except that among the trials within ``tolerance`` of it the
    one with the least table memory wins (shallower interval tables first, then no pair
    table), fastest first."""
    fastest = min(t["ms_search"] for t in trials)
    near = [t for t in trials if t["ms_search"] <= fastest * (1 + tolerance)]
    return min(near, key=lambda t: (t["kmer_depth"], -t["pair_steps"], t["ms_search"]))


def apply(h, cfg: dict):
    """Set the tuned kernel knobs on an index built with cfg['interval']."""
    fmocc.fm_set_tuning(h, warps_per_block=cfg["warps_per_block"],
                        blocks_per_sm=cfg["blocks_per_sm"], chunk=cfg["chunk"])
    if "kmer_depth" in cfg:
        fmocc.fm_set_tuning(h, kmer_depth=cfg["kmer_depth"], pair_steps=cfg["pair_steps"])
