"""Autotuner of the batched inexact search.

It picks the checkpoint interval I (index layout), the warps per CTA and CTAs per SM of the
persistent kernel (occupancy) and the number of queries a warp takes from the work queue at
once (the frontier chunk), by timing the search kernel itself (CUDA events recorded by the
library on the launching stream, ``fm_profile.ms_search``) on a sample of the workload's reads.
In this design every lane expands one node per step, whichever read it belongs to, so the
"lanes per read" of a read-per-lane design is not a knob here; the chunk plays its role.

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
             sample_reads: int = 200_000, cache_path: str | None = None, device: int = -1,
             log=None) -> dict:
    """Return the best configuration {interval, warps_per_block, blocks_per_sm, chunk,
    ms_search, ...} for searching ``reads`` (a synth.Reads batch) in ``ref_codes``."""
    space = dict(DEFAULT_SPACE, **(space or {}))
    workload = dict(workload or {}, n=int(ref_codes.size), z=z, max_gaps=max_gaps,
                    strands=strands, sample=sample_reads)
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
                               "blocks_per_sm": bps, "chunk": chunk, "ms_search": ms})
                if log:
                    log(trials[-1])
        finally:
            h.close()
    best = pick(trials)
    result = dict(best, trials=len(trials), tune_seconds=time.time() - t0, sample_reads=n)
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


def apply(h, cfg: dict):
    """Set the tuned kernel knobs on an index built with cfg['interval']."""
    fmocc.fm_set_tuning(h, warps_per_block=cfg["warps_per_block"],
                        blocks_per_sm=cfg["blocks_per_sm"], chunk=cfg["chunk"])
