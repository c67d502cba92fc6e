"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and the benchmark.

This module holds none of the FM-index arithmetic: it only draws texts, reads and query
positions from a counter-based hash, so that both sides of every parity test see the same
bytes.  Everything is numpy and deterministic for a given seed on a given machine.

Counter-based generator: splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used as a hash of (seed, counter):
    z = seed + (counter + 1) * 0x9E3779B97F4A7C15
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    out = z ^ (z >> 31)            (all arithmetic mod 2^64)

Symbol codes are A=0, C=1, G=2, T=3 (the 2-bit code of Fig. 2 of the paper).

Workload recipes (the paper measures on NA12878 reads against hg38, which are not available;
these genome-shaped stand-ins take their shapes from the configurations below):
  * ``uniform_text``: i.i.d. uniform ACGT (plain exact-search reference, 1 Mbp).
  * ``gc_text``: i.i.d. ACGT at a given GC fraction (41%: P(C)=P(G)=0.205, P(A)=P(T)=0.295),
    the 2 Gbp Occ micro-benchmark reference.
  * ``repeat_text``: a 41% GC background in which 20% of the bases are copies of 500 repeat
    families (consensus 300..6000 bp, each copy 10% substituted, reverse-complemented with
    probability 1/2, copies at non-overlapping uniform positions): the 64 Mbp and 2 Gbp
    inexact-search references.
  * ``sample_reads``: reads copied from uniform positions of either strand with substitution
    and single-base indel errors, plus a fraction of uniform random reads.
  * ``occ_queries_uniform`` / ``occ_queries_mixed``: (k, l) rank-query pairs for fm_occ8.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)

# chunk of hashes evaluated at once (bounds host memory for 2 Gbp texts)
_CHUNK = 1 << 24


def _pmap(fn, starts):
    """Run fn(start) for every chunk start on a thread pool (numpy releases the GIL); every
    draw is keyed by absolute position, so the result does not depend on the schedule."""
    starts = list(starts)
    if len(starts) <= 1:
        for st in starts:
            fn(st)
        return
    workers = min(len(starts), os.cpu_count() or 1, 32)
    with ThreadPoolExecutor(max_workers=workers) as ex:
        list(ex.map(fn, starts))


def splitmix64(seed: int, idx) -> np.ndarray:
    """splitmix64 output for each counter in ``idx`` (uint64 array) under ``seed``."""
    with np.errstate(over="ignore"):
        z = np.asarray(idx, dtype=np.uint64) + np.uint64(1)
        z = z * _GOLDEN + np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        return z ^ (z >> np.uint64(31))


def substream(seed: int, tag: int) -> int:
    """Derive an independent seed for a named sub-stream."""
    return int(splitmix64(seed, np.array([tag], dtype=np.uint64))[0])


def hashes(seed: int, count: int, start: int = 0) -> np.ndarray:
    out = np.empty(count, dtype=np.uint64)

    def one(s):
        e = min(count, s + _CHUNK)
        out[s:e] = splitmix64(seed, np.arange(start + s, start + e, dtype=np.uint64))

    _pmap(one, range(0, count, _CHUNK))
    return out


def uniform01(seed: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each hash."""
    return (hashes(seed, count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def randint(seed: int, count: int, lo, hi) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive; lo/hi may be arrays) as int64."""
    lo = np.asarray(lo, dtype=np.int64)
    hi = np.asarray(hi, dtype=np.int64)
    span = (hi - lo + 1).astype(np.uint64)
    h = hashes(seed, count)
    # multiply-shift range reduction on the top 32 bits (spans here are < 2^32)
    return lo + (((h >> np.uint64(32)) * span) >> np.uint64(32)).astype(np.int64)


# --------------------------------------------------------------------------------------------
# texts
# --------------------------------------------------------------------------------------------

def uniform_text(seed: int, n: int) -> np.ndarray:
    """n i.i.d. uniform codes: base j is bits 2(j%32)..2(j%32)+1 of hash(seed, j//32)."""
    nh = (n + 31) // 32
    out = np.empty(nh * 32, dtype=np.uint8)
    shifts = np.array([0, 2, 4, 6], dtype=np.uint8)

    def one(s):
        e = min(nh, s + _CHUNK)
        b = splitmix64(seed, np.arange(s, e, dtype=np.uint64)).view(np.uint8)
        out[s * 32:e * 32] = ((b[:, None] >> shifts) & 3).reshape(-1)

    _pmap(one, range(0, nh, _CHUNK))
    return out[:n].copy()


def _gc_thresholds(gc: float):
    pa = (1.0 - gc) / 2.0
    pc = gc / 2.0
    t1 = int(round(pa * 65536))
    t2 = int(round((pa + pc) * 65536))
    t3 = int(round((pa + 2 * pc) * 65536))
    return np.uint16(t1), np.uint16(t2), np.uint16(t3)


def gc_text(seed: int, n: int, gc: float = 0.41) -> np.ndarray:
    """n i.i.d. codes with P(C)=P(G)=gc/2: base j from 16-bit field j%4 of hash(seed, j//4)."""
    t1, t2, t3 = _gc_thresholds(gc)
    nh = (n + 3) // 4
    out = np.empty(nh * 4, dtype=np.uint8)

    def one(s):
        e = min(nh, s + _CHUNK)
        u = splitmix64(seed, np.arange(s, e, dtype=np.uint64)).view(np.uint16)
        c = (u >= t1).astype(np.uint8)
        c += (u >= t2)
        c += (u >= t3)
        out[s * 4:e * 4] = c

    _pmap(one, range(0, nh, _CHUNK))
    return out[:n].copy()


def revcomp(codes: np.ndarray) -> np.ndarray:
    return (3 - codes[::-1]).astype(np.uint8)


def _substitute(seed: int, codes: np.ndarray, rate: float) -> np.ndarray:
    """Replace each base with probability ``rate`` by one of the three other bases."""
    m = codes.size
    if m == 0 or rate <= 0:
        return codes.copy()
    h = hashes(seed, m)
    thr = np.uint64(int(rate * 2.0 ** 32))
    hit = (h & np.uint64(0xFFFFFFFF)) < thr
    shift = ((h >> np.uint64(32)) % np.uint64(3)).astype(np.uint8) + 1
    out = codes.copy()
    out[hit] = (out[hit] + shift[hit]) & 3
    return out


def repeat_text(seed: int, n: int, gc: float = 0.41, repeat_frac: float = 0.2,
                families: int = 500, min_len: int = 300, max_len: int = 6000,
                divergence: float = 0.10, rc_prob: float = 0.5) -> np.ndarray:
    """Genome-shaped reference: 41% GC background plus copies of repeat families.

    Each family has a consensus of uniform length in [min_len, max_len] and receives an equal
    expected share repeat_frac*n/families of repeat bases, i.e. round(share/len) copies (at
    least one, so when the share is below the longer consensus lengths the copies cover more
    than repeat_frac: 41% at n = 4e6 with 500 families, 20.0% at 6.4e7 and 2e9).  Every copy is substituted independently at ``divergence`` and reversed and
    complemented with probability ``rc_prob``.  The copies are shuffled and laid at
    non-overlapping uniform positions: sorted uniform offsets in [0, n - total] are shifted
    by the lengths of the copies before them.
    """
    text = gc_text(substream(seed, 1), n, gc)
    lens = randint(substream(seed, 2), families, min_len, max_len)
    share = repeat_frac * n / families
    ncopy = np.maximum(1, np.rint(share / lens)).astype(np.int64)
    total = int((ncopy * lens).sum())
    if total > n:
        raise ValueError("repeat copies do not fit the reference")
    cons_all = gc_text(substream(seed, 3), int(lens.sum()), gc)
    cons_off = np.concatenate([[0], np.cumsum(lens)])
    fam_of_copy = np.repeat(np.arange(families), ncopy)
    ncopies = fam_of_copy.size
    order = np.argsort(hashes(substream(seed, 4), ncopies), kind="stable")
    fam_of_copy = fam_of_copy[order]
    clen = lens[fam_of_copy]
    gaps = np.sort(randint(substream(seed, 5), ncopies, 0, n - total))
    starts = gaps + np.concatenate([[0], np.cumsum(clen)[:-1]])
    flips = uniform01(substream(seed, 6), ncopies) < rc_prob
    # all copy bases laid out in placement order, then substituted in one vectorised pass
    body = np.empty(total, dtype=np.uint8)
    pos = 0
    for c in range(ncopies):
        f = fam_of_copy[c]
        seg = cons_all[cons_off[f]:cons_off[f + 1]]
        if flips[c]:
            seg = 3 - seg[::-1]
        body[pos:pos + seg.size] = seg
        pos += seg.size
    body = _substitute(substream(seed, 7), body, divergence)
    pos = 0
    for c in range(ncopies):
        L = int(clen[c])
        s = int(starts[c])
        text[s:s + L] = body[pos:pos + L]
        pos += L
    return text


# --------------------------------------------------------------------------------------------
# reads
# --------------------------------------------------------------------------------------------

class Reads:
    """Concatenated read codes with offsets (read r is codes[offs[r]:offs[r+1]])."""

    def __init__(self, codes: np.ndarray, offs: np.ndarray):
        self.codes = np.ascontiguousarray(codes, dtype=np.uint8)
        self.offs = np.ascontiguousarray(offs, dtype=np.uint32)

    def __len__(self):
        return self.offs.size - 1

    def read(self, r: int) -> np.ndarray:
        return self.codes[self.offs[r]:self.offs[r + 1]]

    def lengths(self) -> np.ndarray:
        return np.diff(self.offs.astype(np.int64))

    def subset(self, idx) -> "Reads":
        idx = np.asarray(idx, dtype=np.int64)
        lens = self.lengths()[idx]
        offs = np.zeros(idx.size + 1, dtype=np.int64)
        np.cumsum(lens, out=offs[1:])
        if idx.size:
            src = np.repeat(self.offs[idx].astype(np.int64) - offs[:-1], lens) + \
                np.arange(offs[-1], dtype=np.int64)
        else:
            src = np.zeros(0, dtype=np.int64)
        return Reads(self.codes[src], offs.astype(np.uint32))


def sample_reads(seed: int, text: np.ndarray, n_reads: int, min_len: int, max_len: int,
                 sub_rate: float = 0.0, indel_rate: float = 0.0, both_strands: bool = False,
                 random_frac: float = 0.0, chunk: int = 1 << 17) -> Reads:
    """Reads sampled from ``text`` with sequencing-like errors.

    Read r: length uniform in [min_len, max_len]; with probability ``random_frac`` a uniform
    random string, otherwise copied from a uniform start position.  Along the read each output
    base is, with probability indel_rate/2 each, an inserted random base (consumes no
    reference) or preceded by one deleted reference base; every copied base is substituted
    with probability ``sub_rate`` by one of the three other bases.  With ``both_strands`` half
    of the copied reads (chosen by hash) are reverse-complemented.

    Per output position one hash h supplies every draw: bits 0..31 the substitution test,
    bits 32..47 the substituted base, bits 48..49 a random base, bits 50..63 the indel test.
    """
    n = int(text.size)
    lens = randint(substream(seed, 11), n_reads, min_len, max_len)
    offs = np.zeros(n_reads + 1, dtype=np.int64)
    np.cumsum(lens, out=offs[1:])
    is_rand = uniform01(substream(seed, 12), n_reads) < random_frac
    flip = (uniform01(substream(seed, 13), n_reads) < 0.5) & both_strands
    # reference span needed: len plus room for a few deletions (clipped at the text end)
    maxspan = np.minimum(lens + (16 if indel_rate > 0 else 0), n)
    starts = randint(substream(seed, 14), n_reads, 0, n - maxspan)
    total = int(offs[-1])
    codes = np.empty(total, dtype=np.uint8)
    s_pos = substream(seed, 15)
    sub_thr = np.uint64(int(sub_rate * 2.0 ** 32))
    ins_thr = np.uint64(int(indel_rate / 2 * 2.0 ** 14))
    del_thr = np.uint64(int(indel_rate * 2.0 ** 14))
    def one(r0):
        r1 = min(n_reads, r0 + chunk)
        a, b = int(offs[r0]), int(offs[r1])
        m = b - a
        L = lens[r0:r1]
        rid = np.repeat(np.arange(r0, r1), L)
        seg0 = offs[r0:r1] - a
        tpos = np.arange(m, dtype=np.int64) - np.repeat(seg0, L)    # position within read
        h = splitmix64(s_pos, np.arange(a, b, dtype=np.uint64))
        if indel_rate > 0:
            ev = h >> np.uint64(50)
            ins = ev < ins_thr
            dele = (ev >= ins_thr) & (ev < del_thr)
            # reference offset consumed: t - (#ins up to t) + (#del up to t)
            step = dele.astype(np.int64) - ins.astype(np.int64)
            cs = np.cumsum(step)
            base = np.repeat(cs[seg0] - step[seg0], L)
            refoff = tpos + (cs - base)
        else:
            ins = None
            refoff = tpos
        src = starts[rid] + refoff
        np.clip(src, 0, n - 1, out=src)
        seq = text[src]
        rnd = ((h >> np.uint64(48)) & np.uint64(3)).astype(np.uint8)
        if ins is not None:
            seq[ins] = rnd[ins]
        if sub_rate > 0:
            hit = (h & np.uint64(0xFFFFFFFF)) < sub_thr
            shift = ((((h >> np.uint64(32)) & np.uint64(0xFFFF)) * np.uint64(3)) >> np.uint64(16)
                     ).astype(np.uint8) + 1
            seq[hit] = (seq[hit] + shift[hit]) & 3
        rr = np.repeat(is_rand[r0:r1], L)
        seq[rr] = rnd[rr]
        # reverse-complement flipped reads inside their segments
        fl = np.repeat(flip[r0:r1] & ~is_rand[r0:r1], L)
        if fl.any():
            rev = np.repeat(seg0 + L - 1, L) - tpos
            seq[fl] = 3 - seq[rev[fl]]
        codes[a:b] = seq

    _pmap(one, range(0, n_reads, chunk))
    return Reads(codes, offs.astype(np.uint32))


def exact_reads(seed: int, text: np.ndarray, n_reads: int = 10000, m: int = 32,
                copy_frac: float = 0.9) -> Reads:
    """Plain exact-search reads: ``copy_frac`` copied from uniform forward-strand positions,
    the rest uniform random strings."""
    return sample_reads(seed, text, n_reads, m, m, random_frac=1.0 - copy_frac)


# --------------------------------------------------------------------------------------------
# occ8 query positions
# --------------------------------------------------------------------------------------------

def occ_queries_uniform(seed: int, n: int, count: int):
    """k uniform in [0, n], l uniform in [k, n] (uint32 arrays)."""
    k = randint(substream(seed, 21), count, 0, n)
    l = randint(substream(seed, 22), count, k, n)
    return k.astype(np.uint32), l.astype(np.uint32)


def occ_queries_mixed(seed: int, n: int, count: int, interval: int, same_frac: float = 0.5,
                      gap_mean: float = 1000.0, chunk: int = 1 << 22):
    """Occ micro-benchmark queries.

    With probability ``same_frac`` the pair lies in one checkpoint block: block j uniform,
    then two distinct rank positions p1 < p2 uniform in that block (clipped to [0, n+1]),
    k = p1, l = p2 - 1, so k/I == (l+1)/I.  Otherwise k is uniform in [0, n] and
    l = k + g with g geometric (mean ``gap_mean``, support >= 1), redrawn while l > n.
    Query q draws from two hashes, 2q and 2q+1 of the seed.
    """
    I = interval
    nblk = max((n + 1) // I, 1)       # blocks with at least two rank positions in [0, n+1]
    k_out = np.empty(count, dtype=np.uint32)
    l_out = np.empty(count, dtype=np.uint32)
    lq = np.log1p(-1.0 / gap_mean)
    sthr = np.uint64(int(same_frac * 2.0 ** 16))
    M32 = np.uint64(0xFFFFFFFF)

    def one(c0):
        c1 = min(count, c0 + chunk)
        m = c1 - c0
        h = splitmix64(seed, np.arange(2 * c0, 2 * c1, dtype=np.uint64))
        h1, h2 = h[0::2], h[1::2]
        same = (h1 >> np.uint64(48)) < sthr
        # same block: j from the low 32 bits of h1, the two positions from h2
        j = (((h1 & M32) * np.uint64(nblk)) >> np.uint64(32)).astype(np.int64)
        lo = j * I
        hi = np.minimum(lo + I - 1, n + 1)                          # inclusive last position
        span_a = (hi - lo).astype(np.uint64)                        # a in [lo, hi-1]
        a = lo + (((h2 & M32) * span_a) >> np.uint64(32)).astype(np.int64)
        span_b = np.maximum(hi - a, 1).astype(np.uint64)            # b in [0, hi-a-1]
        b = (((h2 >> np.uint64(32)) * span_b) >> np.uint64(32)).astype(np.int64)
        ks = a
        ls = a + b                                                  # p2 - 1 with p2 = a + 1 + b
        # geometric gap: k from h1's bits 16..47, u from h2's top 53 bits
        k = ((((h1 >> np.uint64(16)) & M32) * np.uint64(n + 1)) >> np.uint64(32)).astype(np.int64)
        u = (h2 >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        l = k + 1 + np.floor(np.log1p(-u) / lq).astype(np.int64)
        bad = np.flatnonzero(~same & (l > n))
        tries = 0
        while bad.size:
            hb = splitmix64(substream(seed, 1_000_003 + tries),
                            np.arange(c0, c0 + bad.size, dtype=np.uint64))
            ub = (hb >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
            l[bad] = k[bad] + 1 + np.floor(np.log1p(-ub) / lq).astype(np.int64)
            bad = bad[l[bad] > n]
            tries += 1
            if tries > 200:
                l[bad] = n
                break
        k_out[c0:c1] = np.where(same, ks, k)
        l_out[c0:c1] = np.where(same, ls, l)

    _pmap(one, range(0, count, chunk))
    return k_out, l_out


def random_strings(seed: int, count: int, min_len: int, max_len: int) -> Reads:
    lens = randint(substream(seed, 31), count, min_len, max_len)
    offs = np.zeros(count + 1, dtype=np.int64)
    np.cumsum(lens, out=offs[1:])
    codes = uniform_text(substream(seed, 32), int(offs[-1]))
    return Reads(codes, offs.astype(np.uint32))


def to_ascii(codes: np.ndarray) -> bytes:
    return np.frombuffer(b"ACGT", dtype=np.uint8)[codes].tobytes()


def from_ascii(s) -> np.ndarray:
    if isinstance(s, str):
        s = s.encode()
    a = np.frombuffer(s, dtype=np.uint8)
    lut = np.full(256, 255, dtype=np.uint8)
    for i, ch in enumerate(b"ACGT"):
        lut[ch] = i
        lut[ch + 32] = i
    out = lut[a]
    if (out == 255).any():
        raise ValueError("text holds symbols outside ACGTacgt")
    return out
