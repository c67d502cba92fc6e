"""Parity at the full workload sizes, in the bench's launch configuration.

The oracle cannot index a 2 Gbp reference in test time (its SA-IS takes over ten minutes), so
here it computes sampled outputs one by one without an index, from the closed form of an
interval: for a string W, k = #{suffixes smaller than W} and the eight Occ values at rows k-1
and l come from one scan over all suffixes (oracle.interval_naive); the Hamming count of a
read is one sliding-window pass.  Every other output is checked through properties that hold
at any size.  All comparisons are exact (integers).
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_1811_06127_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_2G = 2_000_000_000
SEED_OCC, SEED_SEARCH = 1811061272, 1811061274


@pytest.fixture(scope="module")
def fm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1811_06127_gb300 import _build, fmocc
    _build.build()
    fmocc.load_library()
    return fmocc


def _strings(R, seed, count=24):
    """Sampled probe strings: substrings of R of length 8..30 and uniform random strings."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(count):
        m = int(rng.integers(8, 31))
        if t % 3 == 2:
            out.append(rng.integers(0, 4, m).astype(np.uint8))
        else:
            p = int(rng.integers(0, R.size - m))
            out.append(R[p:p + m].copy())
    codes = np.concatenate(out).astype(np.uint8)
    offs = np.concatenate([[0], np.cumsum([w.size for w in out])]).astype(np.uint32)
    return synth.Reads(codes, offs)


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def test_occ8_2gbp_sampled_and_properties(fm):
    """Config 2: 2 Gbp i.i.d. 41% GC index, 2^28 mixed queries (the bench's launch)."""
    R = synth.gc_text(SEED_OCC, N_2G, 0.41)
    h = fm.fm_build(R, interval=64, forward_only=True)
    n = R.size
    # sampled outputs the oracle computes one by one
    probes = _strings(R, 7)
    kn, ln, o8 = oracle.interval_naive(R, probes.codes, probes.offs)
    # the row holding $: rows below it are the suffixes smaller than R itself
    dk, _, _ = oracle.interval_naive(R, R, np.array([0, n], np.uint32), threads=1)
    dollar = int(dk[0])
    assert fm.fm_info(h)["dollar_row"] == dollar
    got = _u32(fm.fm_occ8(h, torch.from_numpy(kn.astype(np.uint32).view(np.int32)).cuda(),
                          torch.from_numpy(ln.astype(np.uint32).view(np.int32)).cuda()))
    assert np.array_equal(got.astype(np.int64), o8)
    # the bench's 2^28 queries: properties of every output on a 2^24 slice, all launched
    k, l = synth.occ_queries_mixed(SEED_OCC, n, 1 << 28, 64)
    kd = torch.from_numpy(k.view(np.int32)).cuda()
    ld = torch.from_numpy(l.view(np.int32)).cuda()
    out = fm.fm_occ8(h, kd, ld)
    sl = slice(0, 1 << 24)
    o = _u32(out[sl]).astype(np.int64)
    kk, ll = k[sl].astype(np.int64), l[sl].astype(np.int64)
    # the four counts at a rank position p sum to p minus the $ row when below p
    assert np.array_equal(o[:, :4].sum(1), kk - (dollar < kk))
    assert np.array_equal(o[:, 4:].sum(1), ll + 1 - (dollar <= ll))
    assert (o[:, 4:] >= o[:, :4]).all()
    # Occ(c, n) is the symbol count of R (the C array)
    C = np.asarray(fm.fm_info(h)["C"], dtype=np.int64)
    assert np.array_equal(C, oracle.count(R))
    at_n = ll == n
    if at_n.any():
        assert np.array_equal(o[at_n, 4:], np.tile(np.diff(C), (int(at_n.sum()), 1)))
    h.close()


def test_exact_and_mismatch_counts_2gbp_repeats(fm):
    """Config 4's reference (2 Gbp, repeat families) and read model: exact intervals against
    the closed form, and the z=2 mismatch-only interval sizes against sliding-window Hamming
    counts, for sampled reads; persistent = plain on a 100k-read slice of the batch."""
    R = synth.repeat_text(SEED_SEARCH, N_2G)
    h = fm.fm_build(R, interval=64)
    reads = synth.sample_reads(SEED_SEARCH, R, 100_000, 50, 250, sub_rate=0.01,
                               indel_rate=0.0005, both_strands=True)
    codes, offs = fm.to_device_reads(reads)
    # persistent and plain kernels agree bit for bit (z=2, 1 gap, both strands)
    a = fm.fm_inexact(h, codes, offs, 2, 1, strands=2, kernel="persistent")
    b = fm.fm_inexact(h, codes, offs, 2, 1, strands=2, kernel="plain")
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    counts, offsets, pairs = a
    pr = _u32(pairs).astype(np.int64)
    assert ((pr[:, 0] >= 1) & (pr[:, 0] <= pr[:, 1]) & (pr[:, 1] <= R.size)).all()
    # the optimisations change nothing at this size: canonical enumeration, interval tables and
    # two-symbol steps (the defaults) against every call of Listing 2, one symbol per step, no
    # tables, with costs, on a 20k-read slice
    sl = reads.subset(np.arange(20_000))
    lc, lo = fm.to_device_reads(sl)
    fast = fm.fm_inexact(h, lc, lo, 2, 1, strands=2, costs=True)
    fm.fm_set_tuning(h, canonical=2, kmer_depth=fm.KMER_OFF, pair_steps=2)
    literal = fm.fm_inexact(h, lc, lo, 2, 1, strands=2, costs=True)
    ke, le = fm.fm_exact(h, codes, offs)
    fm.fm_set_tuning(h, canonical=1, kmer_depth=fm.KMER_AUTO, pair_steps=1)
    for x, y in zip(fast, literal):
        assert torch.equal(x, y)
    k1, l1 = fm.fm_exact(h, codes, offs)
    assert torch.equal(ke, k1) and torch.equal(le, l1)
    # the cost-0 intervals of a read's search are exactly its exact-match interval
    fc, fo, fp, fcost = (t.cpu().numpy() for t in fast)
    ks, ls = _u32(k1)[:len(sl)], _u32(l1)[:len(sl)]
    for r in range(len(sl)):
        q = 2 * r
        zero = fp[fo[q]:fo[q + 1]][fcost[fo[q]:fo[q + 1]] == 0].view(np.uint32)
        want0 = [[ks[r], ls[r]]] if ks[r] <= ls[r] else []
        assert zero.tolist() == want0, r
    # exact intervals of sampled reads against the closed form
    sample = reads.subset(np.arange(8))
    kn, ln, _ = oracle.interval_naive(R, sample.codes, sample.offs)
    sc, so = fm.to_device_reads(sample)
    k, l = fm.fm_exact(h, sc, so)
    assert np.array_equal(_u32(k).astype(np.int64), kn)
    assert np.array_equal(_u32(l).astype(np.int64), ln)
    # mismatch-only search: the intervals of distinct equal-length strings are disjoint, so
    # their sizes add up to the number of text positions within Hamming distance 2
    c2, o2, p2 = fm.fm_inexact(h, sc, so, 2, 0, strands=2)
    o2 = o2.cpu().numpy()
    p2 = _u32(p2).astype(np.int64)
    jobs = []
    for r in range(len(sample)):
        for s in range(2):
            W = sample.read(r) if s == 0 else synth.revcomp(sample.read(r))
            jobs.append((2 * r + s, W))
    with ThreadPoolExecutor(max_workers=oracle.default_threads()) as ex:
        want = list(ex.map(lambda j: oracle.hamming_count(R, j[1], 2), jobs))
    for (q, _), w in zip(jobs, want):
        seg = p2[o2[q]:o2[q + 1]]
        assert int((seg[:, 1] - seg[:, 0] + 1).sum()) == w
    h.close()


def test_inexact_64mbp_sample_matches_oracle(fm):
    """Config 3: 64 Mbp repeat reference, 100 bp reads (0.5% substitutions, 5% random, both
    strands), z=2 mismatches only; a 20,000-read sample against the oracle's full index."""
    R = synth.repeat_text(1811061273, 64_000_000)
    reads = synth.sample_reads(1811061273, R, 20_000, 100, 100, sub_rate=0.005,
                               both_strands=True, random_frac=0.05)
    h = fm.fm_build(R, interval=64)
    fm.fm_set_tuning(h, pair_steps=2)   # node totals as the oracle counts them
    codes, offs = fm.to_device_reads(reads)
    stats = torch.zeros(4, dtype=torch.int64, device="cuda")
    counts, offsets, pairs = fm.fm_inexact(h, codes, offs, 2, 0, strands=2, stats=stats)
    want = oracle.Index(R, "sais").inexact(reads.codes, reads.offs, 2, 0, strands=2)
    assert np.array_equal(_u32(counts), want["counts"])
    assert np.array_equal(offsets.cpu().numpy().astype(np.uint64), want["offsets"])
    assert np.array_equal(_u32(pairs), want["pairs"])
    assert stats.cpu().numpy()[0] == want["nodes"].sum()
    h.close()


def test_config1_occ8_million(fm):
    """Config 1: 1 Mbp uniform reference, 10^6 fm_occ8 calls with k <= l."""
    R = synth.uniform_text(1811061271, 1_000_000)
    h = fm.fm_build(R)
    k, l = synth.occ_queries_uniform(1811061271, R.size, 1_000_000)
    got = _u32(fm.fm_occ8(h, torch.from_numpy(k.view(np.int32)).cuda(),
                          torch.from_numpy(l.view(np.int32)).cuda()))
    assert np.array_equal(got, oracle.Index(R, "sais").occ8(k, l))
    h.close()
