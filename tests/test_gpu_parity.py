"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

Every result here is integer and must be bit-exact (tolerance 0).  Sizes span several
checkpoint blocks and leave ragged tails; the full-size configurations have their own file.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_1811_06127_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1811_06127_gb300 import _build, fmocc
    _build.build()
    fmocc.load_library()
    return fmocc


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def test_fig1_acag(fm):
    h = fm.fm_build("ACAG")
    inf = fm.fm_info(h)
    assert inf["C"] == [0, 2, 3, 4, 4]
    assert inf["dollar_row"] == 1
    assert "".join("ACGT$"[c] for c in fm.fm_get_bwt(h)) == "G$CAA"
    k = torch.tensor([0, 1, 2, 3, 4, 5], dtype=torch.int32, device="cuda")
    l = torch.tensor([0, 1, 2, 3, 4, 4], dtype=torch.int32, device="cuda")
    out = _u32(fm.fm_occ8(h, k, l))
    fig1 = np.array([[0, 0, 1, 0], [0, 0, 1, 0], [0, 1, 1, 0], [1, 1, 1, 0], [2, 1, 1, 0]])
    for q in range(6):
        kk, ll = int(k[q]), int(l[q])
        want_k = fig1[kk - 1] if kk >= 1 else np.zeros(4)
        assert out[q, :4].tolist() == want_k.tolist()
        assert out[q, 4:].tolist() == fig1[ll].tolist()
    for w, exp in (("A", (1, 2)), ("G", (4, 4)), ("CA", (3, 3)), ("AG", (2, 2)), ("T", (5, 4))):
        codes = torch.from_numpy(synth.from_ascii(w)).cuda()
        offs = torch.tensor([0, len(w)], dtype=torch.int32, device="cuda")
        kk, ll = fm.fm_exact(h, codes, offs)
        assert (int(kk[0]), int(ll[0])) == exp
    h.close()


TEXTS = [("uniform", 1), ("uniform", 2), ("uniform", 31), ("uniform", 63), ("uniform", 64),
         ("uniform", 65), ("uniform", 127), ("uniform", 128), ("uniform", 255), ("uniform", 256),
         ("uniform", 257), ("uniform", 1000), ("periodic", 3000), ("homopolymer", 777),
         ("repeat", 100_000), ("uniform", 1_000_000)]


def _text(kind, n):
    if kind == "uniform":
        return synth.uniform_text(1000 + n, n)
    if kind == "periodic":
        return synth.from_ascii(("ACGTTGCA" * (n // 8 + 1))[:n])
    if kind == "homopolymer":
        return synth.from_ascii(("A" * 300 + "C" + "A" * 300 + "GT" * 100)[:n])
    return synth.repeat_text(77, n, families=20, min_len=300, max_len=3000)


@pytest.mark.parametrize("interval", [32, 64, 128, 256])
@pytest.mark.parametrize("kind,n", TEXTS)
def test_bwt_c_dollar(fm, kind, n, interval):
    R = _text(kind, n)
    h = fm.fm_build(R, interval=interval)
    ix = oracle.Index(R, "sais")
    inf = fm.fm_info(h)
    assert inf["C"] == ix.C.tolist()
    assert inf["dollar_row"] == ix.dollar_row
    assert np.array_equal(fm.fm_get_bwt(h), ix.bwt)
    # the reverse index is the index of reverse(R)
    ixr = oracle.Index(R[::-1].copy(), "sais")
    assert inf["rev_dollar_row"] == ixr.dollar_row
    assert np.array_equal(fm.fm_get_bwt(h, rev=True), ixr.bwt)
    h.close()


def _edge_queries(n, I):
    ks, ls = [], []
    cand = sorted({0, 1, n, n + 1, *[j * I + d for j in range(0, (n + 1) // I + 1)
                                     for d in (-1, 0, 1, I - 1) if 0 <= j * I + d <= n + 1]})
    cand = cand[:400]
    for k in cand:
        for l in (k - 1, k, k + 1, n, 0):
            if 0 <= l <= n and 0 <= k <= n + 1:
                ks.append(k)
                ls.append(l)
    return np.array(ks, np.uint32), np.array(ls, np.uint32)


@pytest.mark.parametrize("interval", [32, 64, 128, 256])
@pytest.mark.parametrize("kind,n", [("uniform", 1), ("uniform", 65), ("uniform", 1000),
                                    ("repeat", 100_000), ("uniform", 1_000_000)])
def test_occ8_matches_oracle(fm, kind, n, interval):
    R = _text(kind, n)
    h = fm.fm_build(R, interval=interval, forward_only=True)
    ix = oracle.Index(R, "sais")
    k1, l1 = synth.occ_queries_uniform(5, n, 200_000)
    k2, l2 = synth.occ_queries_mixed(6, n, 200_000, interval)
    k3, l3 = _edge_queries(n, interval)
    k = np.concatenate([k1, k2, k3])
    l = np.concatenate([l1, l2, l3])
    got = _u32(fm.fm_occ8(h, torch.from_numpy(k.view(np.int32)).cuda(),
                          torch.from_numpy(l.view(np.int32)).cuda()))
    want = ix.occ8(k, l)
    assert np.array_equal(got, want)
    h.close()


def test_occ8_domain_error_and_empty(fm):
    R = _text("uniform", 1000)
    h = fm.fm_build(R)
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    assert fm.fm_occ8(h, e, e).shape == (0, 8)
    k = torch.tensor([0, 1002], dtype=torch.int32, device="cuda")
    l = torch.tensor([5, 5], dtype=torch.int32, device="cuda")
    with pytest.raises(fm.FmError) as ei:
        fm.fm_occ8(h, k, l)
    assert ei.value.code == fm.FM_EINVAL
    # the handle stays usable
    k = torch.tensor([0, 1001], dtype=torch.int32, device="cuda")
    out = _u32(fm.fm_occ8(h, k, l))
    assert np.array_equal(out, oracle.Index(R).occ8(np.array([0, 1001], np.uint32),
                                                    np.array([5, 5], np.uint32)))
    h.close()


@pytest.mark.parametrize("interval", [32, 64, 128, 256])
def test_exact_matches_oracle(fm, interval):
    R = synth.uniform_text(1811061271, 1_000_000)
    h = fm.fm_build(R, interval=interval)
    ix = oracle.Index(R, "sais")
    reads = synth.exact_reads(1811061271, R, 10_000, 32)
    ragged = synth.sample_reads(3, R, 3000, 0, 200, sub_rate=0.01, random_frac=0.2)
    for rd in (reads, ragged):
        codes, offs = fm.to_device_reads(rd)
        k, l = fm.fm_exact(h, codes, offs)
        kw, lw = ix.exact(rd.codes, rd.offs)
        assert np.array_equal(_u32(k), kw)
        assert np.array_equal(_u32(l), lw)
    h.close()


@pytest.mark.parametrize("n", [1, 2, 3, 30, 31, 32, 62, 63, 64, 65, 127, 128, 4095, 16382,
                               16383, 16384, 32767, 32768, 70000])
def test_exact_pair_steps_edge_sizes(fm, n):
    """Listing 1 two symbols per step over the pair table on texts whose row count (n + 1)
    falls on and around pair-record (32 rows) and count-run (512 records, 16384 rows)
    boundaries, and around the checkpoint intervals: every string of length <= 5
    and random reads, occurring or not (insertion points included), with and without pair
    steps and tables, equal the oracle's."""
    R = synth.uniform_text(900 + n, n) if n > 3 else np.array([0, 0, 1][:n], np.uint8)
    ix = oracle.Index(R, "sais" if n > 64 else "naive")
    words = [np.array([(c >> (2 * t)) & 3 for t in range(j)], np.uint8)
             for j in range(0, 6) for c in range(4 ** j)]
    rng = np.random.default_rng(n)
    for _ in range(300):
        m = int(rng.integers(1, 40))
        if n > m and rng.random() < 0.7:
            p = int(rng.integers(0, n - m + 1))
            words.append(R[p:p + m].copy())
        else:
            words.append(rng.integers(0, 4, m).astype(np.uint8))
    codes = np.concatenate(words).astype(np.uint8)
    offs = np.concatenate([[0], np.cumsum([w.size for w in words])]).astype(np.uint32)
    rd = synth.Reads(codes, offs)
    kw, lw = ix.exact(codes, offs)
    h = fm.fm_build(R)
    c, o = fm.to_device_reads(rd)
    for pairs, kmer in ((1, fm.KMER_AUTO), (1, fm.KMER_OFF), (2, fm.KMER_OFF)):
        fm.fm_set_tuning(h, pair_steps=pairs, kmer_depth=kmer)
        k, l = fm.fm_exact(h, c, o)
        assert np.array_equal(_u32(k), kw), (pairs, kmer)
        assert np.array_equal(_u32(l), lw), (pairs, kmer)
    h.close()


@pytest.mark.parametrize("depth", [1, 2, 6, 9, 11])
def test_exact_interval_tables(fm, depth):
    """Listing 1 started from the interval tables: every string of length <= 6 (so every table
    entry of levels <= 6, occurring or not: the empty ones hold the insertion point), and
    ragged reads shorter and longer than the table depth, equal the oracle's search."""
    R = synth.repeat_text(41, 200_000, families=20, min_len=300, max_len=3000)
    h = fm.fm_build(R)
    fm.fm_set_tuning(h, kmer_depth=depth)
    assert fm.fm_get_tuning(h)["kmer_depth"] == depth
    ix = oracle.Index(R, "sais")
    words = [np.array([(c >> (2 * t)) & 3 for t in range(j)], np.uint8)
             for j in range(0, 7) for c in range(4 ** j)]
    codes = np.concatenate(words).astype(np.uint8)
    offs = np.concatenate([[0], np.cumsum([w.size for w in words])]).astype(np.uint32)
    every = synth.Reads(codes, offs)
    ragged = synth.sample_reads(43, R, 2000, 0, 40, sub_rate=0.05, random_frac=0.3)
    for rd in (every, ragged):
        c, o = fm.to_device_reads(rd)
        k, l = fm.fm_exact(h, c, o)
        kw, lw = ix.exact(rd.codes, rd.offs)
        assert np.array_equal(_u32(k), kw)
        assert np.array_equal(_u32(l), lw)
    h.close()


def test_exact_bad_code(fm):
    h = fm.fm_build(_text("uniform", 1000))
    codes = torch.tensor([0, 1, 7, 2], dtype=torch.uint8, device="cuda")
    offs = torch.tensor([0, 2, 4], dtype=torch.int32, device="cuda")
    with pytest.raises(fm.FmError):
        fm.fm_exact(h, codes, offs)
    h.close()


@pytest.mark.parametrize("interval", [32, 64, 256])
def test_dcalc_matches_oracle(fm, interval):
    R = synth.repeat_text(5, 300_000, families=30, min_len=300, max_len=3000)
    h = fm.fm_build(R, interval=interval)
    ix = oracle.Index(R, "sais")
    reads = synth.sample_reads(9, R, 1500, 1, 255, sub_rate=0.03, indel_rate=0.01,
                               both_strands=True, random_frac=0.1)
    codes, offs = fm.to_device_reads(reads)
    want = [(ix.dcalc(reads.read(r)), ix.dcalc(synth.revcomp(reads.read(r))))
            for r in range(len(reads))]
    # without interval or pair tables, then with tables of reverse(R) at several depths (a
    # search builds them; the D bound then takes each window's first symbols from them and its
    # further symbols two at a time from the pair table of reverse(R)), then pairs without
    # interval tables, then interval tables without pair steps
    ek, eo = fm.to_device_reads(reads.subset(np.arange(4)))
    for depth in (None, 1, 2, 7, fm.KMER_AUTO, fm.KMER_OFF, "no pairs"):
        if depth == "no pairs":
            fm.fm_set_tuning(h, kmer_depth=fm.KMER_AUTO, pair_steps=2)
            fm.fm_exact(h, ek, eo)
        elif depth is not None:
            fm.fm_set_tuning(h, kmer_depth=depth)
            fm.fm_exact(h, ek, eo)
        D = fm.fm_dcalc(h, codes, offs, strands=2).cpu().numpy()
        for r in range(len(reads)):
            m = int(reads.offs[r + 1] - reads.offs[r])
            s = 2 * int(reads.offs[r])
            assert np.array_equal(D[s:s + m], want[r][0]), (depth, r)
            assert np.array_equal(D[s + m:s + 2 * m], want[r][1]), (depth, r)
    h.close()


def _inexact_case(fm, R, reads, z, gaps, interval, kernels=("plain", "persistent"),
                  modes=("canonical", "listing"), kmers=(0xFE, 0xFF)):   # tables auto, off
    """Both kernels, with the canonical enumeration (default) and with every call of Listing 2,
    with and without interval tables, one symbol per exact step: result sets equal the
    oracle's Listing 2 sets, node counts equal the oracle's for the same enumeration, and so do
    block counts without tables (with tables, nodes shorter than the table depth read no
    checkpoint block).  Then with two-symbol exact steps (the default): same sets, no more
    nodes than the oracle's."""
    h = fm.fm_build(R, interval=interval)
    ix = oracle.Index(R, "sais")
    want_c = ix.inexact(reads.codes, reads.offs, z, gaps, strands=2, interval=interval,
                        canonical=True)
    # the two enumerations report the same sets (pinned on the CPU); Listing 2's own run is
    # skipped where its repeated subtrees make it too slow
    want = ix.inexact(reads.codes, reads.offs, z, gaps, strands=2, interval=interval) \
        if "listing" in modes else want_c
    codes, offs = fm.to_device_reads(reads)
    for mode in modes:
        for kmer in kmers:
            fm.fm_set_tuning(h, canonical=1 if mode == "canonical" else 2, kmer_depth=kmer,
                             pair_steps=2)
            ref = want_c if mode == "canonical" else want
            for kern in kernels:
                stats = torch.zeros(4, dtype=torch.int64, device="cuda")
                counts, offsets, pairs = fm.fm_inexact(h, codes, offs, z, gaps, strands=2,
                                                       kernel=kern, stats=stats)
                tag = (kern, mode, kmer)
                assert np.array_equal(_u32(counts), want["counts"]), tag
                assert np.array_equal(offsets.cpu().numpy().astype(np.uint64),
                                      want["offsets"]), tag
                assert np.array_equal(_u32(pairs), want["pairs"]), tag
                st = stats.cpu().numpy()
                assert st[0] == ref["nodes"].sum(), tag
                if fm.fm_get_tuning(h)["kmer_depth"] == fm.KMER_OFF:
                    assert st[1] == ref["blocks"].sum(), tag
                    assert st[3] == 0, tag
                else:
                    assert st[1] <= ref["blocks"].sum(), tag
                    assert st[3] <= st[0], tag   # at most one table sector per node
    fm.fm_set_tuning(h, canonical=1, kmer_depth=fm.KMER_AUTO, pair_steps=1)
    for kern in kernels:
        stats = torch.zeros(4, dtype=torch.int64, device="cuda")
        counts, offsets, pairs = fm.fm_inexact(h, codes, offs, z, gaps, strands=2, kernel=kern,
                                               stats=stats)
        assert np.array_equal(_u32(counts), want["counts"]), (kern, "pairs")
        assert np.array_equal(offsets.cpu().numpy().astype(np.uint64), want["offsets"])
        assert np.array_equal(_u32(pairs), want["pairs"]), (kern, "pairs")
        assert stats.cpu().numpy()[0] <= want_c["nodes"].sum()
    h.close()


@pytest.mark.parametrize("z,gaps", [(0, 0), (1, 0), (2, 0), (1, 1), (2, 1), (2, 2), (3, 1)])
def test_inexact_matches_oracle(fm, z, gaps):
    R = synth.repeat_text(1811061273, 400_000, families=40, min_len=300, max_len=4000)
    n_reads = 400 if z < 3 else 80
    reads = synth.sample_reads(31 + z, R, n_reads, 20, 150, sub_rate=0.01, indel_rate=0.003,
                               both_strands=True, random_frac=0.05)
    _inexact_case(fm, R, reads, z, gaps, 64)


@pytest.mark.parametrize("z,gaps,n_reads,min_len,max_len", [(2, 1, 600, 30, 150), (5, 3, 40, 8, 20)])
def test_scheduler_options_same_results(fm, z, gaps, n_reads, min_len, max_len):
    """The persistent kernel's scheduler options change speed only: queries staged in shared
    memory or read through L1, the threshold for stepping second exact chains, and the pool
    level below which a warp takes queries, each equal to Listing 2.  The second case (short
    reads, z = 5 with 3 gaps) fills the pools past their size and spills."""
    R = synth.repeat_text(1811061282, 300_000, families=30, min_len=300, max_len=3000)
    reads = synth.sample_reads(33, R, n_reads, min_len, max_len, sub_rate=0.02,
                               indel_rate=0.005, both_strands=True, random_frac=0.05)
    want = oracle.Index(R, "sais").inexact(reads.codes, reads.offs, z, gaps, strands=2,
                                           canonical=True)
    h = fm.fm_build(R)
    codes, offs = fm.to_device_reads(reads)
    for stage in (1, 2):
        for chain2_min, refill in ((1, 32), (16, 32), (32, 96), (16, 288)):
            fm.fm_set_tuning(h, stage=stage, chain2_min=chain2_min, refill=refill, chunk=8)
            t = fm.fm_get_tuning(h)
            assert (t["stage"], t["chain2_min"], t["refill"]) == (stage, chain2_min, refill)
            for _ in range(2):   # eager, then graph replay
                c, o, p = fm.fm_inexact(h, codes, offs, z, gaps, strands=2)
                tag = (stage, chain2_min, refill)
                assert np.array_equal(_u32(c), want["counts"]), tag
                assert np.array_equal(o.cpu().numpy().astype(np.uint64), want["offsets"]), tag
                assert np.array_equal(_u32(p), want["pairs"]), tag
    h.close()


def _best_of(want):
    """Per query, the intervals of its minimum cost (from the oracle's sets and costs)."""
    counts, pairs, costs = [], [], []
    o = want["offsets"]
    for q in range(want["counts"].size):
        c = want["costs"][o[q]:o[q + 1]]
        keep = c == c.min() if c.size else np.zeros(0, bool)
        counts.append(int(keep.sum()))
        pairs.append(want["pairs"][o[q]:o[q + 1]][keep])
        costs.append(c[keep])
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint64)
    return (np.array(counts, np.uint32), offsets, np.concatenate(pairs).reshape(-1, 2),
            np.concatenate(costs))


@pytest.mark.parametrize("z,gaps", [(1, 0), (2, 0), (2, 1), (2, 2), (3, 1)])
def test_inexact_costs_and_best_hits(fm, z, gaps):
    """Per interval the fewest differences of its alignments, and best-hit reporting (only each
    query's minimum-cost intervals): equal to the oracle's, for both kernels, with the
    canonical enumeration and interval tables (the defaults) and without them."""
    R = synth.repeat_text(1811061273, 300_000, families=30, min_len=300, max_len=3000)
    reads = synth.sample_reads(61 + z, R, 300 if z < 3 else 80, 1, 150, sub_rate=0.015,
                               indel_rate=0.005, both_strands=True, random_frac=0.05)
    h = fm.fm_build(R)
    want = oracle.Index(R, "sais").inexact(reads.codes, reads.offs, z, gaps, strands=2)
    bc, bo, bp, bcost = _best_of(want)
    codes, offs = fm.to_device_reads(reads)
    for tuning in ({}, {"canonical": 2, "kmer_depth": fm.KMER_OFF}):
        if tuning:
            fm.fm_set_tuning(h, **tuning)
        for kern in ("plain", "persistent"):
            tag = (kern, tuning)
            c, o, p, cs = fm.fm_inexact(h, codes, offs, z, gaps, strands=2, kernel=kern,
                                        costs=True)
            assert np.array_equal(_u32(c), want["counts"]), tag
            assert np.array_equal(o.cpu().numpy().astype(np.uint64), want["offsets"]), tag
            assert np.array_equal(_u32(p), want["pairs"]), tag
            assert np.array_equal(cs.cpu().numpy(), want["costs"]), tag
            c, o, p, cs = fm.fm_inexact(h, codes, offs, z, gaps, strands=2, kernel=kern,
                                        costs=True, best=True)
            assert np.array_equal(_u32(c), bc), tag
            assert np.array_equal(o.cpu().numpy().astype(np.uint64), bo), tag
            assert np.array_equal(_u32(p), bp), tag
            assert np.array_equal(cs.cpu().numpy(), bcost), tag
            c, o, p = fm.fm_inexact(h, codes, offs, z, gaps, strands=2, kernel=kern, best=True)
            assert np.array_equal(_u32(p), bp), tag
    # too small a buffer: counts and offsets complete, the binding repeats the call
    c, o, p, cs = fm.fm_inexact(h, codes, offs, z, gaps, strands=2, costs=True, pair_capacity=2)
    assert np.array_equal(_u32(p), want["pairs"])
    assert np.array_equal(cs.cpu().numpy(), want["costs"])
    h.close()


def test_costs_rejected_where_unsupported(fm):
    R = synth.uniform_text(7, 2000)
    h = fm.fm_build(R)
    reads = synth.sample_reads(8, R, 10, 10, 20)
    codes, offs = fm.to_device_reads(reads)
    sp = fm.fm_search_params(1, 0, 1, fm.FM_KERNEL_PERSISTENT, None, None, None, 1, 0)
    counts = torch.empty(10, dtype=torch.int32, device="cuda")
    offsets = torch.empty(11, dtype=torch.int64, device="cuda")
    pairs = torch.empty((100, 2), dtype=torch.int32, device="cuda")
    need = fm.C.c_uint64(0)
    lib = fm.load_library()
    rc = lib.fm_inexact_noalloc(h.ptr, fm._dptr(codes, fm._U8, "r"), fm._dptr(offs, fm._U32, "o"),
                                10, fm.C.byref(sp), fm._dptr(counts, fm._U32, "c"),
                                fm._dptr(offsets, fm._U64, "f"), fm._dptr(pairs, fm._U32, "p"), 100,
                                fm.C.byref(need), None)
    assert rc == fm.FM_EINVAL
    sp.best, sp.indel_end_skip = 2, 0
    rc = lib.fm_inexact(h.ptr, fm._dptr(codes, fm._U8, "r"), fm._dptr(offs, fm._U32, "o"), 10,
                        fm.C.byref(sp), fm._dptr(counts, fm._U32, "c"),
                        fm._dptr(offsets, fm._U64, "f"), fm._dptr(pairs, fm._U32, "p"), 100,
                        fm.C.byref(need), None)
    assert rc == fm.FM_EINVAL
    # an end restriction above 255 (longer than any read can use) is rejected by both calls
    sp = fm.fm_search_params(1, 1, 1, fm.FM_KERNEL_PERSISTENT, None, None, None, 0, 256)
    for call in (lib.fm_inexact, lib.fm_inexact_noalloc):
        rc = call(h.ptr, fm._dptr(codes, fm._U8, "r"), fm._dptr(offs, fm._U32, "o"), 10,
                  fm.C.byref(sp), fm._dptr(counts, fm._U32, "c"), fm._dptr(offsets, fm._U64, "f"),
                  fm._dptr(pairs, fm._U32, "p"), 100, fm.C.byref(need), None)
        assert rc == fm.FM_EINVAL
    h.close()


@pytest.mark.parametrize("z,gaps,e", [(1, 1, 1), (2, 1, 5), (2, 2, 3), (3, 2, 12)])
def test_inexact_end_restriction(fm, z, gaps, e):
    """Indel columns only where at least e read symbols lie on each side (reads of 1..150
    symbols, so some fit no indel at all): sets, costs and best hits equal the oracle's, for
    both kernels, with interval tables and two-symbol steps (the defaults) and without; node
    counts equal those of the oracle's Listing 2 enumeration with one symbol per step (the
    canonical rewrites do not apply under the restriction).  A captured graph is not reused
    across restrictions, and the allocation-free call agrees."""
    R = synth.repeat_text(1811061273, 300_000, families=30, min_len=300, max_len=3000)
    reads = synth.sample_reads(71 + e, R, 300 if z < 3 else 60, 1, 150, sub_rate=0.01,
                               indel_rate=0.01, both_strands=True, random_frac=0.05)
    ix = oracle.Index(R, "sais")
    want = ix.inexact(reads.codes, reads.offs, z, gaps, strands=2, end_skip=e)
    full = ix.inexact(reads.codes, reads.offs, z, gaps, strands=2)
    assert want["counts"].sum() < full["counts"].sum()
    bc, bo, bp, bcost = _best_of(want)
    h = fm.fm_build(R)
    codes, offs = fm.to_device_reads(reads)

    def same(got, ref, tag):
        c, o, p = got[:3]
        assert np.array_equal(_u32(c), ref["counts"]), tag
        assert np.array_equal(o.cpu().numpy().astype(np.uint64), ref["offsets"]), tag
        assert np.array_equal(_u32(p), ref["pairs"]), tag

    for tuning in ({"pair_steps": 2}, {"pair_steps": 2, "kmer_depth": fm.KMER_OFF},
                   {"pair_steps": 1, "kmer_depth": fm.KMER_AUTO}):
        fm.fm_set_tuning(h, **tuning)
        for kern in ("plain", "persistent"):
            tag = (kern, tuning)
            stats = torch.zeros(4, dtype=torch.int64, device="cuda")
            got = fm.fm_inexact(h, codes, offs, z, gaps, strands=2, kernel=kern, costs=True,
                                end_skip=e, stats=stats)
            same(got, want, tag)
            assert np.array_equal(got[3].cpu().numpy(), want["costs"]), tag
            st = stats.cpu().numpy()
            if tuning["pair_steps"] == 2:
                assert st[0] == want["nodes"].sum(), tag
                if tuning.get("kmer_depth") == fm.KMER_OFF:
                    assert st[1] == want["blocks"].sum(), tag
            else:
                assert st[0] <= want["nodes"].sum(), tag
            c, o, p, cs = fm.fm_inexact(h, codes, offs, z, gaps, strands=2, kernel=kern,
                                        costs=True, best=True, end_skip=e)
            assert np.array_equal(_u32(c), bc) and np.array_equal(_u32(p), bp), tag
            assert np.array_equal(cs.cpu().numpy(), bcost), tag
    # the default search (graph replay): restricted, unrestricted, restricted again
    for ref, skip in ((want, e), (full, 0), (want, e)):
        same(fm.fm_inexact(h, codes, offs, z, gaps, strands=2, end_skip=skip), ref, ("graph", skip))
    # the allocation-free call on the first 100 reads (well inside its fixed scratch)
    sub_offs = reads.offs[:101].copy()
    sub_codes = reads.codes[:int(sub_offs[-1])].copy()
    want_sub = ix.inexact(sub_codes, sub_offs, z, gaps, strands=2, end_skip=e)
    room = torch.empty((int(want_sub["offsets"][-1]) + 16, 2), dtype=torch.int32, device="cuda")
    c, o, p, rc = fm.fm_inexact_noalloc(h, torch.from_numpy(sub_codes).cuda(),
                                        torch.from_numpy(sub_offs.view(np.int32)).cuda(), z,
                                        gaps, strands=2, end_skip=e, pairs=room)
    assert rc == fm.FM_OK
    same((c, o, p), want_sub, "noalloc")
    h.close()


@pytest.mark.parametrize("depth", [1, 3, 7, 10, 13, 14, 15])
def test_inexact_interval_table_depths(fm, depth):
    """Tables of every depth, up to deeper than the strings of the search's first steps on this
    text: same intervals and nodes as the oracle, and no more checkpoint blocks."""
    R = synth.repeat_text(47, 300_000, families=30, min_len=300, max_len=3000)
    reads = synth.sample_reads(48, R, 300, 1, 150, sub_rate=0.02, indel_rate=0.005,
                               both_strands=True, random_frac=0.05)
    _inexact_case(fm, R, reads, 2, 1, 64, modes=("canonical",), kmers=(depth,))


@pytest.mark.parametrize("z,gaps,n_reads,min_len,max_len", [(4, 2, 40, 6, 16), (5, 1, 40, 6, 16),
                                                             (6, 2, 40, 6, 16), (7, 7, 6, 4, 8)])
def test_inexact_high_differences(fm, z, gaps, n_reads, min_len, max_len):
    """z up to 7 with up to 7 indel columns (the limits of the node's 4-bit fields): both
    kernels against the oracle's canonical enumeration (the literal recursion explodes here),
    results and node counts with one symbol per exact step, results with the defaults.  The
    batches are small (millions of nodes per query at z = 7), and the pair buffer holds the
    whole result, so no call is repeated."""
    R = synth.repeat_text(81, 50_000, families=5, min_len=300, max_len=1500)
    ix = oracle.Index(R, "sais")
    reads = synth.sample_reads(82, R, n_reads, min_len, max_len, sub_rate=0.1, indel_rate=0.05,
                               both_strands=True, random_frac=0.1)
    want = ix.inexact(reads.codes, reads.offs, z, gaps, strands=2, canonical=True)
    cap = int(want["offsets"][-1]) + 64
    h = fm.fm_build(R)
    codes, offs = fm.to_device_reads(reads)
    for pairs in (2, 1):
        fm.fm_set_tuning(h, pair_steps=pairs)
        for kern in ("plain", "persistent"):
            stats = torch.zeros(4, dtype=torch.int64, device="cuda")
            c, o, p, cs = fm.fm_inexact(h, codes, offs, z, gaps, strands=2, kernel=kern,
                                        stats=stats, costs=True, pair_capacity=cap)
            tag = (kern, pairs)
            assert np.array_equal(_u32(c), want["counts"]), tag
            assert np.array_equal(o.cpu().numpy().astype(np.uint64), want["offsets"]), tag
            assert np.array_equal(_u32(p), want["pairs"]), tag
            assert np.array_equal(cs.cpu().numpy(), want["costs"]), tag
            if pairs == 2:
                assert stats.cpu().numpy()[0] == want["nodes"].sum(), tag
    h.close()


@pytest.mark.parametrize("interval", [32, 128, 256])
def test_inexact_intervals(fm, interval):
    R = synth.repeat_text(11, 200_000, families=20, min_len=300, max_len=3000)
    reads = synth.sample_reads(12, R, 300, 30, 100, sub_rate=0.02, both_strands=True)
    _inexact_case(fm, R, reads, 2, 1, interval)


def test_inexact_edge_reads(fm):
    """Length-0, length-1, length-255 reads, all-A reads and reads over a homopolymer text.
    (Over a homopolymer the literal recursion of Listing 2 reaches the same state by very many
    indel placements, so the gap budget is kept small for the long reads; the canonical
    enumeration takes each placement once and runs z = 3 with 3 gaps on the long reads.)"""
    R = _text("homopolymer", 777)
    short = [np.zeros(0, np.uint8), np.array([0], np.uint8), np.array([3], np.uint8),
             np.zeros(12, np.uint8), np.array([0, 1], np.uint8), synth.uniform_text(4, 20)]
    long_ = [np.zeros(40, np.uint8), synth.uniform_text(4, 255), np.zeros(255, np.uint8),
             np.concatenate([np.zeros(120, np.uint8), [1], np.zeros(100, np.uint8)]).astype(np.uint8)]

    def batch(parts):
        codes = np.concatenate(parts).astype(np.uint8)
        offs = np.concatenate([[0], np.cumsum([p.size for p in parts])]).astype(np.uint32)
        return synth.Reads(codes, offs)

    for z, g in ((0, 0), (2, 0), (2, 1)):
        _inexact_case(fm, R, batch(short + long_), z, g, 64)
    _inexact_case(fm, R, batch(short), 3, 3, 64)
    _inexact_case(fm, R, batch(short + long_), 3, 3, 64, modes=("canonical",))


def test_empty_batches(fm):
    """Zero reads, zero queries and zero rows: every call returns with empty outputs (offsets
    = [0], no intervals) and launches no search; a normal batch on the same handle afterwards
    still equals the oracle."""
    R = synth.uniform_text(17, 5000)
    h = fm.fm_build(R)
    codes = torch.empty(0, dtype=torch.uint8, device="cuda")
    offs = torch.zeros(1, dtype=torch.int32, device="cuda")
    k, l = fm.fm_exact(h, codes, offs)
    assert k.numel() == 0 and l.numel() == 0
    assert fm.fm_dcalc(h, codes, offs, strands=2).numel() == 0
    assert fm.fm_locate(h, torch.empty(0, dtype=torch.int32, device="cuda")).numel() == 0
    for kern in ("plain", "persistent"):
        c, o, p = fm.fm_inexact(h, codes, offs, 2, 1, strands=2, kernel=kern)
        assert c.numel() == 0 and o.tolist() == [0] and p.shape[0] == 0, kern
        c, o, p, cs = fm.fm_inexact(h, codes, offs, 2, 1, strands=2, kernel=kern, costs=True,
                                    best=True)
        assert c.numel() == 0 and o.tolist() == [0] and p.shape[0] == 0 and cs.numel() == 0
    c, o, p, rc = fm.fm_inexact_noalloc(h, codes, offs, 2, 1, strands=2)
    assert rc == fm.FM_OK and c.numel() == 0 and o.tolist() == [0] and p.shape[0] == 0
    reads = synth.sample_reads(18, R, 50, 10, 40, sub_rate=0.02, both_strands=True)
    want = oracle.Index(R, "sais").inexact(reads.codes, reads.offs, 2, 1, strands=2)
    c, o, p = fm.fm_inexact(h, *fm.to_device_reads(reads), 2, 1, strands=2)
    assert np.array_equal(_u32(c), want["counts"]) and np.array_equal(_u32(p), want["pairs"])
    h.close()


def test_canonical_knob(fm):
    h = fm.fm_build(_text("uniform", 5000))
    assert fm.fm_get_tuning(h)["canonical"] == 1
    fm.fm_set_tuning(h, canonical=2)
    assert fm.fm_get_tuning(h)["canonical"] == 2
    with pytest.raises(fm.FmError) as ei:
        fm.fm_set_tuning(h, canonical=3)
    assert ei.value.code == fm.FM_EINVAL
    assert fm.fm_get_tuning(h)["canonical"] == 2
    h.close()


def test_inexact_truncation_and_fetch(fm):
    R = synth.repeat_text(21, 100_000, families=10, min_len=300, max_len=2000)
    reads = synth.sample_reads(22, R, 200, 30, 80, sub_rate=0.02, both_strands=True)
    h = fm.fm_build(R)
    codes, offs = fm.to_device_reads(reads)
    c0, o0, p0 = fm.fm_inexact(h, codes, offs, 2, 1, strands=2)
    total = int(o0[-1])
    assert total > 10
    # a capacity below the total: FM_ETRUNC, then the binding fetches into a larger buffer
    c1, o1, p1 = fm.fm_inexact(h, codes, offs, 2, 1, strands=2, pair_capacity=3)
    assert torch.equal(c0, c1) and torch.equal(o0, o1) and torch.equal(p0, p1)
    h.close()


def test_inexact_too_long_read(fm):
    h = fm.fm_build(_text("uniform", 5000))
    codes = torch.zeros(300, dtype=torch.uint8, device="cuda")
    offs = torch.tensor([0, 300], dtype=torch.int32, device="cuda")
    with pytest.raises(fm.FmError) as ei:
        fm.fm_inexact(h, codes, offs, 1, 0)
    assert ei.value.code == fm.FM_EINVAL
    h.close()


@pytest.mark.parametrize("graphs", [1, 2])
def test_bad_read_reported_before_truncation(fm, graphs):
    """A batch holding a code above 3 fails with FM_EINVAL even when the pairs buffer is also
    too small: the truncation status would send the caller to fm_inexact_fetch, which must not
    hand out the intervals of a failed call.  Graph replay (1) and the eager path (2)."""
    R = synth.repeat_text(31, 100_000, families=10, min_len=300, max_len=2000)
    reads = synth.sample_reads(32, R, 300, 30, 80, sub_rate=0.02, both_strands=True)
    h = fm.fm_build(R)
    fm.fm_set_tuning(h, graphs=graphs)
    codes, offs = fm.to_device_reads(reads)
    c0, o0, p0 = fm.fm_inexact(h, codes, offs, 2, 1, strands=2)   # sizes the scratch
    assert int(o0[-1]) > 10
    pairs = torch.empty((2, 2), dtype=torch.int32, device="cuda")
    good = codes.clone()
    codes[int(offs[7]) + 3] = 5                                    # one bad symbol
    for _ in range(2):   # the second call of the same key replays the captured graph
        with pytest.raises(fm.FmError) as ei:
            fm.fm_inexact(h, codes, offs, 2, 1, strands=2, pairs=pairs)
        assert ei.value.code == fm.FM_EINVAL
        with pytest.raises(fm.FmError) as ei:   # nothing of the failed call can be fetched
            fm.fm_inexact_fetch(h, pairs)
        assert ei.value.code == fm.FM_EINVAL
    codes.copy_(good)
    c1, o1, p1 = fm.fm_inexact(h, codes, offs, 2, 1, strands=2)
    assert torch.equal(c0, c1) and torch.equal(o0, o1) and torch.equal(p0, p1)
    h.close()


def test_save_load_roundtrip(fm):
    R = synth.repeat_text(8, 50_000, families=5, min_len=300, max_len=1000)
    h = fm.fm_build(R, interval=128)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ix.fm")
        fm.fm_save(h, path)
        h2 = fm.fm_load(path)
        assert fm.fm_info(h2) == fm.fm_info(h)
        assert np.array_equal(fm.fm_get_bwt(h2), fm.fm_get_bwt(h))
        assert np.array_equal(fm.fm_get_bwt(h2, rev=True), fm.fm_get_bwt(h, rev=True))
        raw = bytearray(open(path, "rb").read())
        raw[200] ^= 1
        open(path, "wb").write(bytes(raw))
        with pytest.raises(fm.FmError) as ei:
            fm.fm_load(path)
        assert ei.value.code == fm.FM_EIO
        h2.close()
    h.close()


def test_invalid_reference(fm):
    with pytest.raises(fm.FmError) as ei:
        fm.fm_build("ACGTN")
    assert ei.value.code == fm.FM_EINVAL
    h = fm.fm_build("acgtACGT")
    assert fm.fm_info(h)["n"] == 8
    h.close()
