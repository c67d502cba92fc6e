"""Oracle parity at the shapes of the benchmark's configurations, element by element.

The oracle's SA-IS takes over ten minutes at 2 Gbp, so the headline read model (50-250 bp,
1% substitutions + 0.05% single-base indels, both strands, z = 2 with at most one gap) is
checked against Listing 2 on a 256 Mbp reference from the same repeat generator, with the code
paths of the 2 Gbp index forced on: interval tables of depth 14 (the automatic depth at
2 Gbp; at 256 Mbp it would be 12), pair steps, and the scheduler point the autotuner picks at
full size (I = 64, 8 warps per CTA, as many CTAs per SM as fit, chunk 8).  Every other point
the autotuner can return is run on a smaller reference.  The occ8 micro-benchmark's query mix
is checked value by value against the oracle's sorted sweep over its own BWT at 256 Mbp for
I = 64, 128 and 256, and the 64 Mbp mismatch-only configuration on all of its 10^6 reads.

All results are integers: the tolerance is 0.  The oracle's indexes are built on host threads
at the start of the module (ctypes releases the GIL), so their suffix sorts overlap the GPU work.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_1811_06127_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SEED_OCC, SEED_SEARCH, SEED_CFG3 = 1811061272, 1811061274, 1811061273
N_HEAD = 256_000_000        # the headline read model's reference here
N_OCC = 256_000_000         # the occ8 query mix's reference here
N_CFG3 = 64_000_000


@pytest.fixture(scope="module")
def fm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1811_06127_gb300 import _build, fmocc
    _build.build()
    fmocc.load_library()
    return fmocc


@pytest.fixture(scope="module")
def texts():
    return {"head": synth.repeat_text(SEED_SEARCH, N_HEAD),
            "occ": synth.gc_text(SEED_OCC, N_OCC, 0.41),
            "cfg3": synth.repeat_text(SEED_CFG3, N_CFG3)}


@pytest.fixture(scope="module")
def oracle_ix(texts):
    """Futures of the oracle's indexes, started together on host threads."""
    oracle.load()
    ex = ThreadPoolExecutor(max_workers=3)
    fut = {k: ex.submit(oracle.Index, R, "sais") for k, R in texts.items()}
    yield fut
    ex.shutdown(wait=True)


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _same(got, want, what):
    c, o, p = got[:3]
    assert np.array_equal(_u32(c), want["counts"]), f"{what}: counts differ"
    assert np.array_equal(o.cpu().numpy().astype(np.uint64), want["offsets"]), f"{what}: offsets"
    assert np.array_equal(_u32(p), want["pairs"]), f"{what}: intervals differ"
    if len(got) > 3:
        assert np.array_equal(got[3].cpu().numpy(), want["costs"]), f"{what}: costs differ"


def test_headline_read_model_256mbp_vs_listing2(fm, texts, oracle_ix):
    """10^5 reads of the headline read model (2 x 10^5 queries), z = 2 with one gap, at the
    tuned scheduler point with depth-14 tables and pair steps: intervals (graph replay and the
    eager path) and per-interval costs against every call of the oracle's Listing 2."""
    R = texts["head"]
    reads = synth.sample_reads(SEED_SEARCH + 17, R, 100_000, 50, 250, sub_rate=0.01,
                               indel_rate=0.0005, both_strands=True)
    h = fm.fm_build(R, interval=64)
    fm.fm_set_tuning(h, warps_per_block=8, blocks_per_sm=32, chunk=8, kmer_depth=14,
                     pair_steps=1, canonical=1, graphs=1)
    t = fm.fm_get_tuning(h)
    assert (t["kmer_depth"], t["pair_steps"], t["chunk"]) == (14, 1, 8)
    codes, offs = fm.to_device_reads(reads)
    stats = torch.zeros(4, dtype=torch.int64, device="cuda")
    first = fm.fm_inexact(h, codes, offs, 2, 1, strands=2)               # eager, sizes scratch
    prof = fm.fm_profile()
    replay = fm.fm_inexact(h, codes, offs, 2, 1, strands=2, stats=stats, profile=prof)
    assert prof.graph == 1                                               # the captured graph ran
    assert int(stats[3]) > 0 and int(stats[1]) > 0    # table/pair sectors and blocks were read
    with_costs = fm.fm_inexact(h, codes, offs, 2, 1, strands=2, costs=True)
    h.close()
    want = oracle_ix["head"].result().inexact(reads.codes, reads.offs, 2, 1, strands=2)
    assert int(want["offsets"][-1]) > 100_000
    _same(first, want, "eager")
    _same(replay, want, "graph replay")
    _same(with_costs, want, "with costs")


def test_every_tuner_point_vs_listing2(fm):
    """Every configuration the autotuner can return (checkpoint interval, warps per CTA, CTAs
    per SM, queue chunk, interval-table depth, pair steps) on the headline read model over an
    8 Mbp repeat reference: each equal to Listing 2 (graph replay)."""
    from paper_1811_06127_gb300 import autotune
    R = synth.repeat_text(SEED_SEARCH + 3, 8_000_000, families=100, min_len=300, max_len=6000)
    reads = synth.sample_reads(SEED_SEARCH + 19, R, 40_000, 50, 250, sub_rate=0.01,
                               indel_rate=0.0005, both_strands=True)
    want = oracle.Index(R, "sais").inexact(reads.codes, reads.offs, 2, 1, strands=2)
    codes, offs = fm.to_device_reads(reads)
    pts = autotune.points(R.size)
    assert len(pts) == 324
    for I in sorted({p["interval"] for p in pts}):
        h = fm.fm_build(R, interval=I)
        for p in (q for q in pts if q["interval"] == I):
            fm.fm_set_tuning(h, warps_per_block=p["warps_per_block"],
                             blocks_per_sm=p["blocks_per_sm"], chunk=p["chunk"],
                             kmer_depth=p["kmer_depth"], pair_steps=p["pair_steps"])
            for _ in range(2):   # the first call of a configuration may run eagerly
                _same(fm.fm_inexact(h, codes, offs, 2, 1, strands=2), want, str(p))
        h.close()


@pytest.mark.parametrize("gaps", [1, 2, 4])
def test_z4_canonical_vs_literal_listing2_run_poor(fm, gaps):
    """z = 4 on a text without runs of one symbol, where every call of Listing 2 is still
    affordable: the default search (canonical enumeration, tables, pair steps) against the
    oracle's literal recursion, intervals and costs."""
    rng = np.random.default_rng(1811061290)
    R = (np.cumsum(rng.integers(1, 4, 100_000)) % 4).astype(np.uint8)   # R[i] != R[i-1]
    reads = synth.sample_reads(91, R, 500, 20, 45, sub_rate=0.03, indel_rate=0.01,
                               both_strands=True)
    want = oracle.Index(R, "sais").inexact(reads.codes, reads.offs, 4, gaps, strands=2)
    h = fm.fm_build(R)
    codes, offs = fm.to_device_reads(reads)
    _same(fm.fm_inexact(h, codes, offs, 4, gaps, strands=2), want, "persistent")
    _same(fm.fm_inexact(h, codes, offs, 4, gaps, strands=2, costs=True), want, "costs")
    _same(fm.fm_inexact(h, codes, offs, 4, gaps, strands=2, kernel="plain"), want, "plain")
    h.close()


def test_occ8_query_mix_256mbp_all_values(fm, texts, oracle_ix):
    """2^24 queries of the occ8 micro-benchmark's mix (half inside one checkpoint block, half
    at a geometric gap of mean 1000) on a 41% GC reference, for I = 64, 128 and 256: all
    2^27 values against the oracle's sorted sweep over its own BWT (Occ by definition)."""
    R = texts["occ"]
    ix = oracle_ix["occ"].result()
    for I in (64, 128, 256):
        k, l = synth.occ_queries_mixed(SEED_OCC, R.size, 1 << 24, I)
        same = (k.astype(np.int64) // I) == ((l.astype(np.int64) + 1) // I)
        assert 0.45 < same.mean() < 0.56
        h = fm.fm_build(R, interval=I, forward_only=True)
        got = _u32(fm.fm_occ8(h, torch.from_numpy(k.view(np.int32)).cuda(),
                              torch.from_numpy(l.view(np.int32)).cuda()))
        h.close()
        want = ix.occ8_sweep(k, l)
        assert np.array_equal(got, want), f"I={I}"


def test_cfg3_all_reads_vs_listing2(fm, texts, oracle_ix):
    """The 64 Mbp configuration in full: 10^6 reads of 100 bp (0.5% substitutions, 5% random),
    both strands, z = 2 mismatches only: every query's interval set against Listing 2."""
    R = texts["cfg3"]
    reads = synth.sample_reads(SEED_CFG3, R, 1_000_000, 100, 100, sub_rate=0.005,
                               both_strands=True, random_frac=0.05)
    h = fm.fm_build(R, interval=64)
    codes, offs = fm.to_device_reads(reads)
    got = fm.fm_inexact(h, codes, offs, 2, 0, strands=2)
    h.close()
    want = oracle_ix["cfg3"].result().inexact(reads.codes, reads.offs, 2, 0, strands=2)
    _same(got, want, "cfg3")
