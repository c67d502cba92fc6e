"""The persistent search replayed as a CUDA graph gives the same interval sets as the eager
launches and the oracle, call after call (integer results, tolerance 0)."""
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


@pytest.fixture(scope="module")
def case():
    R = synth.repeat_text(1811061280, 300_000, families=30, min_len=300, max_len=3000)
    reads = synth.sample_reads(81, R, 600, 40, 200, sub_rate=0.01, indel_rate=0.002,
                               both_strands=True, random_frac=0.05)
    ix = oracle.Index(R, "sais")
    want = ix.inexact(reads.codes, reads.offs, 2, 1, strands=2, canonical=True)
    plain = ix.inexact(reads.codes, reads.offs, 2, 1, strands=2)
    for key in ("counts", "offsets", "pairs"):
        assert np.array_equal(want[key], plain[key])
    return R, reads, want


def _bufs(nq, cap):
    return (torch.empty(nq, dtype=torch.int32, device="cuda"),
            torch.empty(nq + 1, dtype=torch.int64, device="cuda"),
            torch.empty((cap, 2), dtype=torch.int32, device="cuda"))


def _check(want, counts, offsets, pairs):
    assert np.array_equal(counts.cpu().numpy().view(np.uint32), want["counts"])
    assert np.array_equal(offsets.cpu().numpy().astype(np.uint64), want["offsets"])
    assert np.array_equal(pairs.cpu().numpy().view(np.uint32), want["pairs"])


def test_graph_replay_matches_oracle(fm, case):
    R, reads, want = case
    h = fm.fm_build(R)
    codes, offs = fm.to_device_reads(reads)
    nq = 2 * len(reads)
    counts, offsets, pairs = _bufs(nq, 4 * nq + 1024)
    stats = torch.zeros(4, dtype=torch.int64, device="cuda")
    # node and block totals as the oracle counts them: no tables, one symbol per exact step
    fm.fm_set_tuning(h, kmer_depth=fm.KMER_OFF, pair_steps=2)
    kinds = []
    for _ in range(4):
        prof = fm.fm_profile()
        c, o, p = fm.fm_inexact(h, codes, offs, 2, 1, strands=2, stats=stats, counts=counts,
                                offsets=offsets, pairs=pairs, profile=prof)
        _check(want, c, o, p)
        kinds.append(prof.graph)
        assert prof.launches >= 10
    assert kinds[0] == 0 and all(k == 1 for k in kinds[1:])
    st = stats.cpu().numpy()
    assert st[0] == 4 * want["nodes"].sum()
    assert st[1] == 4 * want["blocks"].sum()
    # interval tables on: a new graph, results and nodes unchanged
    fm.fm_set_tuning(h, kmer_depth=fm.KMER_AUTO)
    stats.zero_()
    for _ in range(2):
        c, o, p = fm.fm_inexact(h, codes, offs, 2, 1, strands=2, stats=stats, counts=counts,
                                offsets=offsets, pairs=pairs)
        _check(want, c, o, p)
    assert stats.cpu().numpy()[0] == 2 * want["nodes"].sum()
    # two-symbol exact steps: a new graph, the same results
    fm.fm_set_tuning(h, pair_steps=1)
    for _ in range(2):
        c, o, p = fm.fm_inexact(h, codes, offs, 2, 1, strands=2, counts=counts,
                                offsets=offsets, pairs=pairs)
        _check(want, c, o, p)
    # new output buffers: a new graph is captured, results unchanged
    counts2, offsets2, pairs2 = _bufs(nq, 4 * nq + 1024)
    prof = fm.fm_profile()
    c, o, p = fm.fm_inexact(h, codes, offs, 2, 1, strands=2, counts=counts2, offsets=offsets2,
                            pairs=pairs2, profile=prof)
    assert prof.graph == 1
    _check(want, c, o, p)
    h.close()


def test_graph_off_and_truncation(fm, case):
    R, reads, want = case
    h = fm.fm_build(R)
    codes, offs = fm.to_device_reads(reads)
    nq = 2 * len(reads)
    fm.fm_set_tuning(h, graphs=2)
    assert fm.fm_get_tuning(h)["graphs"] == 2
    counts, offsets, pairs = _bufs(nq, 4 * nq + 1024)
    for _ in range(2):
        prof = fm.fm_profile()
        c, o, p = fm.fm_inexact(h, codes, offs, 2, 1, strands=2, counts=counts,
                                offsets=offsets, pairs=pairs, profile=prof)
        assert prof.graph == 0
        _check(want, c, o, p)
    fm.fm_set_tuning(h, graphs=1)
    # a pairs buffer below the total under replay: counts and offsets complete, then fetched
    small = torch.empty((2, 2), dtype=torch.int32, device="cuda")
    for _ in range(3):
        c, o, p = fm.fm_inexact(h, codes, offs, 2, 1, strands=2, counts=counts,
                                offsets=offsets, pairs=small)
        _check(want, c, o, p)
    h.close()


def test_rejected_tuning_changes_nothing(fm):
    h = fm.fm_build(synth.uniform_text(5, 5000))
    before = fm.fm_get_tuning(h)
    for bad in ({"warps_per_block": 4, "graphs": 3}, {"chunk": 8, "occ_per_thread": 3},
                {"blocks_per_sm": 2, "l2_fetch_bytes": 48}, {"warps_per_block": 9},
                {"chunk": 4, "kmer_depth": 16}, {"canonical": 2, "kmer_depth": 0x80}):
        with pytest.raises(fm.FmError) as ei:
            fm.fm_set_tuning(h, **bad)
        assert ei.value.code == fm.FM_EINVAL
        assert fm.fm_get_tuning(h) == before
    h.close()
