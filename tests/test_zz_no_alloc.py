"""fm_inexact_noalloc: the inexact search for callers that cannot let the library allocate
device memory (a serving process whose memory manager reserved the GPU up front, or a loop
that must not pay for cudaMalloc/cudaFree).  Its scratch lives in a fixed static device array
inside the library; its results must equal fm_inexact's exactly (integer intervals, tolerance
0), call after call, since the array keeps the previous call's contents.

This file sorts last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

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


def test_noalloc_matches_fm_inexact_twice(fm):
    R = synth.repeat_text(1811061279, 300_000, families=30, min_len=300, max_len=3000)
    h = fm.fm_build(R)
    batches = [synth.sample_reads(40 + b, R, 700, 30, 200, sub_rate=0.01, indel_rate=0.002,
                                  both_strands=True, random_frac=0.05) for b in range(2)]
    for z, gaps in ((2, 1), (1, 0)):
        for reads in batches:   # two different calls in a row share the static array
            codes, offs = fm.to_device_reads(reads)
            c0, o0, p0 = fm.fm_inexact(h, codes, offs, z, gaps, strands=2)
            for _ in range(2):
                c1, o1, p1, rc = fm.fm_inexact_noalloc(h, codes, offs, z, gaps, strands=2)
                assert rc == fm.FM_OK
                assert torch.equal(c1, c0)
                assert torch.equal(o1, o0)
                assert torch.equal(p1, p0)
    h.close()


def test_noalloc_limits_and_truncation(fm):
    R = synth.uniform_text(5, 100_000)
    h = fm.fm_build(R)
    # more queries than the static scratch holds: rejected before any device work
    big = synth.Reads(np.zeros(20_000, np.uint8), np.arange(20_001, dtype=np.uint32))
    codes, offs = fm.to_device_reads(big)
    with pytest.raises(fm.FmError) as ei:
        fm.fm_inexact_noalloc(h, codes, offs, 1, 0, strands=2)
    assert ei.value.code == fm.FM_EINVAL
    assert "static scratch" in str(ei.value)
    # a pairs buffer below the count: FM_ETRUNC with complete counts and offsets
    reads = synth.sample_reads(3, R, 200, 30, 60, sub_rate=0.02, both_strands=True)
    codes, offs = fm.to_device_reads(reads)
    c0, o0, p0 = fm.fm_inexact(h, codes, offs, 2, 0, strands=2)
    small = torch.empty((1, 2), dtype=torch.int32, device="cuda")
    c1, o1, _, rc = fm.fm_inexact_noalloc(h, codes, offs, 2, 0, strands=2, pairs=small)
    assert rc == fm.FM_ETRUNC
    assert torch.equal(c1, c0) and torch.equal(o1, o0)
    h.close()


def test_noalloc_raw_limit_then_exact(fm, orc):
    """Fewer queries than the static limit can still produce more intervals before
    deduplication than the array holds (262,144): short reads at z = 3 with 3 gaps on a
    uniform text.  The call must fail with FM_ENOMEM, grow nothing, and leave the array fit for
    the next call, whose results must equal the oracle's."""
    import oracle
    R = synth.uniform_text(1811061280, 1_000_000)
    h = fm.fm_build(R)
    many = synth.sample_reads(81, R, 300, 12, 12, sub_rate=0.0, both_strands=True)
    codes, offs = fm.to_device_reads(many)
    stats = torch.zeros(4, dtype=torch.int64, device="cuda")
    fm.fm_inexact(h, codes, offs, 3, 3, strands=2, stats=stats)
    raw = int(stats[2])
    assert 2 * len(many) < 32768 and raw > 262_144, raw   # the case this test is about
    with pytest.raises(fm.FmError) as ei:
        fm.fm_inexact_noalloc(h, codes, offs, 3, 3, strands=2)
    assert ei.value.code == fm.FM_ENOMEM
    assert "static" in str(ei.value)
    few = synth.sample_reads(82, R, 300, 20, 60, sub_rate=0.02, both_strands=True)
    codes, offs = fm.to_device_reads(few)
    c1, o1, p1, rc = fm.fm_inexact_noalloc(h, codes, offs, 2, 1, strands=2)
    assert rc == fm.FM_OK
    want = oracle.Index(R, "sais").inexact(few.codes, few.offs, 2, 1, strands=2)
    assert np.array_equal(c1.cpu().numpy().astype(np.uint32), want["counts"])
    assert np.array_equal(o1.cpu().numpy().astype(np.uint64), want["offsets"])
    assert np.array_equal(p1.cpu().numpy().view(np.uint32), want["pairs"])
    h.close()


def test_noalloc_results_are_not_fetchable(fm):
    """fm_inexact_fetch serves fm_inexact's results only.  After a truncated
    fm_inexact_noalloc call it must fail with FM_EINVAL rather than hand out the intervals of
    the earlier fm_inexact call, which are unrelated to this batch."""
    R = synth.repeat_text(1811061281, 200_000, families=20, min_len=300, max_len=2000)
    h = fm.fm_build(R)
    a = synth.sample_reads(83, R, 200, 30, 90, sub_rate=0.01, both_strands=True)
    b = synth.sample_reads(84, R, 200, 30, 90, sub_rate=0.03, both_strands=True)
    ca, oa = fm.to_device_reads(a)
    fm.fm_inexact(h, ca, oa, 2, 1, strands=2)
    cb, ob = fm.to_device_reads(b)
    small = torch.empty((1, 2), dtype=torch.int32, device="cuda")
    _, o1, _, rc = fm.fm_inexact_noalloc(h, cb, ob, 2, 1, strands=2, pairs=small)
    assert rc == fm.FM_ETRUNC and int(o1[-1]) > 1
    with pytest.raises(fm.FmError) as ei:
        fm.fm_inexact_fetch(h, torch.empty((int(o1[-1]), 2), dtype=torch.int32, device="cuda"))
    assert ei.value.code == fm.FM_EINVAL
    h.close()
