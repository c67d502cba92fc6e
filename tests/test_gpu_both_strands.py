"""Index of R . revcomp(R) (FM_BUILD_BOTH_STRANDS): one query finds both strands' occurrences.
Results equal the oracle's on the text T = R . revcomp(R); occurrence counts on T equal those of
W and revcomp(W) on R plus the occurrences that straddle the junction."""
import os

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


def _count(text, W):
    """Occurrences of W in text (sliding-window comparison)."""
    if W.size > text.size:
        return 0
    win = np.lib.stride_tricks.sliding_window_view(text, W.size)
    return int((win == W).all(axis=1).sum())


@pytest.fixture(scope="module")
def case():
    R = synth.repeat_text(71, 150_000, families=15, min_len=300, max_len=3000)
    T = np.concatenate([R, synth.revcomp(R)]).astype(np.uint8)
    reads = synth.sample_reads(72, R, 400, 12, 120, sub_rate=0.01, indel_rate=0.003,
                               both_strands=True, random_frac=0.05)
    return R, T, reads, oracle.Index(T, "sais")


def test_exact_and_counts(fm, case, tmp_path):
    R, T, reads, ixT = case
    h = fm.fm_build(R, both_strands=True)
    inf = fm.fm_info(h)
    assert inf["both_strands"] and inf["n"] == 2 * R.size
    codes, offs = fm.to_device_reads(reads)
    k, l = fm.fm_exact(h, codes, offs)
    kw, lw = ixT.exact(reads.codes, reads.offs)
    assert np.array_equal(_u32(k), kw) and np.array_equal(_u32(l), lw)
    n = R.size
    for r in range(0, len(reads), 7):
        W = reads.read(r)
        m = W.size
        on_t = max(int(lw[r]) - int(kw[r]) + 1, 0)
        straddle = _count(T[max(0, n - m + 1):n + m - 1], W)   # starts in (n - m, n)
        assert on_t == _count(R, W) + _count(R, synth.revcomp(W)) + straddle, r
    # save / load keeps the layout
    path = str(tmp_path / "both.fmi")
    fm.fm_save(h, path)
    h2 = fm.fm_load(path)
    assert fm.fm_info(h2)["both_strands"]
    k2, l2 = fm.fm_exact(h2, codes, offs)
    assert torch.equal(k, k2) and torch.equal(l, l2)
    h2.close()
    h.close()


@pytest.mark.parametrize("z,gaps", [(1, 1), (2, 1)])
def test_inexact_one_query_per_read(fm, case, z, gaps):
    R, T, reads, ixT = case
    h = fm.fm_build(R, both_strands=True)
    want = ixT.inexact(reads.codes, reads.offs, z, gaps, strands=1)
    codes, offs = fm.to_device_reads(reads)
    for kern in ("plain", "persistent"):
        c, o, p, cs = fm.fm_inexact(h, codes, offs, z, gaps, strands=1, kernel=kern, costs=True)
        assert np.array_equal(_u32(c), want["counts"]), kern
        assert np.array_equal(o.cpu().numpy().astype(np.uint64), want["offsets"]), kern
        assert np.array_equal(_u32(p), want["pairs"]), kern
        assert np.array_equal(cs.cpu().numpy(), want["costs"]), kern
    h.close()


def test_locate_positions_on_both_strands(fm, case):
    R, T, reads, ixT = case
    h = fm.fm_build(R, both_strands=True)
    sub = reads.subset(np.arange(60))
    codes, offs = fm.to_device_reads(sub)
    k, l = fm.fm_exact(h, codes, offs)
    k, l = _u32(k), _u32(l)
    rows = np.concatenate([np.arange(k[r], l[r] + 1) for r in range(len(sub))]).astype(np.int32)
    pos = fm.fm_locate(h, torch.from_numpy(rows).cuda()).cpu().numpy()
    assert np.array_equal(pos, ixT.sa[rows])
    at = 0
    for r in range(len(sub)):
        W = sub.read(r)
        for p in pos[at:at + max(int(l[r]) - int(k[r]) + 1, 0)]:
            assert np.array_equal(T[p:p + W.size], W)
        at += max(int(l[r]) - int(k[r]) + 1, 0)
    h.close()
