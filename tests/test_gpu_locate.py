"""Locate (Sec. 2, Eq. 4-5): the SA value of any row, recovered on the GPU from the SA kept at
rows that are multiples of 32 by Psi^-1 walks, equals the oracle's suffix array exactly."""
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


@pytest.mark.parametrize("interval", [32, 64, 128, 256])
@pytest.mark.parametrize("kind,n", [("uniform", 1), ("uniform", 31), ("uniform", 33),
                                    ("acag", 4), ("repeat", 200_000), ("periodic", 5000)])
def test_locate_every_row(fm, kind, n, interval):
    if kind == "uniform":
        R = synth.uniform_text(50 + n, n)
    elif kind == "acag":
        R = synth.from_ascii("ACAG")
    elif kind == "periodic":
        R = synth.from_ascii(("ACGTTGCA" * 1000)[:n])
    else:
        R = synth.repeat_text(51, n, families=20, min_len=300, max_len=3000)
    h = fm.fm_build(R, interval=interval)
    sa = oracle.Index(R, "sais").sa
    rows = torch.arange(R.size + 1, dtype=torch.int32, device="cuda")
    steps = torch.zeros(1, dtype=torch.int64, device="cuda")
    pos = fm.fm_locate(h, rows, steps=steps).cpu().numpy().astype(np.int64)
    assert np.array_equal(pos, sa)
    assert int(steps.item()) >= 0
    h.close()


def test_locate_interval_rows_are_occurrences(fm):
    R = synth.repeat_text(52, 300_000, families=30, min_len=300, max_len=3000)
    text = R
    h = fm.fm_build(R)
    reads = synth.sample_reads(53, R, 200, 8, 20, random_frac=0.2)
    codes, offs = fm.to_device_reads(reads)
    k, l = fm.fm_exact(h, codes, offs)
    k, l = k.cpu().numpy(), l.cpu().numpy()
    rows = np.concatenate([np.arange(k[r], l[r] + 1) for r in range(len(reads))]).astype(np.int32)
    pos = fm.fm_locate(h, torch.from_numpy(rows).cuda()).cpu().numpy()
    at = 0
    for r in range(len(reads)):
        W = reads.read(r)
        m = W.size
        want = [p for p in range(R.size - m + 1) if np.array_equal(text[p:p + m], W)] \
            if r < 40 else None
        got = sorted(pos[at:at + (l[r] - k[r] + 1)].tolist())
        at += max(l[r] - k[r] + 1, 0)
        for p in got:
            assert np.array_equal(text[p:p + m], W)
        if want is not None:
            assert got == want
    h.close()


def test_locate_domain_error(fm):
    R = synth.uniform_text(3, 1000)
    h = fm.fm_build(R)
    with pytest.raises(fm.FmError) as ei:
        fm.fm_locate(h, torch.tensor([0, 1001], dtype=torch.int32, device="cuda"))
    assert ei.value.code == fm.FM_EINVAL
    h.close()
