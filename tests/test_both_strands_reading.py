"""Reading of the both-strands index, pinned on the CPU with the oracle: on T = R . revcomp(R)
a read's exact-match count equals its count on R plus its reverse complement's count on R plus
the occurrences that straddle the junction at |R|."""
import numpy as np

import oracle
from paper_1811_06127_gb300 import synth


def _count(text, W):
    if W.size > text.size:
        return 0
    win = np.lib.stride_tricks.sliding_window_view(text, W.size)
    return int((win == W).all(axis=1).sum())


def test_count_identity_on_t():
    R = synth.repeat_text(91, 20_000, families=4, min_len=300, max_len=900)
    T = np.concatenate([R, synth.revcomp(R)]).astype(np.uint8)
    ixT = oracle.Index(T, "sais")
    reads = synth.sample_reads(92, R, 200, 1, 40, sub_rate=0.02, both_strands=True,
                               random_frac=0.1)
    k, l = ixT.exact(reads.codes, reads.offs)
    n = R.size
    for r in range(len(reads)):
        W = reads.read(r)
        m = W.size
        straddle = _count(T[max(0, n - m + 1):n + m - 1], W)
        want = _count(R, W) + _count(R, synth.revcomp(W)) + straddle
        assert max(int(l[r]) - int(k[r]) + 1, 0) == want, r
