"""The arithmetic of the two-symbol (pair) step, checked on the CPU against the oracle.

For row i of the BWT matrix the pair is the two symbols before suffix SA[i]; the GPU builds it
as (BWT[LF(i)], BWT[i]) with LF(i) = C[b] + Occ(b, i-1) + 1 (Eq. 4-5), and moves an interval
two symbols back with one rank over pairs plus pc2[pair], the number of rows that sort before
every string starting with the pair: 1 (the $ row) + C[b1] + [R ends with b1] + the pairs
(b1, y) with y < b2.  This test restates those definitions independently of the GPU code and
pins them: the LF form equals the definition through the suffix array, pc2 equals a direct
count over the suffixes, and a pair step equals two single steps of Listing 1 for every pair
and every interval, empty ones (insertion points) included."""
import numpy as np
import pytest

import oracle
from paper_1811_06127_gb300 import synth


def _texts():
    rng = np.random.default_rng(5)
    out = [np.array([0], np.uint8), np.array([2, 2], np.uint8), synth.from_ascii("ACAG")]
    for n in (5, 17, 64, 65, 130):
        out.append(rng.integers(0, 4, n).astype(np.uint8))
    out.append(np.array([0, 1] * 40, np.uint8))
    out.append(np.zeros(50, np.uint8))
    return out


@pytest.mark.parametrize("R", _texts(), ids=lambda R: f"n{R.size}")
def test_pair_step_equals_two_single_steps(R):
    ix = oracle.Index(R, "naive")
    n = R.size
    sa, L, C, drow = ix.sa, ix.bwt, ix.C, ix.dollar_row

    def occ(b, k):   # Occ(b, k): b among BWT[0..k], inclusive; Occ(b, -1) = 0
        return 0 if k < 0 else int(ix.occ4(k)[b])

    def step(b, k, l):   # Listing 1, one symbol
        return int(C[b]) + occ(b, k - 1) + 1, int(C[b]) + occ(b, l)

    # the pair of each row: by definition (suffix array) and as the GPU builds it (LF)
    pair_def, pair_lf = [], []
    for i in range(n + 1):
        p = int(sa[i])
        pair_def.append(4 * int(R[p - 2]) + int(R[p - 1]) if p >= 2 else None)
        if i == drow:
            pair_lf.append(None)
            continue
        b = int(L[i])
        lf = int(C[b]) + occ(b, i - 1) + 1
        pair_lf.append(None if lf == drow else 4 * int(L[lf]) + b)
    assert pair_lf == pair_def

    # pc2 by its formula, against a direct count over the suffixes
    count2 = [sum(1 for x in pair_def if x == c) for c in range(16)]
    suffixes = [tuple(R[p:]) for p in range(n + 1)]
    for b1 in range(4):
        for b2 in range(4):
            formula = 1 + int(C[b1]) + (1 if R[n - 1] == b1 else 0) + \
                sum(count2[4 * b1 + y] for y in range(b2))
            direct = sum(1 for s in suffixes if s < (b1, b2))
            assert formula == direct, (b1, b2)

    def rank2(c, p):   # pairs c in rows [0, p)
        return sum(1 for x in pair_def[:p] if x == c)

    def pc2(c):
        b1, b2 = divmod(c, 4)
        return 1 + int(C[b1]) + (1 if R[n - 1] == b1 else 0) + \
            sum(count2[4 * b1 + y] for y in range(b2))

    # every interval (k, l) with 0 <= k <= l + 1 <= n + 1, every pair
    for k in range(0, n + 2):
        for l in range(max(k - 1, 0), n + 1):
            if l < k - 1:
                continue
            for c in range(16):
                b1, b2 = divmod(c, 4)
                k1, l1 = step(b2, k, l)
                want = step(b1, k1, l1)
                got = (pc2(c) + rank2(c, k), pc2(c) + rank2(c, l + 1) - 1)
                assert got == want, (k, l, c)
