"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code: values printed in the paper
(tests/golden), closed forms, brute force on tiny inputs written in plain Python, textbook
routines, and invariants.  Runs without a GPU.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import halfbyte
from paper_1811_06127_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SYM = "ACGT"


def read_golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            rows.setdefault(key, []).append(vals)
    return rows


def s2c(s):
    return synth.from_ascii(s)


def suffixes(text):
    """Sorted suffixes of text$ as (string, start): '$' (0x24) sorts below 'A'."""
    t = text + "$"
    return sorted((t[p:], p) for p in range(len(t)))


def brute_interval(text, w):
    """[k, l] of pattern w by direct comparison with every sorted suffix."""
    suf = suffixes(text)
    rows = [r for r, (s, _) in enumerate(suf) if s.startswith(w)]
    if rows:
        return rows[0], rows[-1]
    k = sum(1 for s, _ in suf if s < w)
    return k, k - 1


def brute_occurrences(text, w):
    return sum(1 for p in range(len(text) - len(w) + 1) if text[p:p + len(w)] == w)


# --------------------------------------------------------------------------------------------
# Fig. 1 and Listing 1
# --------------------------------------------------------------------------------------------

def test_fig1_index(orc):
    g = read_golden("fig1_acag.txt")
    R = s2c(g["text"][0][0])
    for method in ("naive", "sais"):
        ix = oracle.Index(R, method)
        assert ix.sa.tolist() == [int(v) for v in g["sa"][0]]
        bwt = "".join("ACGT$"[c] for c in ix.bwt)
        assert bwt == "".join(g["bwt"][0])
        assert ix.C.tolist() == [int(v) for v in g["c"][0]]
        for row in g["occ"]:
            k = int(row[0])
            assert ix.occ4(k).tolist() == [int(v) for v in row[1:]]
            for b in range(4):
                assert oracle.occ_scan(ix.bwt, b, k) == int(row[1 + b])
        assert ix.occ4(-1).tolist() == [0, 0, 0, 0]


@pytest.mark.parametrize("w,expect", [("A", (1, 2)), ("G", (4, 4)), ("CA", (3, 3)),
                                      ("AG", (2, 2)), ("ACAG", (1, 1)), ("T", (5, 4)),
                                      ("GA", (5, 4)), ("", (0, 4))])
def test_listing1_on_fig1(w, expect):
    """Listing 1 from [0, n] on R = ACAG: rows as read off the SA column of Fig. 1."""
    ix = oracle.Index(s2c("ACAG"), "naive")
    codes = s2c(w) if w else np.zeros(0, np.uint8)
    k, l = ix.exact(codes, np.array([0, len(w)], np.uint32))
    assert (int(k[0]), int(l[0])) == expect
    assert brute_interval("ACAG", w) == expect


# --------------------------------------------------------------------------------------------
# Fig. 2: the 2-bit code and the half-byte count
# --------------------------------------------------------------------------------------------

def test_fig2_halfbyte():
    g = read_golden("fig2_halfbyte.txt")
    s = g["string"][0][0]
    x = "acgt".index(g["symbol"][0][0])
    codes = s2c(s)
    word = halfbyte.pack(codes)
    assert word == int(g["packed"][0][0], 16)
    trace = {}
    cnt = halfbyte.count_in_word(word, x, trace)
    for key in ("lo_nibbles", "hi_nibbles", "lo_lookup", "hi_lookup", "lo_shifted",
                "hi_shifted", "lo_filled", "hi_masked", "sad", "count"):
        assert trace[key] == int(g[key][0][0], 16), key
    assert cnt == s.count("g") == 6
    # the oracle's plain scan agrees on the same symbols read as a BWT fragment
    L = np.concatenate([codes, [4]]).astype(np.uint8)
    assert oracle.occ_scan(L, x, 31) == 6


def test_halfbyte_vs_scan_random():
    rng = np.random.default_rng(5)
    for _ in range(200):
        m = int(rng.integers(1, 200))
        codes = rng.integers(0, 4, m).astype(np.uint8)
        L = np.concatenate([codes, [4]]).astype(np.uint8)
        t = int(rng.integers(0, m + 1))
        for x in range(4):
            assert halfbyte.count_prefix(codes, x, t) == int((codes[:t] == x).sum())
            assert oracle.occ_scan(L, x, t - 1) == int((codes[:t] == x).sum())


# --------------------------------------------------------------------------------------------
# Eq. 1 / Eq. 2 / C / Occ
# --------------------------------------------------------------------------------------------

def _texts():
    rng = np.random.default_rng(1)
    out = [np.zeros(0, np.uint8), s2c("A"), s2c("T"), s2c("AC"), s2c("CA"), s2c("AAAA"),
           s2c("ACAG")]
    out.append(s2c("AC" * 300))
    out.append(s2c("A" * 500))
    out.append(s2c("ACGTTGCA" * 64 + "ACG"))
    for n in (1, 2, 3, 7, 64, 65, 127, 128, 129, 1000):
        out.append(rng.integers(0, 4, n).astype(np.uint8))
    out.append(synth.repeat_text(7, 20000, families=5, min_len=300, max_len=600))
    return out


def test_sa_naive_equals_sais_and_is_sorted():
    for R in _texts():
        sa_n = oracle.sa_naive(R)
        sa_s = oracle.sa_sais(R)
        assert sa_n.tolist() == sa_s.tolist()
        n = R.size
        assert sorted(sa_s.tolist()) == list(range(n + 1))
        assert sa_s[0] == n
        if n <= 1200:
            text = "".join(SYM[c] for c in R)
            assert [p for _, p in suffixes(text)] == sa_s.tolist()


def test_sais_large_random_matches_naive():
    R = synth.uniform_text(11, 200000)
    assert np.array_equal(oracle.sa_naive(R), oracle.sa_sais(R))


def _lf_inverse(L, Cc, dollar):
    """Inverse BWT by LF walks with a plain cumulative count (independent of the oracle)."""
    n = L.size - 1
    cum = np.zeros((n + 2, 4), dtype=np.int64)
    for i in range(n + 1):
        cum[i + 1] = cum[i]
        if L[i] < 4:
            cum[i + 1, L[i]] += 1
    out = []
    r = 0                      # row of the suffix "$": its BWT symbol is R[n-1]
    for _ in range(n):
        b = int(L[r])
        out.append(b)
        r = Cc[b] + cum[r + 1, b]          # LF(r) = C[b] + Occ(b, r)
    assert r == dollar                     # walked back to the suffix R[0..]
    return np.array(out[::-1], dtype=np.uint8)


def test_bwt_inverts_to_text():
    for R in _texts():
        if R.size > 3000:
            continue
        ix = oracle.Index(R, "sais")
        L = ix.bwt
        assert (L == 4).sum() == 1 and L[ix.dollar_row] == 4
        assert np.array_equal(_lf_inverse(L, ix.C, ix.dollar_row), R)


def test_c_and_occ_invariants():
    rng = np.random.default_rng(3)
    for R in _texts():
        ix = oracle.Index(R, "sais")
        n = R.size
        Cc = ix.C
        counts = np.bincount(R, minlength=4) if n else np.zeros(4, np.int64)
        assert Cc.tolist() == [0, *np.cumsum(counts).tolist()]
        assert Cc[4] == n
        L = ix.bwt
        ks = sorted({-1, 0, n, *rng.integers(-1, n + 1, 20).tolist()})
        for k in ks:
            o = ix.occ4(k)
            assert o.sum() == (k + 1) - (1 if ix.dollar_row <= k else 0)
            for b in range(4):
                assert o[b] == int((L[:k + 1] == b).sum())
        assert ix.occ4(n).tolist() == counts.tolist()


def test_occ8_batch_and_sweep_agree():
    R = synth.repeat_text(3, 50000, families=10, min_len=300, max_len=1000)
    ix = oracle.Index(R, "sais")
    n = R.size
    k, l = synth.occ_queries_uniform(9, n, 5000)
    k2, l2 = synth.occ_queries_mixed(10, n, 5000, 64)
    k = np.concatenate([k, k2, [0, n + 1, 0, n]]).astype(np.uint32)
    l = np.concatenate([l, l2, [n, n, 0, 0]]).astype(np.uint32)
    a = ix.occ8(k, l)
    b = ix.occ8_sweep(k, l)
    assert np.array_equal(a, b)
    L = ix.bwt
    cum = np.zeros((n + 2, 4), dtype=np.int64)
    for c in range(4):
        cum[1:, c] = np.cumsum(L == c)
    assert np.array_equal(a[:, :4], cum[k.astype(np.int64)])
    assert np.array_equal(a[:, 4:], cum[l.astype(np.int64) + 1])
    with pytest.raises(ValueError):
        ix.occ8(np.array([n + 2], np.uint32), np.array([0], np.uint32))


# --------------------------------------------------------------------------------------------
# Listing 1 closed form
# --------------------------------------------------------------------------------------------

def test_exact_matches_closed_form_and_counts():
    R = synth.repeat_text(5, 30000, families=8, min_len=300, max_len=800)
    text = "".join(SYM[c] for c in R)
    ix = oracle.Index(R, "sais")
    reads = synth.sample_reads(6, R, 400, 1, 24, random_frac=0.3, sub_rate=0.02)
    k, l = ix.exact(reads.codes, reads.offs)
    kn, ln, o8 = oracle.interval_naive(R, reads.codes, reads.offs)
    assert np.array_equal(k.astype(np.int64), kn)
    assert np.array_equal(l.astype(np.int64), ln)
    sa = ix.sa
    for r in range(60):
        w = "".join(SYM[c] for c in reads.read(r))
        assert int(l[r]) - int(k[r]) + 1 == brute_occurrences(text, w)
        # rows k..l are exactly the suffixes starting with w
        for row in range(int(k[r]), int(l[r]) + 1):
            assert text[sa[row]:].startswith(w)
    # eight Occ values of the closed form equal the index's
    assert np.array_equal(o8, ix.occ8(kn.astype(np.uint32), ln.astype(np.uint32)).astype(np.int64))


def test_exact_tiny_bruteforce():
    rng = np.random.default_rng(8)
    for _ in range(30):
        n = int(rng.integers(1, 40))
        R = rng.integers(0, 4, n).astype(np.uint8)
        text = "".join(SYM[c] for c in R)
        ix = oracle.Index(R, "naive")
        for _ in range(10):
            m = int(rng.integers(0, 6))
            W = rng.integers(0, 4, m).astype(np.uint8)
            w = "".join(SYM[c] for c in W)
            k, l = ix.exact(W, np.array([0, m], np.uint32))
            assert (int(k[0]), int(l[0])) == brute_interval(text, w)


# --------------------------------------------------------------------------------------------
# D lower bound
# --------------------------------------------------------------------------------------------

def brute_D(text, w):
    z, j, D = 0, 0, []
    for i in range(len(w)):
        if w[j:i + 1] not in text:
            z += 1
            j = i + 1
        D.append(z)
    return D


def edit_to_any_substring(text, w):
    """min over substrings X of R of the edit distance(w, X), by the free-start DP."""
    m = len(w)
    best = m
    prev = list(range(m + 1))
    # column DP over the text with free start (row 0 all zeros) and free end
    cur = [0] * (m + 1)
    col = [i for i in range(m + 1)]
    for ch in text:
        new = [0] * (m + 1)
        for i in range(1, m + 1):
            new[i] = min(col[i] + 1, new[i - 1] + 1, col[i - 1] + (w[i - 1] != ch))
        col = new
        best = min(best, col[m])
    del prev, cur
    return best


def test_dcalc_definition_and_lower_bound():
    rng = np.random.default_rng(12)
    for _ in range(40):
        n = int(rng.integers(5, 60))
        R = rng.integers(0, 4, n).astype(np.uint8)
        text = "".join(SYM[c] for c in R)
        ix = oracle.Index(R, "naive")
        for _ in range(8):
            m = int(rng.integers(1, 12))
            if rng.random() < 0.5 and n > m:
                p = int(rng.integers(0, n - m))
                W = R[p:p + m].copy()
                W[rng.integers(0, m)] = rng.integers(0, 4)
            else:
                W = rng.integers(0, 4, m).astype(np.uint8)
            w = "".join(SYM[c] for c in W)
            D = ix.dcalc(W).tolist()
            assert D == brute_D(text, w)
            for i in range(m):
                assert D[i] <= edit_to_any_substring(text, w[:i + 1])


# --------------------------------------------------------------------------------------------
# Listing 2
# --------------------------------------------------------------------------------------------

def canonical_pair_ok(prev, col, i, w):
    """Whether column col may follow column prev in a canonical script (prev = None at the
    start).  Columns: ("I",) insertion of w[i], ("D", b) deletion of reference symbol b,
    ("M", b) match or mismatch with b against w[i]; prev was taken at read position i + 1
    (insertion, match, mismatch) or i (deletion)."""
    if prev is None or (prev[0] == "M" and prev[1] == w[i + 1]):
        return True
    if prev[0] == "I":      # shift the insertion left; mismatch or match first
        return col[0] == "I" or (col[0] == "M" and col[1] == w[i] and w[i] != w[i + 1])
    if prev[0] == "D":      # shift the deletion left (not past w[0]); no deletion+insertion
        if col[0] == "I":
            return False
        if col[0] == "M" and i >= 1:
            return col[1] == w[i] and w[i] != prev[1]
        return True
    # prev is a mismatch with prev[1] at w[i+1]
    if col[0] == "I":
        return w[i] != prev[1]
    if col[0] == "D":
        return col[1] != w[i + 1]
    return True


def brute_inexact(text, w, z, gaps, prune=False, interval=4, canonical=False, end_skip=0):
    """Enumerate every alignment column script of Listing 2's grammar (processing w from its
    right end): insertion (consume w[i]), deletion (emit a reference symbol, i unchanged),
    match/mismatch (emit b, consume w[i]); cost <= z, indel columns <= gaps; stop at i < 0.
    Returns the set of intervals of the reference-side strings that occur in text, and the
    number of script prefixes (states) that reach i >= 0 with an occurring reference string
    (and, with prune, z_left >= D(i)) together with their checkpoint blocks of the given
    width at rank positions k and l+1.  canonical: only scripts whose adjacent columns pass
    canonical_pair_ok; a state counts only when a deletion (needs a gap and a difference
    left), a mismatch (needs a difference left) or the match may follow it.  The fourth value
    maps each interval to the fewest differences of the scripts that reach it.  end_skip: an
    insertion of w[i] needs end_skip <= i <= m-1-end_skip, a deletion taken at i (between
    w[i] and w[i+1]) needs end_skip <= i+1 and i <= m-1-end_skip."""
    strings = {}
    D = brute_D(text, w)
    stats = [0, 0]
    m = len(w)

    def ins_ok(i):
        return end_skip <= i <= m - 1 - end_skip

    def del_ok(i):
        return end_skip <= i + 1 and i <= m - 1 - end_skip

    def ok(prev, col, i):
        return not canonical or canonical_pair_ok(prev, col, i, w)

    def rec(i, zl, g, x, prev):
        if zl < 0:
            return
        if x and x not in text:
            return
        if prune and i >= 0 and zl < D[i]:
            return
        if i < 0:
            if x:
                strings[x] = min(strings.get(x, 99), z - zl)
            return
        if g < gaps and ins_ok(i) and ok(prev, ("I",), i):
            rec(i - 1, zl - 1, g + 1, x, ("I",))
        occ_child = any((col[0] == "D" and g < gaps and zl >= 1 and del_ok(i)) or
                        (col[0] == "M" and (col[1] == w[i] or zl >= 1))
                        for col in [("D", b) for b in SYM] + [("M", b) for b in SYM]
                        if ok(prev, col, i))
        if not occ_child:
            return
        k, l = brute_interval(text, x) if x else (0, len(text))
        stats[0] += 1
        stats[1] += 1 if k // interval == (l + 1) // interval else 2
        for b in SYM:
            if g < gaps and del_ok(i) and ok(prev, ("D", b), i):
                rec(i, zl - 1, g + 1, b + x, ("D", b))
            if ok(prev, ("M", b), i):
                rec(i - 1, zl - (b != w[i]), g, b + x, ("M", b))

    rec(len(w) - 1, z, 0, "", None)
    cost = {}
    for x, c in strings.items():
        k, l = brute_interval(text, x)
        if k <= l:
            cost[(k, l)] = min(cost.get((k, l), 99), c)
    return sorted(cost), stats[0], stats[1], cost


def _pairs_of(res, q):
    o = res["offsets"]
    return [tuple(map(int, p)) for p in res["pairs"][o[q]:o[q + 1]]]


def test_inexact_bruteforce_tiny():
    rng = np.random.default_rng(21)
    cases = 0
    for _ in range(25):
        n = int(rng.integers(8, 48))
        R = synth.uniform_text(int(rng.integers(1 << 30)), n)
        text = "".join(SYM[c] for c in R)
        ix = oracle.Index(R, "naive")
        ws = []
        for _ in range(4):
            m = int(rng.integers(1, 7))
            if rng.random() < 0.6 and n > m:
                p = int(rng.integers(0, n - m))
                W = R[p:p + m].copy()
                if rng.random() < 0.5:
                    W[rng.integers(0, m)] = rng.integers(0, 4)
            else:
                W = rng.integers(0, 4, m).astype(np.uint8)
            ws.append(W)
        codes = np.concatenate(ws).astype(np.uint8)
        offs = np.concatenate([[0], np.cumsum([w.size for w in ws])]).astype(np.uint32)
        for z in (0, 1, 2):
            for gaps in (0, 1, 2):
                res = ix.inexact(codes, offs, z, gaps, strands=1, prune=True, interval=4)
                res_np = ix.inexact(codes, offs, z, gaps, strands=1, prune=False, interval=4)
                res_c = ix.inexact(codes, offs, z, gaps, strands=1, prune=True, interval=4,
                                   canonical=True)
                for q, W in enumerate(ws):
                    w = "".join(SYM[c] for c in W)
                    got = _pairs_of(res, q)
                    assert got == _pairs_of(res_np, q)
                    want, nodes, blocks, cost = brute_inexact(text, w, z, gaps, prune=True)
                    assert got == want, (text, w, z, gaps)
                    # fewest differences per interval
                    o = res["offsets"]
                    assert [int(c) for c in res["costs"][o[q]:o[q + 1]]] == \
                        [cost[p] for p in want], (text, w, z, gaps)
                    assert (int(res["nodes"][q]), int(res["blocks"][q])) == (nodes, blocks)
                    _, nodes, blocks, _ = brute_inexact(text, w, z, gaps, prune=False)
                    assert (int(res_np["nodes"][q]), int(res_np["blocks"][q])) == (nodes, blocks)
                    # canonical enumeration: Listing 2's intervals, the brute-force counts
                    want_c, nodes_c, blocks_c, cost_c = brute_inexact(text, w, z, gaps,
                                                                      prune=True, canonical=True)
                    assert want_c == want and cost_c == cost, (text, w, z, gaps)
                    assert _pairs_of(res_c, q) == want
                    assert (int(res_c["nodes"][q]), int(res_c["blocks"][q])) == \
                        (nodes_c, blocks_c), (text, w, z, gaps)
                    assert nodes_c <= nodes
                    cases += 1
                assert np.array_equal(res_c["costs"], res["costs"])
    assert cases > 500


def min_script_cost(w, x, gaps, end_skip):
    """The fewest differences of a column script that aligns all of w to all of x, read left to
    right: a match or mismatch column takes one symbol of each, an insertion one symbol of w,
    a deletion one symbol of x; at most `gaps` indel columns; a deletion has at least one
    symbol of w on its left (Listing 2 places nothing before w[0]); every indel column has at
    least end_skip symbols of w on each side.  None when no script exists.  A dynamic program
    over (symbols of w used, symbols of x used, indel columns used): an independent statement
    of the set Listing 2 reaches, since a string's suffixes occur wherever it occurs."""
    m, n = len(w), len(x)
    INF = 1 << 20
    f = [[[INF] * (gaps + 1) for _ in range(n + 1)] for _ in range(m + 1)]
    f[0][0][0] = 0
    for i in range(m + 1):
        for j in range(n + 1):
            for g in range(gaps + 1):
                v = f[i][j][g]
                if v >= INF:
                    continue
                if i < m and j < n:
                    c = v + (w[i] != x[j])
                    f[i + 1][j + 1][g] = min(f[i + 1][j + 1][g], c)
                if g < gaps and i < m and end_skip <= i <= m - 1 - end_skip:
                    f[i + 1][j][g + 1] = min(f[i + 1][j][g + 1], v + 1)
                if g < gaps and j < n and i >= max(1, end_skip) and m - i >= end_skip:
                    f[i][j + 1][g + 1] = min(f[i][j + 1][g + 1], v + 1)
    best = min(f[m][n][g] for g in range(gaps + 1))
    return None if best >= INF else best


def defined_inexact(text, w, z, gaps, end_skip):
    """Interval -> fewest differences over the non-empty strings x of text that some script of
    at most z differences aligns w to (min_script_cost), by enumerating the substrings."""
    out = {}
    subs = {text[p:p + t] for t in range(1, len(w) + gaps + 1) for p in range(len(text) - t + 1)}
    for x in subs:
        c = min_script_cost(w, x, gaps, end_skip)
        if c is not None and c <= z:
            k, l = brute_interval(text, x)
            out[(k, l)] = min(out.get((k, l), 99), c)
    return out


def test_end_restriction_bruteforce_and_definition():
    """Indel columns only with at least end_skip read symbols on each side: the oracle's sets,
    costs, node and block counts equal the brute-force scripts', and its sets and costs equal
    the alignment definition (which also pins end_skip = 0, plain Listing 2, a second way)."""
    rng = np.random.default_rng(33)
    cases = 0
    for _ in range(14):
        n = int(rng.integers(8, 40))
        R = synth.uniform_text(int(rng.integers(1 << 30)), n)
        text = "".join(SYM[c] for c in R)
        ix = oracle.Index(R, "naive")
        ws = []
        for _ in range(4):
            m = int(rng.integers(1, 9))
            if rng.random() < 0.7 and n > m + 1:
                p = int(rng.integers(0, n - m - 1))
                W = R[p:p + m].copy()
                u = rng.random()
                if u < 0.3:
                    W[rng.integers(0, m)] = rng.integers(0, 4)
                elif u < 0.6 and m > 1:     # one symbol dropped: an insertion in R's terms
                    W = np.delete(R[p:p + m + 1], rng.integers(1, m))
                elif u < 0.9 and m > 1:
                    W = np.delete(W, rng.integers(0, m))
            else:
                W = rng.integers(0, 4, m).astype(np.uint8)
            ws.append(W.astype(np.uint8))
        codes = np.concatenate(ws).astype(np.uint8)
        offs = np.concatenate([[0], np.cumsum([w.size for w in ws])]).astype(np.uint32)
        for z in (1, 2):
            for gaps in (1, 2):
                for e in (0, 1, 2, 3):
                    res = ix.inexact(codes, offs, z, gaps, strands=1, interval=4, end_skip=e)
                    res_np = ix.inexact(codes, offs, z, gaps, strands=1, interval=4,
                                        end_skip=e, prune=False)
                    o = res["offsets"]
                    for q, W in enumerate(ws):
                        w = "".join(SYM[c] for c in W)
                        got = _pairs_of(res, q)
                        costs = [int(c) for c in res["costs"][o[q]:o[q + 1]]]
                        assert got == _pairs_of(res_np, q)
                        want, nodes, blocks, cost = brute_inexact(text, w, z, gaps, prune=True,
                                                                  end_skip=e)
                        assert got == want and costs == [cost[p] for p in want], (text, w, z, e)
                        assert (int(res["nodes"][q]), int(res["blocks"][q])) == (nodes, blocks)
                        d = defined_inexact(text, w, z, gaps, e)
                        assert got == sorted(d) and costs == [d[p] for p in got], (text, w, z, e)
                        cases += 1
    assert cases > 400


def test_end_restriction_invariants():
    """end_skip = 0 is the unrestricted search; a larger end_skip reports a subset with no
    lower costs; above half the read length no indel fits, which is the mismatch-only search
    (same sets, costs and nodes); the canonical rewrites are not combined with it."""
    R = synth.repeat_text(5, 30_000, families=8, min_len=100, max_len=600)
    reads = synth.sample_reads(6, R, 120, 10, 40, sub_rate=0.02, indel_rate=0.02,
                               both_strands=True)
    ix = oracle.Index(R, "sais")
    base = ix.inexact(reads.codes, reads.offs, 2, 1, strands=2)
    e0 = ix.inexact(reads.codes, reads.offs, 2, 1, strands=2, end_skip=0)
    for key in ("counts", "offsets", "pairs", "costs", "nodes", "blocks"):
        assert np.array_equal(base[key], e0[key])
    prev = base
    for e in (1, 3, 8):
        cur = ix.inexact(reads.codes, reads.offs, 2, 1, strands=2, end_skip=e)
        for q in range(cur["counts"].size):
            a, b = prev["offsets"][q:q + 2], cur["offsets"][q:q + 2]
            old = {tuple(map(int, p)): int(c) for p, c in
                   zip(prev["pairs"][a[0]:a[1]], prev["costs"][a[0]:a[1]])}
            for p, c in zip(cur["pairs"][b[0]:b[1]], cur["costs"][b[0]:b[1]]):
                assert tuple(map(int, p)) in old and int(c) >= old[tuple(map(int, p))]
        assert cur["nodes"].sum() <= prev["nodes"].sum()
        prev = cur
    assert prev["counts"].sum() < base["counts"].sum()
    none = ix.inexact(reads.codes, reads.offs, 2, 1, strands=2, end_skip=21)
    mis = ix.inexact(reads.codes, reads.offs, 2, 0, strands=2)
    for key in ("counts", "offsets", "pairs", "costs", "nodes", "blocks"):
        assert np.array_equal(none[key], mis[key]), key
    with pytest.raises(ValueError):
        ix.inexact(reads.codes, reads.offs, 2, 1, strands=2, end_skip=2, canonical=True)


def _runs_text(rng, n):
    parts, total = [], 0
    while total < n:
        r = np.full(int(rng.integers(1, 6)), int(rng.integers(0, 4)), dtype=np.uint8)
        parts.append(r)
        total += r.size
    return np.concatenate(parts)[:n]


def test_canonical_bruteforce_runs():
    """Texts and reads made of runs of one base (where indels can sit in several places and
    still spell one string), z up to 3: the canonical enumeration reports Listing 2's
    intervals and its node and block counts equal the brute-force canonical scripts'."""
    rng = np.random.default_rng(23)
    cases = 0
    for _ in range(12):
        R = _runs_text(rng, int(rng.integers(10, 40)))
        text = "".join(SYM[c] for c in R)
        ix = oracle.Index(R, "naive")
        ws = [_runs_text(rng, int(rng.integers(1, 7))) for _ in range(3)]
        codes = np.concatenate(ws).astype(np.uint8)
        offs = np.concatenate([[0], np.cumsum([w.size for w in ws])]).astype(np.uint32)
        for z, gaps in ((1, 1), (2, 1), (2, 2), (3, 2), (3, 3)):
            res = ix.inexact(codes, offs, z, gaps, strands=1, interval=4)
            res_c = ix.inexact(codes, offs, z, gaps, strands=1, interval=4, canonical=True)
            for q, W in enumerate(ws):
                w = "".join(SYM[c] for c in W)
                want, nodes_c, blocks_c, _ = brute_inexact(text, w, z, gaps, prune=True,
                                                           canonical=True)
                assert _pairs_of(res_c, q) == _pairs_of(res, q) == want, (text, w, z, gaps)
                assert (int(res_c["nodes"][q]), int(res_c["blocks"][q])) == (nodes_c, blocks_c)
                cases += 1
    assert cases >= 150


@pytest.mark.parametrize("kind", ["runs", "homopolymer", "periodic", "repeat"])
def test_canonical_same_results(kind):
    """Canonical enumeration = Listing 2's result sets (both strands, z <= 3, gaps <= 3)
    on texts where the same string is spelled by many scripts; it never expands more."""
    rng = np.random.default_rng(29)
    if kind == "runs":
        R = _runs_text(rng, 4000)
    elif kind == "homopolymer":
        R = np.zeros(400, np.uint8)
    elif kind == "periodic":
        R = np.array([0, 1] * 1000, np.uint8)
    else:
        R = synth.repeat_text(31, 60_000, families=8, min_len=300, max_len=1500)
    ix = oracle.Index(R, "sais")
    reads = synth.sample_reads(37, R, 60, 1, 30, sub_rate=0.05, indel_rate=0.03,
                               both_strands=True, random_frac=0.1)
    for z, gaps in ((1, 1), (2, 1), (2, 2), (3, 1), (3, 3)):
        a = ix.inexact(reads.codes, reads.offs, z, gaps, strands=2)
        b = ix.inexact(reads.codes, reads.offs, z, gaps, strands=2, canonical=True)
        for key in ("counts", "offsets", "pairs", "costs"):
            assert np.array_equal(a[key], b[key]), (kind, z, gaps, key)
        assert (b["nodes"] <= a["nodes"]).all()
        assert b["nodes"].sum() < a["nodes"].sum()


@pytest.mark.parametrize("z,gaps", [(4, 1), (4, 2), (4, 4), (5, 2), (6, 3)])
def test_canonical_same_results_high_z_run_poor(z, gaps):
    """Beyond z = 3: canonical enumeration = Listing 2's result sets and costs on a text with
    no run of one symbol (R[i] != R[i-1]), where the literal recursion stays affordable at
    z = 4..6.  Reads carry substitutions and indels, so every canonical rule is exercised."""
    rng = np.random.default_rng(1811061290)
    R = (np.cumsum(rng.integers(1, 4, 20_000)) % 4).astype(np.uint8)
    assert (R[1:] != R[:-1]).all()
    ix = oracle.Index(R, "sais")
    m = 40 if z == 4 else 24
    reads = synth.sample_reads(91 + z, R, 120, m // 2, m, sub_rate=0.03, indel_rate=0.01,
                               both_strands=True)
    a = ix.inexact(reads.codes, reads.offs, z, gaps, strands=2)
    b = ix.inexact(reads.codes, reads.offs, z, gaps, strands=2, canonical=True)
    for key in ("counts", "offsets", "pairs", "costs"):
        assert np.array_equal(a[key], b[key]), (z, gaps, key)
    assert int(a["offsets"][-1]) > 100
    assert (b["nodes"] <= a["nodes"]).all() and b["nodes"].sum() < a["nodes"].sum()


def test_inexact_hamming_identity_and_z0():
    R = synth.repeat_text(13, 40000, families=6, min_len=300, max_len=900)
    ix = oracle.Index(R, "sais")
    reads = synth.sample_reads(14, R, 120, 12, 30, sub_rate=0.05, both_strands=True,
                               random_frac=0.1)
    res = ix.inexact(reads.codes, reads.offs, 2, 0, strands=2)
    res0 = ix.inexact(reads.codes, reads.offs, 0, 0, strands=2)
    k, l = ix.exact(reads.codes, reads.offs)
    for r in range(len(reads)):
        for s in range(2):
            q = 2 * r + s
            W = reads.read(r) if s == 0 else synth.revcomp(reads.read(r))
            pairs = _pairs_of(res, q)
            total = sum(b - a + 1 for a, b in pairs)
            assert total == oracle.hamming_count(R, W, 2)
            # mismatches only: an interval's cost is the Hamming distance of W to its string
            o = res["offsets"]
            for (a, _), c in zip(pairs, res["costs"][o[q]:o[q + 1]]):
                p = int(ix.sa[a])
                assert int(c) == int((R[p:p + W.size] != W).sum())
            # disjoint: mismatch-only strings share one length
            for (a0, b0), (a1, b1) in zip(pairs, pairs[1:]):
                assert b0 < a1
            p0 = _pairs_of(res0, q)
            assert not res0["costs"].any()
            if s == 0:
                ke, le = int(k[r]), int(l[r])
                assert p0 == ([(ke, le)] if ke <= le else [])


def test_inexact_prune_is_exact_on_repeats():
    R = synth.repeat_text(17, 30000, families=6, min_len=300, max_len=700)
    ix = oracle.Index(R, "sais")
    reads = synth.sample_reads(18, R, 60, 15, 40, sub_rate=0.02, indel_rate=0.02,
                               both_strands=True, random_frac=0.05)
    for gaps in (0, 1):
        a = ix.inexact(reads.codes, reads.offs, 2, gaps, strands=2, prune=True)
        b = ix.inexact(reads.codes, reads.offs, 2, gaps, strands=2, prune=False)
        assert np.array_equal(a["counts"], b["counts"])
        assert np.array_equal(a["pairs"], b["pairs"])
        assert (a["nodes"] <= b["nodes"]).all()
        assert a["nodes"].sum() < b["nodes"].sum()


def test_inexact_gap_monotone():
    R = synth.repeat_text(19, 20000, families=4, min_len=300, max_len=600)
    ix = oracle.Index(R, "sais")
    reads = synth.sample_reads(20, R, 50, 10, 30, sub_rate=0.03, indel_rate=0.03)
    sets = []
    for z, g in ((0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)):
        res = ix.inexact(reads.codes, reads.offs, z, g)
        sets.append((z, g, [set(_pairs_of(res, q)) for q in range(len(reads))]))
    for za, ga, sa in sets:
        for zb, gb, sb in sets:
            if za <= zb and ga <= gb:
                assert all(x <= y for x, y in zip(sa, sb))


def test_hamming_count_bruteforce():
    rng = np.random.default_rng(4)
    for _ in range(50):
        n = int(rng.integers(1, 80))
        R = rng.integers(0, 4, n).astype(np.uint8)
        m = int(rng.integers(1, 10))
        W = rng.integers(0, 4, m).astype(np.uint8)
        for z in range(3):
            want = sum(1 for p in range(n - m + 1) if int((R[p:p + m] != W).sum()) <= z)
            assert oracle.hamming_count(R, W, z) == want
