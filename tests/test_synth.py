"""The seeded input generators (no search arithmetic; both sides of every parity test read
their output): the counter-based hash against its published definition, independence from
chunking, and the shapes the workload recipes state (GC content, repeat share, read lengths,
error rates, strands, occ8 query mix)."""
import numpy as np

from paper_1811_06127_gb300 import synth


def test_splitmix64_reference_outputs():
    # the first outputs of splitmix64 from state 0 (Steele, Lea and Flood 2014)
    got = synth.splitmix64(0, np.arange(3, dtype=np.uint64)).tolist()
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_draws_are_keyed_by_position():
    a = synth.uniform_text(7, 1_000_003)
    assert np.array_equal(a[:4321], synth.uniform_text(7, 4321))
    text = synth.gc_text(8, 200_000)
    r1 = synth.sample_reads(9, text, 3000, 20, 90, sub_rate=0.02, indel_rate=0.01,
                            both_strands=True, random_frac=0.1)
    r2 = synth.sample_reads(9, text, 3000, 20, 90, sub_rate=0.02, indel_rate=0.01,
                            both_strands=True, random_frac=0.1, chunk=97)
    assert np.array_equal(r1.codes, r2.codes) and np.array_equal(r1.offs, r2.offs)


def test_gc_text_composition():
    t = synth.gc_text(11, 2_000_000, 0.41)
    f = np.bincount(t, minlength=4) / t.size
    assert abs(f[1] + f[2] - 0.41) < 0.003
    assert abs(f[0] - 0.295) < 0.003 and abs(f[3] - 0.295) < 0.003


def test_repeat_text_copies_cover_the_stated_share():
    # at the 64 Mbp reference's size the copies overwrite 20% of a 41% GC background (a random
    # base differs from the background base with probability 1 - sum(p^2) = 0.7418); at small
    # sizes the one-copy minimum per family raises the share (41% at 4 Mbp with 500 families)
    n = 64_000_000
    t = synth.repeat_text(1811061273, n)
    bg = synth.gc_text(synth.substream(1811061273, 1), n, 0.41)
    p = np.array([0.295, 0.205, 0.205, 0.295])
    frac = float((t != bg).mean())
    assert abs(frac - 0.2 * (1 - (p * p).sum())) < 0.01


def test_read_lengths_errors_and_strands():
    text = synth.gc_text(13, 300_000)
    clean = synth.sample_reads(14, text, 4000, 50, 250)
    lens = clean.lengths if not callable(clean.lengths) else clean.lengths()
    assert lens.min() >= 50 and lens.max() <= 250 and abs(lens.mean() - 150) < 3
    s = text.tobytes()
    assert all(s.find(clean.read(r).tobytes()) >= 0 for r in range(0, 4000, 40))
    # substitutions: same starts and lengths, so position-wise comparison gives the rate
    noisy = synth.sample_reads(14, text, 4000, 50, 250, sub_rate=0.01)
    assert np.array_equal(noisy.offs, clean.offs)
    assert abs(float((noisy.codes != clean.codes).mean()) - 0.01) < 0.001
    # both strands: about half of the copied reads come out reverse-complemented
    both = synth.sample_reads(14, text, 4000, 50, 250, both_strands=True)
    flipped = sum(not np.array_equal(both.read(r), clean.read(r)) for r in range(4000))
    assert abs(flipped / 4000 - 0.5) < 0.03
    for r in range(0, 4000, 97):
        w = both.read(r)
        assert np.array_equal(w, clean.read(r)) or np.array_equal(w, synth.revcomp(clean.read(r)))


def test_occ_queries_mixed_shape():
    n, I = 10_000_000, 64
    k, l = synth.occ_queries_mixed(15, n, 1 << 18, I)
    k, l = k.astype(np.int64), l.astype(np.int64)
    assert (k >= 0).all() and (l <= n).all() and (k <= l + 1).all()
    same = k // I == (l + 1) // I
    # half are drawn inside one block; a geometric gap g (mean 1000) puts k and l+1 = k+g+1 in
    # one block too with probability (I - g - 1) / I
    q = 1.0 / 1000.0
    g = np.arange(1, I - 1)
    p_short = float((q * (1 - q) ** (g - 1) * (I - g - 1) / I).sum())
    assert abs(float(same.mean()) - (0.5 + 0.5 * p_short)) < 0.005
    gap = l - k
    assert (gap[~same] >= 1).all()
    # only geometric draws reach gaps >= I; by memorylessness gap - (I - 1) then has mean 1000,
    # and they are half of the queries times P(g >= I)
    far = gap[gap >= I]
    assert abs(far.size / gap.size - 0.5 * (1 - q) ** (I - 1)) < 0.005
    assert abs(float((far - (I - 1)).mean()) - 1000) < 15
