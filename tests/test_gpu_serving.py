"""Serving loop: each request's interval sets are the same alone and in the mix (tolerance 0:
integer intervals), for requests of mixed sizes and search modes arriving from several
threads while batches are on the GPU."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_1811_06127_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MODES = [(0, 0), (1, 0), (2, 1)]   # exact, z=1, z=2 with one gap


@pytest.fixture(scope="module")
def fm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1811_06127_gb300 import _build, fmocc
    _build.build()
    fmocc.load_library()
    return fmocc


def _requests(R, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(1, 300)) if i % 5 else int(rng.integers(1, 4))
        reads = synth.sample_reads(seed * 1000 + i, R, n, 50, 250, sub_rate=0.01,
                                   indel_rate=0.0005, both_strands=True)
        out.append((reads, MODES[i % 3]))
    return out


def test_alone_equals_mixed(fm):
    R = synth.repeat_text(1811061275, 400_000, families=40, min_len=300, max_len=3000)
    h = fm.fm_build(R)
    reqs = _requests(R, 48, 5)
    alone = []
    for reads, (z, g) in reqs:
        codes, offs = fm.to_device_reads(reads)
        c, o, p = fm.fm_inexact(h, codes, offs, z, g, strands=2)
        alone.append((c.cpu().numpy().view(np.uint32), o.cpu().numpy().astype(np.uint64),
                      p.cpu().numpy().view(np.uint32)))
    tickets = [None] * len(reqs)
    with fm.Server(h, max_batch_reads=2000, strands=2) as srv:
        def client(idx):
            for i in idx:
                reads, (z, g) = reqs[i]
                tickets[i] = srv.submit(reads.codes, reads.offs, z, g)
                time.sleep(0.002)
        threads = [threading.Thread(target=client, args=(range(t, len(reqs), 4),))
                   for t in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        results = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["requests"] == len(reqs)
    mixed = 0
    for (reads, _), want, got in zip(reqs, alone, results):
        assert got["status"] == fm.FM_OK
        assert np.array_equal(got["counts"], want[0])
        assert np.array_equal(got["offsets"], want[1])
        assert np.array_equal(got["pairs"], want[2])
        assert got["t_submit_ns"] <= got["t_start_ns"] <= got["t_done_ns"]
        mixed += got["batch_reads"] > len(reads)
    assert mixed > 0          # some requests shared a batch with others
    assert st["batches"] < len(reqs)
    # the mix against the oracle for a few requests
    ix = oracle.Index(R, "sais")
    for (reads, (z, g)), got in list(zip(reqs, results))[:6]:
        w = ix.inexact(reads.codes, reads.offs, z, g, strands=2)
        assert np.array_equal(got["pairs"], w["pairs"])
    h.close()


def _alone(fm, h, reads, z, g):
    codes, offs = fm.to_device_reads(reads)
    c, o, p = fm.fm_inexact(h, codes, offs, z, g, strands=2)
    return (c.cpu().numpy().view(np.uint32), o.cpu().numpy().astype(np.uint64),
            p.cpu().numpy().view(np.uint32))


def _check_same(got, want):
    assert got["status"] == 0
    assert np.array_equal(got["counts"], want[0])
    assert np.array_equal(got["offsets"], want[1])
    assert np.array_equal(got["pairs"], want[2])


@pytest.mark.parametrize("inflight", [1, 2])
def test_request_starts_while_a_batch_runs(fm, inflight):
    """A request submitted while a long batch is on the GPU starts before that batch
    finishes when two batches may be in flight (and only after it with one), and its result is
    what fm_inexact returns for it alone."""
    R = synth.repeat_text(1811061277, 8_000_000, families=100, min_len=300, max_len=6000)
    h = fm.fm_build(R)
    # a batch of about a second: z = 4 with 2 gaps on long reads
    big = synth.sample_reads(71, R, 200_000, 150, 250, sub_rate=0.02, indel_rate=0.002,
                             both_strands=True)
    small = synth.sample_reads(72, R, 50, 50, 150, sub_rate=0.01, both_strands=True)
    want_big, want_small = _alone(fm, h, big, 4, 2), _alone(fm, h, small, 1, 0)
    with fm.Server(h, max_batch_reads=200_000, strands=2, inflight=inflight) as srv:
        ta = srv.submit(big.codes, big.offs, 4, 2)
        time.sleep(0.1)   # the long batch has been taken by a worker
        tb = srv.submit(small.codes, small.offs, 1, 0)
        ra, rb = srv.wait(ta), srv.wait(tb)
    _check_same(ra, want_big)
    _check_same(rb, want_small)
    # the premise: the small request arrived while the long batch ran
    assert ra["t_start_ns"] < rb["t_submit_ns"] < ra["t_done_ns"], \
        (ra["t_start_ns"], rb["t_submit_ns"], ra["t_done_ns"])
    assert ra["batch_id"] != rb["batch_id"]
    if inflight == 2:
        # it started before the long batch finished (its kernels take SMs as the long
        # batch's persistent CTAs drain)
        assert rb["t_start_ns"] < ra["t_done_ns"]
    else:
        assert rb["t_start_ns"] >= ra["t_done_ns"]        # one batch at a time
    h.close()


def test_one_batch_mixes_search_modes(fm):
    """Requests of different search modes that wait together are searched in one batch
    (z and max_gaps are carried read by read), each with its own mode's result."""
    R = synth.repeat_text(1811061278, 4_000_000, families=60, min_len=300, max_len=4000)
    h = fm.fm_build(R)
    blockers = [synth.sample_reads(73 + i, R, 100_000, 100, 250, sub_rate=0.02,
                                   indel_rate=0.002, both_strands=True) for i in range(2)]
    reqs = [(synth.sample_reads(80 + i, R, 20 + 7 * i, 50, 250, sub_rate=0.01,
                                indel_rate=0.0005, both_strands=True), MODES[i % 3])
            for i in range(24)]
    want = [_alone(fm, h, r, z, g) for r, (z, g) in reqs]
    with fm.Server(h, max_batch_reads=200_000, strands=2, inflight=2) as srv:
        tk = [srv.submit(b.codes, b.offs, 3, 2) for b in blockers]   # both workers busy
        time.sleep(0.02)
        ts = [srv.submit(r.codes, r.offs, z, g) for r, (z, g) in reqs]
        res = [srv.wait(t) for t in ts]
        for t in tk:
            srv.wait(t)
    for got, w in zip(res, want):
        _check_same(got, w)
    modes_by_batch = {}
    for got, (_, m) in zip(res, reqs):
        modes_by_batch.setdefault(got["batch_id"], set()).add(m)
    assert max(len(v) for v in modes_by_batch.values()) == 3
    h.close()


def test_frontier_budget_splits_batches(fm):
    """With a frontier budget that holds the search scratch of only part of the backlog, the
    backlog runs as several batches (sized by the scratch model, and split when a search
    would outgrow the budget), and every result is still the request's own."""
    R = synth.repeat_text(1811061279, 4_000_000, families=60, min_len=300, max_len=4000)
    h = fm.fm_build(R)
    reqs = [synth.sample_reads(90 + i, R, 4000, 50, 250, sub_rate=0.01, indel_rate=0.0005,
                               both_strands=True) for i in range(16)]
    want = [_alone(fm, h, r, 2, 1) for r in reqs]
    budget = 420 << 20   # the spill region of the persistent kernel plus a few tens of MB
    with fm.Server(h, max_batch_reads=262_144, strands=2, inflight=1,
                   frontier_budget=budget) as srv:
        ts = [srv.submit(r.codes, r.offs, 2, 1) for r in reqs]
        res = [srv.wait(t) for t in ts]
        st = srv.stats()
    for got, w in zip(res, want):
        _check_same(got, w)
    assert len({g["batch_id"] for g in res}) >= 2
    assert st["batches"] >= 2
    h.close()


def test_server_errors(fm):
    R = synth.uniform_text(3, 50_000)
    h = fm.fm_build(R)
    with fm.Server(h, strands=2) as srv:
        with pytest.raises(fm.FmError):
            srv.submit(np.array([0, 9], np.uint8), np.array([0, 2], np.uint32), 1)
        # one bad code deep inside a request of several reads, whatever its high bits
        for bad in (4, 128, 255):
            codes = np.zeros(1000, np.uint8)
            codes[777] = bad
            with pytest.raises(fm.FmError) as ei:
                srv.submit(codes, np.arange(0, 1001, 200, dtype=np.uint32), 1)
            assert ei.value.code == fm.FM_EINVAL
        with pytest.raises(fm.FmError):
            srv.poll(123456)
        t = srv.submit(np.zeros(0, np.uint8), np.array([0], np.uint32), 1)
        res = srv.wait(t)
        assert res["status"] == fm.FM_OK and res["offsets"].tolist() == [0]
    h.close()
