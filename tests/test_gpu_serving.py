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


def test_server_errors(fm):
    R = synth.uniform_text(3, 50_000)
    h = fm.fm_build(R)
    with fm.Server(h, strands=2) as srv:
        with pytest.raises(fm.FmError):
            srv.submit(np.array([0, 9], np.uint8), np.array([0, 2], np.uint32), 1)
        with pytest.raises(fm.FmError):
            srv.poll(123456)
        t = srv.submit(np.zeros(0, np.uint8), np.array([0], np.uint32), 1)
        res = srv.wait(t)
        assert res["status"] == fm.FM_OK and res["offsets"].tolist() == [0]
    h.close()
