"""ctypes front end of the CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()`` and by the
benchmark's CPU-baseline leg.  The product package never imports it.

The shared library is compiled on first use (plain gcc, no CUDA), or by ``build()``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False, extra_flags=(), out: str | None = None) -> str:
    """Compile oracle.c into a shared library and return its path."""
    so = out or _SO
    stale = (not os.path.exists(so) or
             os.path.getmtime(so) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale or out is not None:
        cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", *extra_flags,
               "-o", so + ".tmp", _SRC]
        subprocess.run(cmd, check=True)
        os.replace(so + ".tmp", so)
    return so


class _Results(C.Structure):
    _fields_ = [("nq", C.c_int64), ("counts", C.POINTER(C.c_uint32)),
                ("offsets", C.POINTER(C.c_uint64)), ("pairs", C.POINTER(C.c_uint32)),
                ("costs", C.POINTER(C.c_uint8)),
                ("nodes", C.POINTER(C.c_uint64)), ("blocks", C.POINTER(C.c_uint64)),
                ("total", C.c_uint64)]


def _declare(lib):
    P = C.c_void_p
    i64 = C.c_int64
    lib.or_sa_naive.argtypes = [P, i64, P]
    lib.or_sa_sais.argtypes = [P, i64, P]
    lib.or_sa_sais.restype = C.c_int
    lib.or_bwt.argtypes = [P, i64, P, P]
    lib.or_bwt.restype = i64
    lib.or_count.argtypes = [P, i64, P]
    lib.or_occ_scan.argtypes = [P, i64, C.c_int, i64]
    lib.or_occ_scan.restype = i64
    lib.or_index_new.argtypes = [P, i64, C.c_int]
    lib.or_index_new.restype = P
    lib.or_index_free.argtypes = [P]
    lib.or_index_sa.argtypes = [P]
    lib.or_index_sa.restype = P
    lib.or_index_bwt.argtypes = [P]
    lib.or_index_bwt.restype = P
    lib.or_index_c.argtypes = [P, P]
    lib.or_index_dollar_row.argtypes = [P]
    lib.or_index_dollar_row.restype = i64
    lib.or_occ4.argtypes = [P, i64, P]
    lib.or_occ8_batch.argtypes = [P, P, P, i64, P, C.c_int]
    lib.or_occ8_batch.restype = C.c_int
    lib.or_occ8_sweep.argtypes = [P, i64, P, P, i64, P]
    lib.or_occ8_sweep.restype = C.c_int
    lib.or_exact_batch.argtypes = [P, P, P, i64, P, P, C.c_int]
    lib.or_exact_batch.restype = C.c_int
    lib.or_interval_naive_batch.argtypes = [P, i64, P, P, i64, P, P, P, C.c_int]
    lib.or_dcalc.argtypes = [P, P, i64, P]
    lib.or_inexact_batch.argtypes = [P, P, P, i64, C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.c_int, C.c_int, C.c_int]
    lib.or_inexact_batch.restype = C.POINTER(_Results)
    lib.or_results_free.argtypes = [C.POINTER(_Results)]
    lib.or_hamming_count.argtypes = [P, i64, P, i64, C.c_int]
    lib.or_hamming_count.restype = i64
    lib.or_default_threads.restype = C.c_int


def load(path: str | None = None):
    """Load (building if needed) the oracle library; a path loads a specific build."""
    global _lib
    if path is not None:
        lib = C.CDLL(path)
        _declare(lib)
        return lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB points the tests at another build of oracle.c (planted-mistake tests)
            alt = os.environ.get("ORACLE_LIB")
            lib = C.CDLL(alt if alt else build())
            _declare(lib)
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def sa_naive(R, lib=None) -> np.ndarray:
    lib = lib or load()
    R = _u8(R)
    SA = np.empty(R.size + 1, dtype=np.int64)
    lib.or_sa_naive(_p(R), R.size, _p(SA))
    return SA


def sa_sais(R, lib=None) -> np.ndarray:
    lib = lib or load()
    R = _u8(R)
    SA = np.empty(R.size + 1, dtype=np.int64)
    if lib.or_sa_sais(_p(R), R.size, _p(SA)) != 0:
        raise MemoryError("or_sa_sais")
    return SA


def bwt(R, SA, lib=None):
    lib = lib or load()
    R = _u8(R)
    SA = np.ascontiguousarray(SA, dtype=np.int64)
    L = np.empty(R.size + 1, dtype=np.uint8)
    d = lib.or_bwt(_p(R), R.size, _p(SA), _p(L))
    return L, int(d)


def count(R, lib=None) -> np.ndarray:
    lib = lib or load()
    R = _u8(R)
    Cc = np.zeros(5, dtype=np.int64)
    lib.or_count(_p(R), R.size, _p(Cc))
    return Cc


def occ_scan(L, b: int, k: int, lib=None) -> int:
    lib = lib or load()
    L = _u8(L)
    return int(lib.or_occ_scan(_p(L), L.size - 1, b, k))


def hamming_count(R, W, z: int, lib=None) -> int:
    lib = lib or load()
    R = _u8(R)
    W = _u8(W)
    return int(lib.or_hamming_count(_p(R), R.size, _p(W), W.size, z))


def interval_naive(R, codes, offs, threads: int = 0, lib=None):
    """Closed-form exact intervals and their eight Occ values by scanning every suffix."""
    lib = lib or load()
    R = _u8(R)
    codes = _u8(codes)
    offs = np.ascontiguousarray(offs, dtype=np.uint32)
    npat = offs.size - 1
    k = np.empty(npat, dtype=np.int64)
    l = np.empty(npat, dtype=np.int64)
    o8 = np.empty((npat, 8), dtype=np.int64)
    lib.or_interval_naive_batch(_p(R), R.size, _p(codes), _p(offs), npat, _p(k), _p(l), _p(o8),
                                threads)
    return k, l, o8


def default_threads(lib=None) -> int:
    lib = lib or load()
    return int(lib.or_default_threads())


class Index:
    """Oracle FM-index of a code text (method 'naive' or 'sais')."""

    def __init__(self, R, method: str = "sais", lib=None):
        self.lib = lib or load()
        self.R = _u8(R)          # kept alive: the C index borrows it
        self.n = int(self.R.size)
        m = {"naive": 0, "sais": 1}[method]
        self.h = self.lib.or_index_new(_p(self.R), self.n, m)
        if not self.h:
            raise MemoryError("or_index_new")

    def close(self):
        if self.h:
            self.lib.or_index_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def sa(self) -> np.ndarray:
        ptr = C.cast(self.lib.or_index_sa(self.h), C.POINTER(C.c_int64))
        return np.ctypeslib.as_array(ptr, shape=(self.n + 1,)).copy()

    @property
    def bwt(self) -> np.ndarray:
        ptr = C.cast(self.lib.or_index_bwt(self.h), C.POINTER(C.c_uint8))
        return np.ctypeslib.as_array(ptr, shape=(self.n + 1,)).copy()

    @property
    def C(self) -> np.ndarray:
        out = np.zeros(5, dtype=np.int64)
        self.lib.or_index_c(self.h, _p(out))
        return out

    @property
    def dollar_row(self) -> int:
        return int(self.lib.or_index_dollar_row(self.h))

    def occ4(self, k: int) -> np.ndarray:
        out = np.zeros(4, dtype=np.int64)
        self.lib.or_occ4(self.h, k, _p(out))
        return out

    def occ8(self, k, l, threads: int = 0) -> np.ndarray:
        k = np.ascontiguousarray(k, dtype=np.uint32)
        l = np.ascontiguousarray(l, dtype=np.uint32)
        out = np.empty((k.size, 8), dtype=np.uint32)
        if self.lib.or_occ8_batch(self.h, _p(k), _p(l), k.size, _p(out), threads) != 0:
            raise ValueError("occ8 query outside 0<=k<=n+1, 0<=l<=n")
        return out

    def occ8_sweep(self, k, l) -> np.ndarray:
        k = np.ascontiguousarray(k, dtype=np.uint32)
        l = np.ascontiguousarray(l, dtype=np.uint32)
        out = np.empty((k.size, 8), dtype=np.uint32)
        L = self.bwt
        if self.lib.or_occ8_sweep(_p(L), self.n, _p(k), _p(l), k.size, _p(out)) != 0:
            raise ValueError("occ8_sweep domain or memory")
        return out

    def exact(self, codes, offs, threads: int = 0):
        codes = _u8(codes)
        offs = np.ascontiguousarray(offs, dtype=np.uint32)
        nr = offs.size - 1
        k = np.empty(nr, dtype=np.uint32)
        l = np.empty(nr, dtype=np.uint32)
        if self.lib.or_exact_batch(self.h, _p(codes), _p(offs), nr, _p(k), _p(l), threads) != 0:
            raise ValueError("read code outside 0..3")
        return k, l

    def dcalc(self, W) -> np.ndarray:
        W = _u8(W)
        D = np.empty(W.size, dtype=np.uint8)
        self.lib.or_dcalc(self.h, _p(W), W.size, _p(D))
        return D

    def inexact(self, codes, offs, z: int, max_gaps: int = 0, strands: int = 1,
                prune: bool = True, interval: int = 64, threads: int = 0,
                canonical: bool = False, end_skip: int = 0):
        """Listing 2 result sets: dict with counts, offsets, pairs (total x 2), costs (per
        interval the fewest differences of the alignments reaching it), nodes, blocks.
        canonical: enumerate canonical alignments only (same results; nodes and blocks are
        those of that enumeration).  end_skip: indel columns only with at least that many
        read symbols on each side (not with canonical)."""
        codes = _u8(codes)
        offs = np.ascontiguousarray(offs, dtype=np.uint32)
        nr = offs.size - 1
        res = self.lib.or_inexact_batch(self.h, _p(codes), _p(offs), nr, strands, z, max_gaps,
                                        (1 if prune else 0) | (2 if canonical else 0),
                                        interval, threads, end_skip)
        if not res:
            raise ValueError("or_inexact_batch")
        try:
            r = res.contents
            nq = int(r.nq)
            tot = int(r.total)
            out = {
                "counts": np.ctypeslib.as_array(r.counts, shape=(max(nq, 1),))[:nq].copy(),
                "offsets": np.ctypeslib.as_array(r.offsets, shape=(nq + 1,)).copy(),
                "pairs": np.ctypeslib.as_array(r.pairs, shape=(max(2 * tot, 2),))[:2 * tot]
                .reshape(tot, 2).copy(),
                "costs": np.ctypeslib.as_array(r.costs, shape=(max(tot, 1),))[:tot].copy(),
                "nodes": np.ctypeslib.as_array(r.nodes, shape=(max(nq, 1),))[:nq].copy(),
                "blocks": np.ctypeslib.as_array(r.blocks, shape=(max(nq, 1),))[:nq].copy(),
            }
        finally:
            self.lib.or_results_free(res)
        return out
