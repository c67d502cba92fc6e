"""Python binding of the fmocc C ABI (include/fmocc.h).

Argument marshalling only: every step of the search runs in libfmocc.so's kernels.  Device
buffers are torch CUDA tensors (uint32 values travel in int32 tensors, bit for bit; uint64 in
int64), streams are torch streams.  There is no CPU path: without the built library every call
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libfmocc.so")

FM_OK, FM_EINVAL, FM_ENOMEM, FM_ECUDA, FM_ETRUNC, FM_ETIMEOUT, FM_EIO = range(7)
FM_BUILD_CODES = 1
FM_BUILD_FORWARD_ONLY = 2
FM_BUILD_BOTH_STRANDS = 4
FM_KERNEL_AUTO, FM_KERNEL_PLAIN, FM_KERNEL_PERSISTENT = 0, 1, 2
KMER_AUTO, KMER_OFF = 0xFE, 0xFF
KERNELS = {"auto": FM_KERNEL_AUTO, "plain": FM_KERNEL_PLAIN, "persistent": FM_KERNEL_PERSISTENT}


class FmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fmocc status {code}: {msg}")
        self.code = code


class fm_params(C.Structure):
    _fields_ = [("interval", C.c_uint32), ("flags", C.c_uint32), ("device", C.c_int32),
                ("reserved", C.c_uint32)]


class fm_info_t(C.Structure):
    _fields_ = [("n", C.c_uint64), ("interval", C.c_uint32), ("block_bytes", C.c_uint32),
                ("C", C.c_uint64 * 5), ("dollar_row", C.c_uint64), ("rev_dollar_row", C.c_uint64),
                ("n_blocks", C.c_uint64), ("sa_sample_rate", C.c_uint64),
                ("bytes_device", C.c_uint64), ("has_reverse", C.c_int32), ("device", C.c_int32),
                ("both_strands", C.c_int32), ("reserved", C.c_int32)]


class fm_profile(C.Structure):
    _fields_ = [("ms_dcalc", C.c_float), ("ms_search", C.c_float), ("ms_canon", C.c_float),
                ("ms_total", C.c_float), ("launches", C.c_uint32), ("passes", C.c_uint32),
                ("graph", C.c_uint32), ("fill_counters", C.c_uint32),
                ("exact_steps", C.c_uint64), ("exact_lanes", C.c_uint64),
                ("exact_lanes2", C.c_uint64), ("general_steps", C.c_uint64),
                ("general_lanes", C.c_uint64), ("admissions", C.c_uint64),
                ("admitted", C.c_uint64), ("parked", C.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class fm_search_params(C.Structure):
    _fields_ = [("z", C.c_uint32), ("max_gaps", C.c_uint32), ("strands", C.c_uint32),
                ("kernel", C.c_uint32), ("stats", C.c_void_p),
                ("profile", C.POINTER(fm_profile)), ("costs", C.c_void_p),
                ("best", C.c_uint32), ("indel_end_skip", C.c_uint32)]


class fm_tuning(C.Structure):
    _fields_ = [("warps_per_block", C.c_uint32), ("blocks_per_sm", C.c_uint32),
                ("chunk", C.c_uint32), ("plain_block", C.c_uint32), ("graphs", C.c_uint32),
                ("occ_per_thread", C.c_uint32), ("l2_fetch_bytes", C.c_uint32),
                ("canonical", C.c_uint32), ("kmer_depth", C.c_uint32),
                ("pair_steps", C.c_uint32), ("refill", C.c_uint32), ("chain2_min", C.c_uint32),
                ("stage", C.c_uint32)]


class fm_server_params(C.Structure):
    _fields_ = [("max_batch_reads", C.c_uint32), ("strands", C.c_uint32),
                ("frontier_budget", C.c_uint64), ("kernel", C.c_uint32),
                ("inflight", C.c_uint32)]


class fm_server_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_queries", C.c_uint32),
                ("counts", C.POINTER(C.c_uint32)), ("offsets", C.POINTER(C.c_uint64)),
                ("pairs", C.POINTER(C.c_uint32)), ("t_submit_ns", C.c_uint64),
                ("t_start_ns", C.c_uint64), ("t_done_ns", C.c_uint64),
                ("batch_reads", C.c_uint32), ("batch_id", C.c_uint32)]


# every symbol include/fmocc.h declares
EXPORTS = ["fm_build", "fm_free", "fm_last_error", "fm_info", "fm_get_bwt", "fm_save", "fm_load",
           "fm_occ8", "fm_exact", "fm_dcalc", "fm_inexact", "fm_inexact_fetch", "fm_set_tuning",
           "fm_get_tuning", "fm_inexact_noalloc", "fm_server_start", "fm_server_submit",
           "fm_server_poll", "fm_server_release", "fm_server_stats", "fm_server_stop",
           "fm_probe_gather", "fm_locate"]

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libfmocc.so (raises when it has not been built)."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built: run __graft_entry__.build() (needs nvcc)")
    lib = C.CDLL(path)
    P, u32, u64 = C.c_void_p, C.c_uint32, C.c_uint64
    lib.fm_build.argtypes = [P, u64, C.POINTER(fm_params), C.POINTER(P)]
    lib.fm_free.argtypes = [P]
    lib.fm_free.restype = None
    lib.fm_last_error.argtypes = [P]
    lib.fm_last_error.restype = C.c_char_p
    lib.fm_info.argtypes = [P, C.POINTER(fm_info_t)]
    lib.fm_get_bwt.argtypes = [P, C.c_int, P]
    lib.fm_save.argtypes = [P, C.c_char_p]
    lib.fm_load.argtypes = [C.c_char_p, C.POINTER(fm_params), C.POINTER(P)]
    lib.fm_occ8.argtypes = [P, P, P, P, u64, P]
    lib.fm_exact.argtypes = [P, P, P, u32, P, P, P]
    lib.fm_dcalc.argtypes = [P, P, P, u32, u32, P, P]
    lib.fm_locate.argtypes = [P, P, u64, P, P, P]
    lib.fm_inexact.argtypes = [P, P, P, u32, C.POINTER(fm_search_params), P, P, P, u64,
                               C.POINTER(C.c_uint64), P]
    lib.fm_inexact_fetch.argtypes = [P, P, u64, P]
    lib.fm_inexact_noalloc.argtypes = [P, P, P, u32, C.POINTER(fm_search_params), P, P, P, u64,
                                       C.POINTER(C.c_uint64), P]
    lib.fm_set_tuning.argtypes = [P, C.POINTER(fm_tuning)]
    lib.fm_server_start.argtypes = [P, C.POINTER(fm_server_params), C.POINTER(P)]
    lib.fm_server_submit.argtypes = [P, P, P, u32, u32, u32, C.POINTER(C.c_uint64)]
    lib.fm_server_poll.argtypes = [P, u64, u32, C.POINTER(fm_server_result)]
    lib.fm_server_release.argtypes = [P, u64]
    lib.fm_server_stats.argtypes = [P, P]
    lib.fm_server_stop.argtypes = [P]
    lib.fm_probe_gather.argtypes = [P, u64, u32, u32, u32, u32, u64, P, P]
    lib.fm_get_tuning.argtypes = [P, C.POINTER(fm_tuning)]
    for name in EXPORTS:
        f = getattr(lib, name)
        if name not in ("fm_free", "fm_last_error"):
            f.restype = C.c_int
    if path == LIB_PATH:
        _lib = lib
    return lib


def _check(rc: int, h=None):
    if rc != FM_OK:
        msg = load_library().fm_last_error(h.ptr if h is not None else None)
        raise FmError(rc, (msg or b"").decode(errors="replace"))


def _dptr(t: torch.Tensor | None, dtypes, what: str):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype not in dtypes:
        raise TypeError(f"{what} must have dtype in {dtypes}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return C.c_void_p(t.data_ptr())


_U32 = (torch.int32,) + ((torch.uint32,) if hasattr(torch, "uint32") else ())
_U64 = (torch.int64,) + ((torch.uint64,) if hasattr(torch, "uint64") else ())
_U8 = (torch.uint8,)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Index:
    """Handle of a resident index (fm_index*)."""

    def __init__(self, ptr: int):
        self.ptr = C.c_void_p(ptr)

    def close(self):
        if self.ptr and self.ptr.value:
            load_library().fm_free(self.ptr)
            self.ptr = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # convenience forwards
    def info(self):
        return fm_info(self)

    def occ8(self, k, l, out=None, stream=None):
        return fm_occ8(self, k, l, out, stream)

    def exact(self, reads, offs, stream=None):
        return fm_exact(self, reads, offs, stream=stream)

    def dcalc(self, reads, offs, strands=1, stream=None):
        return fm_dcalc(self, reads, offs, strands, stream=stream)

    def inexact(self, reads, offs, z, max_gaps=0, strands=1, kernel="auto", **kw):
        return fm_inexact(self, reads, offs, z, max_gaps, strands, kernel, **kw)


def fm_build(ref, interval: int = 64, flags: int = 0, device: int = -1,
             forward_only: bool = False, both_strands: bool = False) -> Index:
    """Build the index of ``ref`` (bytes/str over ACGTacgt, or a uint8 numpy array of codes):
    suffix array (Eq. 1), BWT (Eq. 2), C and the interleaved checkpoint table of Sec. 2, and
    the same for reverse(ref), which the D bound needs; with ``both_strands`` the index of
    ref . revcomp(ref)."""
    lib = load_library()
    if isinstance(ref, np.ndarray):
        buf = np.ascontiguousarray(ref, dtype=np.uint8)
        flags |= FM_BUILD_CODES
        ptr, n = buf.ctypes.data_as(C.c_void_p), buf.size
    else:
        if isinstance(ref, str):
            ref = ref.encode()
        buf = ref
        ptr, n = C.c_char_p(buf), len(buf)
    if forward_only:
        flags |= FM_BUILD_FORWARD_ONLY
    if both_strands:
        flags |= FM_BUILD_BOTH_STRANDS
    p = fm_params(interval, flags, device, 0)
    out = C.c_void_p()
    rc = lib.fm_build(C.cast(ptr, C.c_void_p), n, C.byref(p), C.byref(out))
    _check(rc)
    return Index(out.value)


def fm_free(h: Index):
    """Release the index (handle lifetime: no counterpart in the paper)."""
    h.close()


def fm_last_error(h: Index | None = None) -> str:
    """Message of the last failure (error reporting: no counterpart in the paper)."""
    return (load_library().fm_last_error(h.ptr if h is not None else None) or b"").decode()


def fm_info(h: Index) -> dict:
    """Summary of the index: n, the checkpoint layout of Sec. 2, C (Eq. 3), the $ rows."""
    inf = fm_info_t()
    _check(load_library().fm_info(h.ptr, C.byref(inf)), h)
    return {"n": inf.n, "interval": inf.interval, "block_bytes": inf.block_bytes,
            "C": list(inf.C), "dollar_row": inf.dollar_row, "rev_dollar_row": inf.rev_dollar_row,
            "n_blocks": inf.n_blocks, "sa_sample_rate": inf.sa_sample_rate,
            "bytes_device": inf.bytes_device, "has_reverse": bool(inf.has_reverse),
            "device": inf.device, "both_strands": bool(inf.both_strands)}


def fm_get_bwt(h: Index, rev: bool = False) -> np.ndarray:
    """The BWT (Eq. 2, Fig. 1) as host codes 0..3, 4 at the $ row (test access)."""
    n = fm_info(h)["n"]
    out = np.empty(n + 1, dtype=np.uint8)
    _check(load_library().fm_get_bwt(h.ptr, 1 if rev else 0, out.ctypes.data_as(C.c_void_p)), h)
    return out


def fm_save(h: Index, path: str):
    """Write the resident tables of Sec. 2 to a file (persistence: no counterpart in the
    paper)."""
    _check(load_library().fm_save(h.ptr, path.encode()), h)


def fm_load(path: str, device: int = -1) -> Index:
    """Load a file fm_save wrote onto a device (persistence: no counterpart in the paper)."""
    p = fm_params(0, 0, device, 0)
    out = C.c_void_p()
    _check(load_library().fm_load(path.encode(), C.byref(p), C.byref(out)))
    return Index(out.value)


def fm_occ8(h: Index, k: torch.Tensor, l: torch.Tensor, out: torch.Tensor | None = None,
            stream=None) -> torch.Tensor:
    """out[q] = [Occ(A..T, k[q]-1), Occ(A..T, l[q])] as an int32 [N, 8] CUDA tensor: the eight
    Occ values of one backward-search step in one pass (Sec. 2 closing remarks, Sec. 3.3)."""
    N = k.numel()
    if l.numel() != N:
        raise ValueError("k and l differ in length")
    if out is None:
        out = torch.empty((N, 8), dtype=torch.int32, device=k.device)
    rc = load_library().fm_occ8(h.ptr, _dptr(k, _U32, "k"), _dptr(l, _U32, "l"),
                                _dptr(out, _U32, "out"), N, _stream(stream))
    _check(rc, h)
    return out


def fm_exact(h: Index, reads: torch.Tensor, offs: torch.Tensor, k_out=None, l_out=None,
             stream=None):
    """Listing 1 intervals (k, l) per read, int32 CUDA tensors."""
    nr = offs.numel() - 1
    dev = offs.device
    if k_out is None:
        k_out = torch.empty(nr, dtype=torch.int32, device=dev)
    if l_out is None:
        l_out = torch.empty(nr, dtype=torch.int32, device=dev)
    rc = load_library().fm_exact(h.ptr, _dptr(reads, _U8, "reads"), _dptr(offs, _U32, "offs"), nr,
                                 _dptr(k_out, _U32, "k_out"), _dptr(l_out, _U32, "l_out"),
                                 _stream(stream))
    _check(rc, h)
    return k_out, l_out


def fm_locate(h: Index, rows: torch.Tensor, pos_out: torch.Tensor | None = None,
              steps: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """SA[row] for each row (int32 CUDA tensor of the same length), by Psi^-1 walks to a sampled
    row (Sec. 2, Eq. 4-5)."""
    N = rows.numel()
    if pos_out is None:
        pos_out = torch.empty(N, dtype=torch.int32, device=rows.device)
    rc = load_library().fm_locate(h.ptr, _dptr(rows, _U32, "rows"), N,
                                  _dptr(pos_out, _U32, "pos_out"),
                                  _dptr(steps, _U64, "steps") if steps is not None else None,
                                  _stream(stream))
    _check(rc, h)
    return pos_out


def fm_dcalc(h: Index, reads: torch.Tensor, offs: torch.Tensor, strands: int = 1, D_out=None,
             stream=None) -> torch.Tensor:
    """The D lower bound of the inexact search (Li and Durbin 2009, cited with Listing 2), one
    uint8 per query symbol, by forward extension on the index of reverse(R)."""
    nr = offs.numel() - 1
    total = int(reads.numel()) * strands
    if D_out is None:
        D_out = torch.empty(max(total, 1), dtype=torch.uint8, device=offs.device)
    rc = load_library().fm_dcalc(h.ptr, _dptr(reads, _U8, "reads"), _dptr(offs, _U32, "offs"), nr,
                                 strands, _dptr(D_out, _U8, "D_out"), _stream(stream))
    _check(rc, h)
    return D_out[:total]


def fm_inexact(h: Index, reads: torch.Tensor, offs: torch.Tensor, z: int, max_gaps: int = 0,
               strands: int = 1, kernel="auto", stats: torch.Tensor | None = None,
               pair_capacity: int | None = None, counts=None, offsets=None, pairs=None,
               profile: fm_profile | None = None, stream=None, costs=False, best=False,
               end_skip: int = 0):
    """Listing 2 interval sets.  Returns (counts int32[nq], offsets int64[nq+1],
    pairs int32[total, 2]), plus costs uint8[total] (per interval the fewest differences) when
    ``costs`` is True or a uint8 tensor; ``best`` keeps only each query's minimum-cost
    intervals; ``end_skip`` > 0 places indel columns only where at least that many query
    symbols lie on each side of them.  On FM_ETRUNC the pairs buffer is regrown and fetched
    again (or, with costs or best, the call is repeated with larger buffers)."""
    lib = load_library()
    nr = offs.numel() - 1
    nq = nr * strands
    dev = offs.device
    kern = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    if counts is None:
        counts = torch.empty(max(nq, 1), dtype=torch.int32, device=dev)
    if offsets is None:
        offsets = torch.empty(nq + 1, dtype=torch.int64, device=dev)
    if pairs is None:
        cap = pair_capacity if pair_capacity is not None else 4 * nq + 1024
        pairs = torch.empty((max(cap, 1), 2), dtype=torch.int32, device=dev)
    cap = pairs.shape[0]
    want_costs = costs is not False and costs is not None
    if want_costs and not isinstance(costs, torch.Tensor):
        costs = torch.empty(max(cap, 1), dtype=torch.uint8, device=dev)
    if want_costs and costs.numel() < cap:
        raise ValueError("costs must hold pair capacity entries")

    def call(with_stats=True):
        sp = fm_search_params(z, max_gaps, strands, kern,
                              _dptr(stats, _U64, "stats") if stats is not None and with_stats
                              else None,
                              C.pointer(profile) if profile is not None else None,
                              _dptr(costs, _U8, "costs") if want_costs else None,
                              1 if best else 0, end_skip)
        need = C.c_uint64(0)
        rc = lib.fm_inexact(h.ptr, _dptr(reads, _U8, "reads"), _dptr(offs, _U32, "offs"), nr,
                            C.byref(sp), _dptr(counts, _U32, "counts"),
                            _dptr(offsets, _U64, "offsets"), _dptr(pairs, _U32, "pairs"),
                            pairs.shape[0], C.byref(need), _stream(stream))
        return rc, int(need.value)

    rc, need = call()
    if rc == FM_ETRUNC and (want_costs or best):
        # counts and offsets are complete and the truncated call already added its stats:
        # repeat with buffers of the needed size, without stats
        pairs = torch.empty((max(need, 1), 2), dtype=torch.int32, device=dev)
        if want_costs:
            costs = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
        rc, need = call(with_stats=False)
    elif rc == FM_ETRUNC:
        pairs = torch.empty((max(need, 1), 2), dtype=torch.int32, device=dev)
        rc = lib.fm_inexact_fetch(h.ptr, _dptr(pairs, _U32, "pairs"), pairs.shape[0],
                                  _stream(stream))
    _check(rc, h)
    if want_costs:
        return counts[:nq], offsets, pairs[:need], costs[:need]
    return counts[:nq], offsets, pairs[:need]


def fm_inexact_noalloc(h: Index, reads: torch.Tensor, offs: torch.Tensor, z: int,
                       max_gaps: int = 0, strands: int = 1, counts=None, offsets=None,
                       pairs=None, stream=None, end_skip: int = 0):
    """fm_inexact (Listing 2) without device allocation inside the library (fixed static
    scratch; at most 32,768 queries per call).  The caller provides (or this wrapper allocates through torch,
    before the call) the output buffers.  Returns (counts, offsets, pairs, status); status is
    FM_ETRUNC when ``pairs`` is too small (counts and offsets are then complete)."""
    lib = load_library()
    nr = offs.numel() - 1
    nq = nr * strands
    dev = offs.device
    if counts is None:
        counts = torch.empty(max(nq, 1), dtype=torch.int32, device=dev)
    if offsets is None:
        offsets = torch.empty(nq + 1, dtype=torch.int64, device=dev)
    if pairs is None:
        pairs = torch.empty((4 * nq + 1024, 2), dtype=torch.int32, device=dev)
    sp = fm_search_params(z, max_gaps, strands, FM_KERNEL_PERSISTENT, None, None, None, 0,
                          end_skip)
    need = C.c_uint64(0)
    rc = lib.fm_inexact_noalloc(h.ptr, _dptr(reads, _U8, "reads"), _dptr(offs, _U32, "offs"), nr,
                                C.byref(sp), _dptr(counts, _U32, "counts"),
                                _dptr(offsets, _U64, "offsets"), _dptr(pairs, _U32, "pairs"),
                                pairs.shape[0], C.byref(need), _stream(stream))
    if rc not in (FM_OK, FM_ETRUNC):
        _check(rc, h)
    return counts[:nq], offsets, pairs[:min(int(need.value), pairs.shape[0])], rc


def fm_inexact_fetch(h: Index, pairs: torch.Tensor, stream=None):
    """Copy the Listing 2 interval sets of the last fm_inexact call into ``pairs``."""
    _check(load_library().fm_inexact_fetch(h.ptr, _dptr(pairs, _U32, "pairs"), pairs.shape[0],
                                           _stream(stream)), h)
    return pairs


def fm_set_tuning(h: Index, warps_per_block=0, blocks_per_sm=0, chunk=0, plain_block=0,
                  graphs=0, occ_per_thread=0, l2_fetch_bytes=0, canonical=0, kmer_depth=0,
                  pair_steps=0, refill=0, chain2_min=0, stage=0):
    """Zero keeps a knob; graphs, canonical and pair_steps: 1 on, 2 off; kmer_depth: 1..15,
    KMER_AUTO or KMER_OFF.  Speed and memory only, never results (the tables and pair steps
    answer the cache-locality question of Sec. 4.2; the rest have no counterpart in the
    paper)."""
    t = fm_tuning(warps_per_block, blocks_per_sm, chunk, plain_block, graphs, occ_per_thread,
                  l2_fetch_bytes, canonical, kmer_depth, pair_steps, refill, chain2_min, stage)
    _check(load_library().fm_set_tuning(h.ptr, C.byref(t)), h)


def fm_get_tuning(h: Index) -> dict:
    """The knobs in effect (see fm_set_tuning)."""
    t = fm_tuning()
    _check(load_library().fm_get_tuning(h.ptr, C.byref(t)), h)
    return {"warps_per_block": t.warps_per_block, "blocks_per_sm": t.blocks_per_sm,
            "chunk": t.chunk, "plain_block": t.plain_block, "graphs": t.graphs,
            "occ_per_thread": t.occ_per_thread, "l2_fetch_bytes": t.l2_fetch_bytes,
            "canonical": t.canonical, "kmer_depth": t.kmer_depth, "pair_steps": t.pair_steps,
            "refill": t.refill, "chain2_min": t.chain2_min, "stage": t.stage}


def fm_probe_gather(buf: torch.Tensor, granule: int, threads: int, per_thread: int,
                    seed: int = 1, sink: torch.Tensor | None = None, stream=None,
                    inflight: int = 4):
    """Random-gather probe over a CUDA buffer (measurement only: no counterpart in the paper)."""
    if sink is None:
        sink = torch.empty(threads, dtype=torch.int32, device=buf.device)
    rc = load_library().fm_probe_gather(C.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size(),
                                        granule, threads, per_thread, inflight, seed,
                                        _dptr(sink, _U32, "sink"), _stream(stream))
    _check(rc)
    return sink


class Server:
    """Request loop over a resident index (fm_server_*; serving has no counterpart in the paper,
    each request runs the search of Listing 2): submit host read batches, poll for their
    interval sets.  While it runs, the index handle belongs to the server."""

    def __init__(self, h: Index, max_batch_reads: int = 0, strands: int = 2,
                 frontier_budget: int = 0, kernel="persistent", inflight: int = 0):
        self.lib = load_library()
        self.h = h
        self.strands = strands
        kern = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        p = fm_server_params(max_batch_reads, strands, frontier_budget, kern, inflight)
        out = C.c_void_p()
        _check(self.lib.fm_server_start(h.ptr, C.byref(p), C.byref(out)), h)
        self.ptr = out

    def submit(self, codes: np.ndarray, offs: np.ndarray, z: int, max_gaps: int = 0) -> int:
        codes = np.ascontiguousarray(codes, dtype=np.uint8)
        offs = np.ascontiguousarray(offs, dtype=np.uint32)
        t = C.c_uint64(0)
        _check(self.lib.fm_server_submit(self.ptr, codes.ctypes.data_as(C.c_void_p),
                                         offs.ctypes.data_as(C.c_void_p), offs.size - 1, z,
                                         max_gaps, C.byref(t)))
        return t.value

    def poll(self, ticket: int, wait_ms: int = 0):
        """None while not done; else a dict with counts, offsets, pairs and times (ns)."""
        r = fm_server_result()
        rc = self.lib.fm_server_poll(self.ptr, ticket, wait_ms, C.byref(r))
        if rc == FM_ETIMEOUT:
            return None
        _check(rc)
        nq = r.n_queries
        offsets = np.ctypeslib.as_array(r.offsets, shape=(nq + 1,)).copy()
        tot = int(offsets[-1])
        out = {"status": r.status,
               "counts": (np.ctypeslib.as_array(r.counts, shape=(nq,)).copy() if nq
                          else np.zeros(0, np.uint32)),
               "offsets": offsets,
               "pairs": (np.ctypeslib.as_array(r.pairs, shape=(2 * tot,)).reshape(tot, 2).copy()
                         if tot else np.zeros((0, 2), np.uint32)),
               "t_submit_ns": r.t_submit_ns, "t_start_ns": r.t_start_ns,
               "t_done_ns": r.t_done_ns, "batch_reads": r.batch_reads,
               "batch_id": r.batch_id}
        _check(self.lib.fm_server_release(self.ptr, ticket))
        return out

    def wait(self, ticket: int, timeout_ms: int = 600_000):
        res = self.poll(ticket, timeout_ms)
        if res is None:
            raise FmError(FM_ETIMEOUT, f"request {ticket} not done after {timeout_ms} ms")
        return res

    def stats(self):
        a = np.zeros(4, dtype=np.uint64)
        _check(self.lib.fm_server_stats(self.ptr, a.ctypes.data_as(C.c_void_p)))
        return {"batches": int(a[0]), "reads": int(a[1]), "requests": int(a[2]),
                "busy_ms": int(a[3])}

    def stop(self):
        if self.ptr and self.ptr.value:
            self.lib.fm_server_stop(self.ptr)
            self.ptr = C.c_void_p(None)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.stop()


# ---------------------------------------------------------------------------------------------
# host-side helpers (marshalling of read batches)
# ---------------------------------------------------------------------------------------------

def to_device_reads(reads, device="cuda"):
    """(codes uint8, offs int32) CUDA tensors from a synth.Reads batch."""
    codes = torch.from_numpy(np.ascontiguousarray(reads.codes)).to(device)
    offs = torch.from_numpy(np.ascontiguousarray(reads.offs).view(np.int32)).to(device)
    return codes, offs
