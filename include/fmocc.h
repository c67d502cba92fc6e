/*
 * fmocc: FM-index search on one NVIDIA GB300 (sm_103a).
 *
 * The operations follow R. Snytsar, "Vectorized Character Counting for Faster Pattern
 * Matching" (arXiv 1811.06127):
 *   - Sec. 2 (Eq. 1-3, Fig. 1): suffix array, BWT, C and Occ of a reference R over {A,C,G,T};
 *   - Listing 1: exact backward search; Listing 2: inexact (bounded-difference) search;
 *   - Sec. 2 (closing remarks) and Sec. 3.3: one search step consumes eight Occ values,
 *     Occ(c, k-1) and Occ(c, l) for c in ACGT, which this library computes in one pass over
 *     one interleaved checkpoint block (two when k and l+1 fall in different blocks).
 *
 * Conventions shared by every call:
 *   - Symbol codes A=0, C=1, G=2, T=3 (the 2-bit code of Fig. 2).  The terminator $ is
 *     implicit at the end of R and is smaller than every symbol.
 *   - Rows of the Burrows-Wheeler matrix run 0..n (n+1 rows); row 0 is the suffix "$".
 *   - Occ(c,k) = occurrences of c in BWT[0..k] inclusive, k in [-1, n]; Occ(c,-1) = 0;
 *     $ counts for no symbol.  C[c] = symbols of R smaller than c; C[4] = n.
 *   - An SA interval [k, l] holds the rows whose suffix starts with the searched string;
 *     k = l + 1 denotes an empty interval (the insertion point).
 *   - Pointers documented as "device" must point to memory of the index's device (e.g. torch
 *     CUDA tensors); "host" pointers to ordinary host memory.  The caller owns every buffer
 *     it passes; the index owns its own device memory (the resident tables and the scratch
 *     it grows on demand) until fm_free.
 *   - `stream` is a cudaStream_t (NULL: the legacy default stream).  Compute calls enqueue
 *     their kernels on it and then synchronise it, so that the returned status covers the
 *     device work; outputs are complete when the call returns FM_OK.
 *   - Every call returns a status; fm_last_error() returns a message for the last failure.
 *   - An index handle is not thread-safe: calls on one handle must not overlap.
 */
#ifndef FMOCC_H
#define FMOCC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum fm_status {
    FM_OK = 0,
    FM_EINVAL = 1,   /* an argument or an input symbol is outside the documented domain */
    FM_ENOMEM = 2,   /* a device or host allocation failed */
    FM_ECUDA = 3,    /* a CUDA runtime call failed (message in fm_last_error) */
    FM_ETRUNC = 4,   /* an output buffer is too small; the needed size has been written */
    FM_ETIMEOUT = 5, /* a bounded wait expired */
    FM_EIO = 6       /* file I/O or a corrupt index file */
};

typedef struct fm_index fm_index;

/* Build options. */
typedef struct fm_params {
    uint32_t interval; /* checkpoint interval I: 32 or 64 (32-byte blocks), 128 (64-byte
                          blocks) or 256 (96-byte blocks); 0 means 64 */
    uint32_t flags;    /* FM_BUILD_* bits */
    int32_t device;    /* CUDA device ordinal; -1 = the calling thread's current device */
    uint32_t reserved;
} fm_params;

#define FM_BUILD_CODES 1u        /* ref holds codes 0..3 instead of ASCII ACGTacgt */
#define FM_BUILD_FORWARD_ONLY 2u /* skip the index of reverse(R): fm_dcalc and fm_inexact
                                    then return FM_EINVAL */
#define FM_BUILD_BOTH_STRANDS 4u /* index the text T = R . revcomp(R) (length 2|R|, with
                                    revcomp(R)[i] = 3 - R[|R|-1-i]) in place of R: one query
                                    (strands = 1) then finds the occurrences on both strands.
                                    Rows, intervals and locate positions are those of T (a
                                    position p >= |R| is on the reverse strand; occurrences
                                    that straddle the junction at |R| are occurrences of T).
                                    Requires |R| <= 1,073,741,823 */

/* Summary of a built index (fm_info). */
typedef struct fm_info_t {
    uint64_t n;              /* indexed text length: |R|, or 2|R| with FM_BUILD_BOTH_STRANDS */
    uint32_t interval;       /* checkpoint interval I */
    uint32_t block_bytes;    /* bytes per checkpoint block: 32 (I = 32, 64), 64 or 96 */
    uint64_t C[5];           /* C array (Fig. 1) */
    uint64_t dollar_row;     /* row of the forward BWT holding $ */
    uint64_t rev_dollar_row; /* the same for reverse(R) (0 without a reverse index) */
    uint64_t n_blocks;       /* checkpoint blocks per index: (n+1)/I + 1 */
    uint64_t sa_sample_rate; /* stride of the sampled suffix array kept on the device */
    uint64_t bytes_device;   /* device bytes held by the resident tables */
    int32_t has_reverse;
    int32_t device;
    int32_t both_strands;    /* 1: built with FM_BUILD_BOTH_STRANDS (n is then 2|R|) */
    int32_t reserved;
} fm_info_t;

/* Build the FM-index of R (Sec. 2: Eq. 1 suffix array, Eq. 2 BWT, C, and the checkpointed
 * Occ table laid out as interleaved blocks, after the bucket layout described in Sec. 2) and,
 * unless FM_BUILD_FORWARD_ONLY, the same for reverse(R), which the D lower bound of the
 * inexact search needs.  The tables stay resident in device memory.
 *   ref   host, n bytes: ASCII ACGTacgt, or codes 0..3 with FM_BUILD_CODES.
 *   n     1 <= n <= 2,147,483,646.
 *   p     may be NULL (interval 64, both indexes, current device).
 *   out   receives the handle.
 * Errors: FM_EINVAL (bad symbol, n or interval), FM_ENOMEM, FM_ECUDA.  On error *out is
 * NULL and fm_last_error(NULL) holds the message. */
int fm_build(const char *ref, uint64_t n, const fm_params *p, fm_index **out);

/* Release the index and all device memory it holds (handle lifetime: no counterpart in the
 * paper).  NULL is ignored. */
void fm_free(fm_index *h);

/* Message for the last failure on h, or of the last failed fm_build/fm_load on this thread
 * when h is NULL (error reporting: no counterpart in the paper).  The string lives until the
 * next call on the same handle/thread. */
const char *fm_last_error(const fm_index *h);

/* Fill *out with the summary of h: n, the checkpoint interval and layout of Sec. 2, C (Eq. 3),
 * the $ rows and the device bytes.  Errors: FM_EINVAL. */
int fm_info(const fm_index *h, fm_info_t *out);

/* Copy the BWT (Eq. 2, Fig. 1) back to the host (test access).  bwt: host, n+1 bytes, codes
 * 0..3 with 4 at the $ row.  rev != 0 selects the reverse index.  Errors: FM_EINVAL. */
int fm_get_bwt(const fm_index *h, int rev, uint8_t *bwt);

/* Save the resident tables of Sec. 2 to a file (header with n, I, C, $ rows, sizes, then the
 * tables, then a 64-bit FNV-1a checksum) and load them back on a device (persistence: no
 * counterpart in the paper).  fm_load reads a file fm_save wrote; p selects the device.
 * Errors: FM_EIO (open/write/read, bad magic or checksum), FM_ENOMEM, FM_ECUDA. */
int fm_save(const fm_index *h, const char *path);
int fm_load(const char *path, const fm_params *p, fm_index **out);

/* The eight Occ values of one inexact step (Sec. 2, closing remarks of Listing 2; Sec. 3.3),
 * for N queries:
 *   out8[8q+c]   = Occ(c, k[q]-1)   c = A,C,G,T
 *   out8[8q+4+c] = Occ(c, l[q])
 * k, l: device uint32[N] with 0 <= k[q] <= n+1 and 0 <= l[q] <= n.  out8: device uint32[8N].
 * N may be 0.  Queries outside the domain write zeros and make the call return FM_EINVAL. */
int fm_occ8(fm_index *h, const uint32_t *k, const uint32_t *l, uint32_t *out8, uint64_t N,
            void *stream);

/* Listing 1 (ExactRecur) for each read from the whole range [0, n] (Eq. 3 read as one step
 * of Listing 1), without early exit: an absent read ends with k_out = l_out + 1.
 * reads: device uint8, the concatenated codes (0..3) of n_reads reads;
 * offs:  device uint32[n_reads+1], read r = reads[offs[r] .. offs[r+1]);
 * k_out, l_out: device uint32[n_reads].
 * Errors: FM_EINVAL (a code above 3; such reads return k = 0, l = n). */
int fm_exact(fm_index *h, const uint8_t *reads, const uint32_t *offs, uint32_t n_reads,
             uint32_t *k_out, uint32_t *l_out, void *stream);

/* Per-call profile of fm_inexact (optional): phase times from CUDA events recorded on the
 * call's stream around the library's own launches, and the number of kernels launched.
 * With fill_counters set to 1 by the caller (an input; the call keeps it), the persistent
 * kernel also counts how full its warp steps were (measurement only, no counterpart in the
 * paper; the counting adds a few instructions per step). */
typedef struct fm_profile {
    float ms_dcalc;    /* D lower bound (one launch) */
    float ms_search;   /* the search kernel (last pass when scratch had to be regrown) */
    float ms_canon;    /* grouping, sorting, deduplication and compaction of the intervals */
    float ms_total;    /* whole call, first launch to last */
    uint32_t launches; /* kernels launched by the call */
    uint32_t passes;   /* search passes (1 unless scratch was regrown) */
    uint32_t graph;    /* 1 when the call replayed a captured CUDA graph, 0 when eager */
    uint32_t fill_counters; /* in: 1 to collect the counters below (persistent kernel) */
    uint64_t exact_steps;   /* warp steps over exact continuations (z = 0 chains) */
    uint64_t exact_lanes;   /*   lanes stepping their first chain, summed over those steps */
    uint64_t exact_lanes2;  /*   lanes stepping their second chain, summed */
    uint64_t general_steps; /* warp steps of the full eight-Occ expansion */
    uint64_t general_lanes; /*   lanes expanding a node, summed */
    uint64_t admissions;    /* chunks of queries taken from the work queue */
    uint64_t admitted;      /* queries admitted with a root node (length >= 1, z >= D) */
    uint64_t parked;        /* exact steps in which sparse second chains waited */
} fm_profile;

/* Locate (Sec. 2, Eq. 4-5): pos_out[q] = SA[rows[q]], the text position of the suffix in
 * that row, recovered from the suffix array kept at rows that are multiples of 32
 * (fm_info.sa_sample_rate) by applying Psi^-1(i) = C[BWT[i]] + Occ(BWT[i], i) (Eq. 4) until a
 * sampled row (or the $ row, whose suffix starts at 0) is reached j steps later, then
 * SA[row] = SA[sampled] + j (Eq. 5).  Every row of an interval from fm_exact/fm_inexact is one
 * occurrence of the searched string at that position.
 * rows: device uint32[N], each <= n.  pos_out: device uint32[N].  steps: optional device
 * uint64 counter to which the total number of Psi^-1 steps is added.
 * Errors: FM_EINVAL (a row above n: its position reads 0). */
int fm_locate(fm_index *h, const uint32_t *rows, uint64_t N, uint32_t *pos_out, uint64_t *steps,
              void *stream);

/* Inexact search options. */
typedef struct fm_search_params {
    uint32_t z;        /* differences allowed, 0..7 */
    uint32_t max_gaps; /* indel columns allowed among them (0: mismatches only), 0..7 */
    uint32_t strands;  /* 1: reads as given; 2: each read and its reverse complement, as
                          queries q = 2r (read) and q = 2r+1 (reverse complement) */
    uint32_t kernel;   /* FM_KERNEL_* */
    uint64_t *stats;   /* optional device uint64[4], accumulated by each call that completes
                          its search (FM_OK, or FM_ETRUNC with counts and offsets filled):
                          [0] nodes expanded (calls of InexRecur reaching the Occ step; with
                              fm_tuning.canonical on, those of the canonical enumeration),
                          [1] checkpoint blocks read by those expansions (1 when k and l+1
                              share a block, else 2), [2] intervals reported before
                              deduplication, [3] interval-table sectors read (32 bytes each;
                              see fm_tuning.kmer_depth) */
    fm_profile *profile; /* optional host pointer, filled by a successful call */
    uint8_t *costs;    /* optional device uint8[pair_capacity]: for each reported interval, the
                          fewest differences (mismatch and single-symbol indel columns) among
                          the alignments of Listing 2 that reach it; written beside pairs */
    uint32_t best;     /* 1: report, per query, only the intervals of its minimum cost (the
                          best hits); counts and offsets then describe those.  0: all */
    uint32_t indel_end_skip; /* 0: indel columns anywhere Listing 2 allows them.  e > 0 (an option
                          in the manner of BWA, Li and Durbin 2009; not in the paper): an indel
                          column only where at least e symbols of the query lie on each side of
                          it, i.e. inserting W[i] needs e <= i <= m-1-e and a deletion between
                          W[i] and W[i+1] needs e-1 <= i <= m-1-e.  Costs and best hits follow
                          the restricted set.  The search then enumerates every alignment of
                          Listing 2 (fm_tuning.canonical does not apply).  At most 255. */
    /* With costs or best set, FM_ETRUNC leaves counts and offsets complete and the call must
     * be repeated with a larger pairs (and costs) buffer: fm_inexact_fetch does not apply.
     * fm_inexact_noalloc and the serving calls accept neither (FM_EINVAL). */
} fm_search_params;

#define FM_KERNEL_AUTO 0u       /* the persistent kernel */
#define FM_KERNEL_PLAIN 1u      /* one thread per query, depth-first with its own stack */
#define FM_KERNEL_PERSISTENT 2u /* persistent warps pulling queries from a device work queue,
                                   expanding pooled frontiers with warp-ballot compaction */

/* The lower bound D of the inexact search (the BWA bound, Li and Durbin 2009, cited with
 * Listing 2): D(i) = number of disjoint windows, taken greedily from W[0], that do not occur
 * in R, counted within W[0..i].  Computed by forward extension on the index of reverse(R).
 * reads/offs as in fm_exact; read lengths at most 255.
 * D_out: device uint8, strands*offs[n_reads] bytes; query q = r*strands + s has its m_r
 * values at D_out[strands*offs[r] + s*m_r ...].
 * Errors: FM_EINVAL (no reverse index, strands not 1/2, a code above 3, a read over 255). */
int fm_dcalc(fm_index *h, const uint8_t *reads, const uint32_t *offs, uint32_t n_reads,
             uint32_t strands, uint8_t *D_out, void *stream);

/* Listing 2 (InexRecur) with D pruning, for every query, as sets of SA intervals.
 * Readings of Listing 2 applied: fresh k', l' per symbol b; the deletion, match and mismatch
 * recursions run only when k' <= l'; insertions and deletions are single-symbol columns, at
 * most max_gaps of them; a branch with z < D(i) is cut; intervals reached without reading
 * any reference symbol are not reported; the search starts from [0, n].
 * reads/offs as in fm_exact (read lengths 1..255).
 * counts:  device uint32[nq]   distinct intervals of query q (nq = n_reads * strands);
 * offsets: device uint64[nq+1] exclusive prefix sum of counts;
 * pairs:   device uint32[2*pair_capacity]: query q's intervals are
 *          pairs[2*offsets[q] ...] as (k, l), sorted by k then l;
 * pairs_needed: host, receives offsets[nq].
 * When pairs_needed > pair_capacity the call returns FM_ETRUNC after filling counts and
 * offsets; pairs is then left untouched.
 * Errors: FM_EINVAL, FM_ETRUNC, FM_ENOMEM, FM_ECUDA. */
int fm_inexact(fm_index *h, const uint8_t *reads, const uint32_t *offs, uint32_t n_reads,
               const fm_search_params *sp, uint32_t *counts, uint64_t *offsets, uint32_t *pairs,
               uint64_t pair_capacity, uint64_t *pairs_needed, void *stream);

/* Copy the Listing 2 interval sets of the most recent fm_inexact call on h into pairs (device
 * uint32[2*pair_capacity], laid out as in fm_inexact), e.g. after that call returned
 * FM_ETRUNC.  Valid until the next fm_inexact or fm_inexact_noalloc call on h; a call that
 * failed with any other status leaves nothing to fetch.
 * Errors: FM_EINVAL (no earlier search), FM_ETRUNC (capacity below the count found). */
int fm_inexact_fetch(fm_index *h, uint32_t *pairs, uint64_t pair_capacity, void *stream);

/* fm_inexact without any device allocation.  The paper has no counterpart: this entry point
 * exists for callers that cannot let a library call cudaMalloc, such as a serving process whose
 * memory manager has reserved the device's memory up front (a library allocation would fail or
 * fragment its pool), or a latency-critical loop that must not pay for cudaMalloc/cudaFree and
 * the device synchronisation cudaFree implies.  fm_inexact grows its search scratch on demand;
 * this variant takes all of it from one fixed 64 MiB array in the library's device memory,
 * which every GPU that loads the library holds until the process exits.  It runs the
 * depth-first search kernel on a fixed 1536 threads (sp->kernel and sp->profile are ignored),
 * so it is slower than fm_inexact; its results are the same.
 * Arguments, results and errors are those of fm_inexact, with these limits:
 *   - at most 32,768 queries (n_reads * strands) per call, else FM_EINVAL;
 *   - at most 262,144 intervals before deduplication, else FM_ENOMEM (nothing is grown: split
 *     the batch and call again).
 * The index handle itself must already exist (fm_build/fm_load allocate).  This call builds
 * no table: it expands short strings from the interval tables, and takes two-symbol steps
 * over the pair table, only when an earlier fm_inexact, fm_exact or fm_server_start on h
 * built them (results are the same either way; without them it reads more checkpoint blocks
 * and runs slower).  Its results live in the static array, so fm_inexact_fetch does not serve
 * them: after this call, fetch returns FM_EINVAL until the next fm_inexact.  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress, once per device, with
 * that device current); make that first call before any stream capture.  Every call shares the
 * one array and leaves its contents behind; calls that overlap on the GPU, from any thread,
 * stream or handle, race on it and must not be issued. */
int fm_inexact_noalloc(fm_index *h, const uint8_t *reads, const uint32_t *offs, uint32_t n_reads,
                       const fm_search_params *sp, uint32_t *counts, uint64_t *offsets,
                       uint32_t *pairs, uint64_t pair_capacity, uint64_t *pairs_needed,
                       void *stream);

/* ------------------------------------------------------------------------------------------
 * Serving: a request loop over a resident index (the paper has no serving layer; it states the
 * search per read, Listing 1 and Listing 2, and this loop runs those searches for a stream of
 * requests).  Continuous batching with several batches in flight: the server runs `inflight`
 * worker threads, each with its own search scratch, stream and batch buffers on the same
 * resident index.  A worker that is free takes the pending requests in arrival order, of any
 * search mode (z, max_gaps are carried read by read), while their reads fit the batch's read
 * slots and the worker's share of the frontier budget, and searches them as one batch.  A
 * request that arrives while a batch is on the GPU starts as soon as a worker is free, while
 * that batch is still running, and the two batches overlap on the device.  Each request's
 * result is exactly what fm_inexact returns for that request alone.  While a server runs, no
 * other call may use its index handle.
 * ---------------------------------------------------------------------------------------- */
typedef struct fm_server fm_server;

typedef struct fm_server_params {
    uint32_t max_batch_reads; /* read slots per device batch (0: 262,144) */
    uint32_t strands;         /* 1 or 2, for every request */
    uint64_t frontier_budget; /* device bytes the search scratch of the batches in flight may
                                 use together (0: 64 GiB), shared equally by the workers: a
                                 worker sizes each batch by a model of the scratch its search
                                 allocates (raw intervals per query learned from its batches);
                                 a search that would still grow past the worker's share fails
                                 that growth and the batch is split in two (a single request
                                 that does not fit finishes with FM_ENOMEM) */
    uint32_t kernel;          /* FM_KERNEL_* */
    uint32_t inflight;        /* batches in flight, one worker thread each (0: 3; at most 4) */
} fm_server_params;

/* Result of one request, owned by the server until fm_server_release. */
typedef struct fm_server_result {
    int32_t status;          /* FM_OK or the error of the batch that held the request */
    uint32_t n_queries;      /* n_reads * strands */
    const uint32_t *counts;  /* host [n_queries] */
    const uint64_t *offsets; /* host [n_queries+1], from 0 */
    const uint32_t *pairs;   /* host [2*offsets[n_queries]] (k, l), sorted per query */
    uint64_t t_submit_ns;    /* steady-clock times: submission, batch start, completion */
    uint64_t t_start_ns;
    uint64_t t_done_ns;
    uint32_t batch_reads;    /* reads in the batch that held the request */
    uint32_t batch_id;       /* the batch that held it (1, 2, ... in order of completion) */
} fm_server_result;

/* Start the server thread on h (serving: no counterpart in the paper; every request runs the
 * search of Listing 2 exactly as fm_inexact does), after building the interval and pair tables
 * the tuning asks for (so no request waits for them).  Errors: FM_EINVAL, FM_ENOMEM,
 * FM_ECUDA. */
int fm_server_start(fm_index *h, const fm_server_params *p, fm_server **out);

/* Queue a request for the search of Listing 2: reads are host memory (codes 0..3,
 * concatenated, offs[n_reads+1]); they are copied before the call returns.  z <= 7,
 * max_gaps <= 7, read lengths 1..255 (else FM_EINVAL).  *ticket identifies the request. */
int fm_server_submit(fm_server *s, const uint8_t *reads, const uint32_t *offs, uint32_t n_reads,
                     uint32_t z, uint32_t max_gaps, uint64_t *ticket);

/* Wait up to wait_ms milliseconds (0: do not wait) for a request (serving: no counterpart in
 * the paper).  FM_OK fills *res with its Listing 2 interval sets; FM_ETIMEOUT when it is not
 * done yet; FM_EINVAL for an unknown ticket. */
int fm_server_poll(fm_server *s, uint64_t ticket, uint32_t wait_ms, fm_server_result *res);

/* Drop a finished request's result memory (serving: no counterpart in the paper). */
int fm_server_release(fm_server *s, uint64_t ticket);

/* Serving counters (no counterpart in the paper): batches run, reads searched, requests
 * finished, and the milliseconds the batches took, summed over the workers (batches in
 * flight together count once each). */
int fm_server_stats(fm_server *s, uint64_t out[4]);

/* Finish the queued requests, stop the thread and free the server (results not released are
 * freed too; serving: no counterpart in the paper).  NULL is ignored. */
int fm_server_stop(fm_server *s);

/* Measurement probe, exported for the benchmark only (no counterpart in the paper, and not a
 * search call): `threads` threads (a multiple of 256) each
 * read `per_thread` (a multiple of `inflight`) granules of `granule` bytes (32, 64 or 128) at
 * uniformly random granule-aligned offsets of the device buffer buf[0, bytes), `inflight`
 * (1, 2, 4 or 8) at a time in flight, and write one folded word each to sink (device
 * uint32[threads]).  The launch is enqueued on
 * `stream` and not synchronised.  It gives the empirical random-gather ceiling of this device
 * for the index gathers.  Errors: FM_EINVAL (alignment, sizes), FM_ECUDA. */
int fm_probe_gather(const void *buf, uint64_t bytes, uint32_t granule, uint32_t threads,
                    uint32_t per_thread, uint32_t inflight, uint64_t seed, uint32_t *sink,
                    void *stream);

/* Tuning knobs of the search kernels (the autotuner writes them).  Zero fields keep the
 * current value.  Errors: FM_EINVAL for out-of-range values. */
typedef struct fm_tuning {
    uint32_t warps_per_block;   /* persistent kernel: warps per CTA (1..8) */
    uint32_t blocks_per_sm;     /* persistent kernel: resident CTAs per SM (occupancy) */
    uint32_t chunk;             /* queries a warp takes from the work queue at once (1..32; default 8) */
    uint32_t plain_block;       /* plain kernel threads per CTA (a multiple of 32, <= 256) */
    uint32_t graphs;            /* 1: run the persistent search as a CUDA graph (captured on the
                                   first call with given buffers and sizes, replayed after);
                                   2: always launch eagerly */
    uint32_t occ_per_thread;    /* fm_occ8 queries per thread: 1, 2 or 4 */
    uint32_t l2_fetch_bytes;    /* 32, 64 or 128: the calling process's L2 fetch granularity
                                   (cudaLimitMaxL2FetchGranularity of its CUDA context, set at
                                   each compute call; it ends with the process) */
    uint32_t canonical;         /* 1 (default): the inexact search enumerates only canonical
                                   alignments: an indel next to a mismatch, or inside a run of
                                   one base, is taken in one fixed order or place, so the
                                   alignments that differ only there are searched once; the
                                   reported intervals are those of Listing 2, the nodes fewer.
                                   2: every call of Listing 2 (with pair_steps = 2 as well,
                                   stats count its nodes exactly) */
    uint32_t kmer_depth;        /* interval tables of short strings (Sec. 4.2 leaves the
                                   memory-bound search to better cache locality of the
                                   FM-index; this is one such method): for every string X of
                                   length j <= depth, the interval Listing 1 reaches after
                                   reading X, and whether X occurs.  Search nodes whose string
                                   is shorter than depth are expanded from the tables, with no
                                   checkpoint-block read; exact search starts depth steps in.
                                   Results, and node counts, are unchanged; stats[1] counts
                                   only checkpoint blocks.  Values: 1..15 the depth
                                   (2 x 4^depth x 8 bytes of device memory, built on the first
                                   search that needs them); FM_KMER_AUTO (default) the depth
                                   floor(log4(n + 1)) - 1, clamped to [0, 15] (14 at n = 2e9:
                                   4.3 GB, and as much again for the index of reverse(R),
                                   whose tables the D bound reads);
                                   FM_KMER_OFF none.  fm_get_tuning reports the depth in effect
                                   (FM_KMER_OFF for none) */
    uint32_t pair_steps;        /* 1 (default): searches advance exact continuations two symbols
                                   per step over a pair table (for each row, the two symbols
                                   before its suffix; one 8-byte record per pair code and 32
                                   rows, 4 B per row, 8 GB at n = 2e9, and as much again for
                                   the index of reverse(R), over which the D bound steps two
                                   symbols at a time; built from the index on the first call
                                   that needs it).  Intervals, insertion points
                                   and results are unchanged; an inexact search's stats[0] then
                                   omits the middle node of a two-symbol step that ends the
                                   branch.  2: one symbol per step (stats exactly as described) */
    uint32_t refill;            /* persistent kernel: a warp takes more queries from the work
                                   queue when its node pools hold fewer nodes than this
                                   (1..288; default 40) */
    uint32_t chain2_min;        /* persistent kernel: each lane holds up to two exact chains;
                                   the warp steps the second ones only while at least this many
                                   lanes hold one, else they wait for a first place (1..32;
                                   default 12; 1: always) */
    uint32_t stage;             /* persistent kernel: 1 stages each query a warp works on in
                                   shared memory (its 2-bit symbols, D breakpoints, length, mode
                                   and number; 16 slots per warp, taken and freed in groups of
                                   4); 2 (default) reads them through L1 from device memory,
                                   which measured faster on GB300: staging bounds the queries a
                                   warp holds at once, and its expansions run fewer nodes per
                                   step.  Results are the same either way */
} fm_tuning;

#define FM_KMER_AUTO 0xfeu
#define FM_KMER_OFF 0xffu

/* Set or read the knobs above.  They change speed and memory only, never results; the
 * interval tables and pair steps answer the cache-locality question Sec. 4.2 leaves open, the
 * rest have no counterpart in the paper.  fm_set_tuning checks every value before applying
 * any: a rejected call changes nothing. */
int fm_set_tuning(fm_index *h, const fm_tuning *t);
int fm_get_tuning(const fm_index *h, fm_tuning *t);

#ifdef __cplusplus
}
#endif
#endif
