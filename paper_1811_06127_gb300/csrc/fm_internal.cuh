// Internal declarations of the fmocc CUDA library (sm_103a).
//
// Resident layout (per index, forward and reverse): an array of checkpoint blocks.  Block j
// covers BWT rows [j*I, (j+1)*I):
//   bytes  0..15  uint32 cnt[4]: rank(c, j*I) for c = A,C,G,T ($ excluded)
//   bytes 16..    the I BWT symbols of the block, 2 bits each, symbol t of the block at bits
//                 2(t%32)..2(t%32)+1 of 64-bit word t/32 (the little-endian 2-bit code of
//                 Fig. 2); $ is stored as A and corrected for through dollar_row
//   I = 32: 32-byte blocks (24 used), I = 64: 32-byte blocks (one DRAM sector);
//   I = 128: 64 bytes; I = 256: 96 bytes (80 used).
// One extra final block holds the totals, so rank(c, n+1) needs no special case.
// This interleaving of counters and symbols in one block follows the bucket layout the paper
// describes in Sec. 2 (128 symbols with 4 x 64-bit counters); here the counters are uint32
// and the block is sized to the 32-byte sector.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/fmocc.h"

namespace fm {

constexpr int kMaxReadLen = 255;   // read length limit of the search kernels (8-bit position)
constexpr int kMaxZ = 7;
constexpr int kMaxGaps = 7;

__host__ __device__ constexpr uint32_t block_bytes(uint32_t I) {
    return I <= 64 ? 32u : (I == 128 ? 64u : 96u);
}

// Device view of one resident index.
struct IndexView {
    const uint8_t *blocks;   // n_blocks * block_bytes(I)
    uint32_t n;              // reference length
    uint32_t dollar;         // row holding $
    uint32_t C[5];
    // Interval tables of short strings (0 levels: none).  For every string X of length j <= kdepth,
    // with code(X) = sum_t X[t] 4^t (X[0], the symbol a backward step prepends last, least
    // significant, so the four one-symbol extensions bX of X have the consecutive codes
    // 4 code(X) + b): kt[4^j + code(X)] = the interval Listing 1 reaches from [0, n] after
    // reading X (also when empty: k = l + 1 is its insertion point), and bit 4^j + code(X) of
    // kbits = X occurs (k <= l).
    const uint2 *kt;
    const uint32_t *kbits;
    uint32_t kdepth;
    // Pair table (0 when absent): for every row i, the two symbols before suffix SA[i],
    // BWT[LF(i)] and BWT[i], as one 4-bit code 4 b1 + b2, so that one rank over pairs moves an
    // interval back two symbols.  One 8-byte record per (pair code c, 32-row block j), at
    // uint2 entry c * pnblk + j of prec: x = rows before block j holding pair c, y = which
    // rows of the block hold pair c (row 32 j + r at bit r).  A rank of one pair is one
    // record: one 8-byte load.  The $ row and the row whose LF is the $ row
    // have no pair and are in no record's rows.  pc2[c]: rows whose suffix sorts before every
    // string starting with pair c.
    const uint2 *prec;
    const uint32_t *pc2;
    uint32_t pnblk;
    uint32_t pairs;
};

// Per-search device pointers (scratch owned by the handle).
struct Scratch {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// What a captured search graph depends on; a call with another key captures a new graph.
struct GraphKey {
    const void *reads, *offs, *counts, *offsets, *pairs, *stats;
    const void *qmeta, *raw, *spill, *group, *misc, *kt, *modes;
    uint64_t pair_capacity, raw_cap;
    uint32_t n_reads, strands, z, max_gaps, interval, grid, block, chunk, spill_cap, profile, canon,
        kdepth, end_skip, refill, chain2, pool;
    bool operator==(const GraphKey &o) const {
        return reads == o.reads && offs == o.offs && counts == o.counts && offsets == o.offsets &&
               pairs == o.pairs && stats == o.stats && qmeta == o.qmeta && raw == o.raw &&
               modes == o.modes &&
               spill == o.spill && group == o.group && misc == o.misc &&
               pair_capacity == o.pair_capacity && raw_cap == o.raw_cap && n_reads == o.n_reads &&
               strands == o.strands && z == o.z && max_gaps == o.max_gaps &&
               interval == o.interval && grid == o.grid && block == o.block && chunk == o.chunk &&
               spill_cap == o.spill_cap && profile == o.profile && canon == o.canon && kt == o.kt &&
               kdepth == o.kdepth && end_skip == o.end_skip && refill == o.refill &&
               chain2 == o.chain2 && pool == o.pool;
    }
};

struct Tuning {
    uint32_t warps_per_block = 8;
    uint32_t blocks_per_sm = 0;     // 0: from the occupancy calculator
    uint32_t chunk = 8;      // queries a warp takes from the work queue at once
    uint32_t plain_block = 128;
    uint32_t occ_q = 2;
    uint32_t canon = 1;      // inexact search enumerates canonical alignments only
    uint32_t kmer = FM_KMER_AUTO;   // interval-table depth setting (FM_KMER_AUTO, FM_KMER_OFF, 1..15)
    uint32_t pairs = 1;             // exact continuations two symbols per step from the pair table
    uint32_t l2_fetch = 0;   // 0: leave the context's limit alone
    uint32_t refill = 40;    // a warp takes more queries when its pools hold fewer nodes
    uint32_t chain2_min = 12; // lanes whose second exact chain is live for the warp to step it
    uint32_t stage = 0;      // persistent kernel stages its queries in shared memory
};

}  // namespace fm

struct fm_index {
    int device = 0;
    int sms = 0;
    uint64_t n = 0;
    uint32_t interval = 64;
    uint32_t bbytes = 32;
    uint64_t n_blocks = 0;
    uint64_t C[5] = {0, 0, 0, 0, 0};
    uint64_t dollar = 0, rev_dollar = 0;
    bool has_rev = false;
    bool both_strands = false;       // the text is R . revcomp(R)
    uint8_t *d_fwd = nullptr;        // forward checkpoint blocks
    uint8_t *d_rev = nullptr;        // reverse(R) checkpoint blocks
    uint32_t *d_sa_sample = nullptr; // SA[j * sa_rate]
    uint64_t sa_rate = 32;
    uint64_t n_sa_sample = 0;
    uint32_t *d_err = nullptr;       // device error word (1 word per call kind)
    uint2 *d_kt = nullptr;           // interval tables of short strings (forward index)
    uint32_t *d_kbits = nullptr;     // their occurrence bits
    uint32_t kt_depth = 0;           // levels built (0: none)
    uint2 *d_kt_rev = nullptr;       // the same tables of the index of reverse(R) (D bound)
    uint32_t *d_kbits_rev = nullptr;
    uint2 *d_prec = nullptr;         // pair table (see IndexView)
    uint2 *d_prec_rev = nullptr;     // the pair table of the index of reverse(R) (D pass)
    uint32_t *d_pc2_rev = nullptr;
    uint32_t *d_pc2 = nullptr;       // its pc2[16]
    bool pairs_built = false;
    // grow-on-demand scratch of the search calls
    fm::Scratch s_qmeta, s_raw, s_spill, s_group, s_scan, s_plain, s_misc;
    uint64_t scratch_budget = 0;     // 0: unbounded; else growth past it fails with FM_ENOMEM
    bool borrowed = false;           // a search context: the index tables belong to another
                                     // handle (see new_search_context)
    fm::Tuning tune;
    std::string err;
    // canonical results of the last search (in s_group), for fm_inexact_fetch
    uint32_t last_nq = 0;
    uint64_t last_total = 0;
    bool last_valid = false;
    size_t last_off_ucnt = 0, last_off_start = 0, last_off_uoff = 0, last_off_grp = 0;
    // CUDA graph of the persistent search call (captured once per key, replayed after)
    bool use_graphs = true;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    fm::GraphKey gkey{};
    uint32_t glaunches = 0;
    cudaEvent_t gev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    uint64_t graph_replays = 0, graph_captures = 0;
};

namespace fm {

// error plumbing -------------------------------------------------------------------------
int set_error(fm_index *h, int code, const std::string &msg);
int set_global_error(int code, const std::string &msg);
int cuda_status(fm_index *h, cudaError_t e, const char *what);
int ensure_scratch(fm_index *h, Scratch &s, size_t bytes);
uint64_t scratch_total(const fm_index *h);
// A search context: a second handle onto h's resident index (every table shared, none owned)
// with scratch, error words, graph state and fetchable results of its own, so that searches
// on h and on its contexts can run at the same time on different streams and host threads.
// Valid while h lives and its tables are not rebuilt; freed by free_search_context only.
fm_index *new_search_context(fm_index *h);
void free_search_context(fm_index *c);
int device_sms(int device);

#define FM_CUDA_TRY(h, call)                                   \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) return fm::cuda_status(h, _e, #call); \
    } while (0)

// build entry (fm_build.cu) ----------------------------------------------------------------
int build_index(fm_index *h, const uint8_t *d_codes, uint64_t n, bool reverse, uint8_t **out_blocks,
                uint64_t *out_dollar, uint64_t C[5], uint32_t **out_sa_sample, cudaStream_t st);

// search entries (fm_search.cu, fm_inexact.cu) ------------------------------------------
IndexView view_fwd(const fm_index *h);
IndexView view_rev(const fm_index *h);

int launch_occ8(fm_index *h, const uint32_t *k, const uint32_t *l, uint32_t *out8, uint64_t N,
                cudaStream_t st);
int launch_locate(fm_index *h, const uint32_t *rows, uint64_t N, uint32_t *pos,
                  unsigned long long *steps, cudaStream_t st);
int launch_exact(fm_index *h, const uint8_t *reads, const uint32_t *offs, uint32_t n_reads,
                 uint32_t *k_out, uint32_t *l_out, cudaStream_t st);
// interval tables: the depth the tuning asks for on this index, and (re)building them to it
uint32_t kmer_depth_for(const fm_index *h);
int ensure_kmer(fm_index *h, cudaStream_t st);
// pair table: built on first use when the tuning asks for pair steps
int ensure_pairs(fm_index *h, cudaStream_t st);
constexpr uint32_t kPairRows = 32;
constexpr uint32_t kPairScanBlocks = 512;   // blocks one thread of the pair count pass sums
constexpr uint32_t kMaxKmerDepth = 15;   // 2 x 4^15 entries: 32-bit table indices
// D lower bound per query; qmeta (one uint4 per query, or with stride kStageU4 the staging
// record of the persistent search: that uint4, then the query as 2-bit symbols) and/or D_out
// (uint8 per position)
constexpr uint32_t kStageU4 = 5;
// modes: optional device uint8 per read, its search mode (z | max_gaps << 4); else defmode
int launch_dcalc(fm_index *h, const uint8_t *reads, const uint32_t *offs, uint32_t n_reads,
                 uint32_t strands, uint4 *qmeta, uint8_t *D_out, cudaStream_t st,
                 uint32_t stride = 1, const uint8_t *modes = nullptr, uint32_t defmode = 0);
int fetch_inexact(fm_index *h, uint32_t *pairs, uint64_t pair_capacity, cudaStream_t st);
// grow h's search scratch now to the sizes a persistent search of nq queries starts from (so
// that such searches allocate, and free, nothing)
int reserve_search_scratch(fm_index *h, uint64_t nq);
// modes: optional device uint8 per read (z | max_gaps << 4), overriding sp->z and
// sp->max_gaps read by read (serving batches that mix search modes)
int run_inexact(fm_index *h, const uint8_t *reads, const uint32_t *offs, uint32_t n_reads,
                const fm_search_params *sp, uint32_t *counts, uint64_t *offsets, uint32_t *pairs,
                uint64_t pair_capacity, uint64_t *pairs_needed, cudaStream_t st,
                const uint8_t *modes = nullptr);

// error word slots
enum ErrSlot { kErrOcc = 0, kErrExact = 1, kErrDcalc = 2, kErrSearch = 3, kErrBuild = 4,
               kErrSlots = 8 };
// error bits
enum ErrBits : uint32_t {
    kErrDomain = 1u,      // a query or symbol outside the domain
    kErrSpill = 2u,       // frontier spill capacity exceeded
    kErrStack = 4u,       // plain-kernel stack capacity exceeded
    kErrReadLen = 8u,     // read longer than kMaxReadLen
};

// -----------------------------------------------------------------------------------------
// device helpers
// -----------------------------------------------------------------------------------------

// 256-bit read-only load of one 32-byte sector (sm_100+ PTX).  Not volatile: the tables are
// read-only while a kernel runs, so the compiler may hoist and batch these loads.
__device__ __forceinline__ void ldg256(const void *p, uint4 &a, uint4 &b) {
    asm("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z),
                   "=r"(b.w)
                 : "l"(p));
}

// L1 policy of the random gathers.  Checkpoint blocks, pair records and the interval-table
// sectors of levels >= kL1TableLevel are read once per search node at uniformly random places
// of a table far larger than L1; they are loaded without allocating L1 lines, so that they do
// not evict the lines that are reused (the shallow table levels, the occurrence bits, the
// query data), which stay in L1 across nodes, queries and warps of the SM.
constexpr bool kGatherNoL1 = true;
constexpr uint32_t kL1TableLevel = 8;
__device__ __forceinline__ void ldg256_na(const void *p, uint4 &a, uint4 &b) {
    if constexpr (kGatherNoL1) {
        asm("ld.global.nc.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
            : "l"(p));
    } else {
        ldg256(p, a, b);
    }
}

__device__ __forceinline__ uint32_t ldg32_na(const uint32_t *p) {
    uint32_t v;
    if constexpr (kGatherNoL1) asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    else v = __ldg(p);
    return v;
}

__device__ __forceinline__ uint2 ldg64_na(const uint2 *p) {
    uint2 v;
    if constexpr (kGatherNoL1) asm("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    else v = __ldg(p);
    return v;
}

__device__ __forceinline__ uint64_t u64of(uint32_t lo, uint32_t hi) {
    return (uint64_t)lo | ((uint64_t)hi << 32);
}

// Symbols A,C,G,T counted among the first t symbols (t in [0,32]) of a 64-bit word of 2-bit
// codes: lo bit set for C(01) and T(11), hi bit set for G(10) and T(11).
__device__ __forceinline__ void count_word(uint64_t w, uint32_t t, uint32_t &c, uint32_t &g,
                                           uint32_t &tt) {
    const uint64_t m55 = 0x5555555555555555ull;
    uint64_t mask = t >= 32 ? ~0ull : ((1ull << (2 * t)) - 1ull);
    uint64_t lo = w & m55 & mask;
    uint64_t hi = (w >> 1) & m55 & mask;
    uint32_t both = __popcll(lo & hi);
    tt += both;
    c += __popcll(lo) - both;
    g += __popcll(hi) - both;
}

// Loaded checkpoint block: counters plus up to 8 words (I <= 256).
template <int I>
struct Blk {
    uint4 cnt;
    uint64_t w[I / 32];
};

// Load the block of rank position p (only the sectors the offsets up to `upto` need are
// read for I >= 128).
template <int I>
__device__ __forceinline__ void load_block(const uint8_t *blocks, uint32_t j, uint32_t upto,
                                           Blk<I> &B) {
    const uint8_t *p = blocks + (size_t)j * block_bytes(I);
    uint4 a, b;
    ldg256_na(p, a, b);
    B.cnt = a;
    B.w[0] = u64of(b.x, b.y);
    if constexpr (I >= 64) B.w[1] = u64of(b.z, b.w);
    if constexpr (I >= 128) {
        // every word is assigned once; a sector no offset needs is not read
        uint4 c = make_uint4(0, 0, 0, 0), d = make_uint4(0, 0, 0, 0);
        if (upto > 64) ldg256_na(p + 32, c, d);
        B.w[2] = u64of(c.x, c.y);
        B.w[3] = u64of(c.z, c.w);
        if constexpr (I == 256) {
            uint4 e = make_uint4(0, 0, 0, 0), f;
            B.w[4] = u64of(d.x, d.y);
            B.w[5] = u64of(d.z, d.w);
            if (upto > 192) ldg256_na(p + 64, e, f);
            B.w[6] = u64of(e.x, e.y);
            B.w[7] = u64of(e.z, e.w);
        }
    }
}

// Interval-table access (see IndexView): level j starts at entry (and bit) 4^j.
__device__ __forceinline__ uint32_t kt_base(uint32_t j) { return 1u << (2u * j); }
__device__ __forceinline__ uint2 kt_get(const IndexView &ix, uint32_t j, uint32_t code) {
    return j >= kL1TableLevel ? ldg64_na(ix.kt + kt_base(j) + code) : __ldg(ix.kt + kt_base(j) + code);
}
// occurrence bits of the four extensions 4c .. 4c+3 at level j >= 1 (bit b: extension b)
__device__ __forceinline__ uint32_t kt_occ4(const IndexView &ix, uint32_t j, uint32_t c) {
    const uint32_t bit = kt_base(j) + 4u * c;
    return (__ldg(ix.kbits + (bit >> 5)) >> (bit & 31u)) & 15u;
}
__device__ __forceinline__ uint32_t kt_occ1(const IndexView &ix, uint32_t j, uint32_t code) {
    const uint32_t bit = kt_base(j) + code;
    return (__ldg(ix.kbits + (bit >> 5)) >> (bit & 31u)) & 1u;
}
// intervals of the four extensions 4c .. 4c+3 at level j >= 1: one 32-byte sector
__device__ __forceinline__ void kt_get4(const IndexView &ix, uint32_t j, uint32_t c, uint32_t k[4],
                                        uint32_t l[4]) {
    uint4 a, b;
    if (j >= kL1TableLevel) ldg256_na(ix.kt + kt_base(j) + 4u * c, a, b);
    else ldg256(ix.kt + kt_base(j) + 4u * c, a, b);
    k[0] = a.x; l[0] = a.y; k[1] = a.z; l[1] = a.w;
    k[2] = b.x; l[2] = b.y; k[3] = b.z; l[3] = b.w;
}

// Mask of the low `width` bits (width in [0, 32]).
__device__ __forceinline__ uint32_t low_mask(uint32_t width) {
    uint32_t m;
    asm("bmsk.clamp.b32 %0, %1, %2;" : "=r"(m) : "r"(0u), "r"(width));
    return m;
}

// One record of the pair table (a read-only load that allocates no L1 line).  Measured on the
// headline search: 8-byte records of 32 rows 518 ms, 16-byte records of 64 rows 534 ms,
// 32-byte records of 128 rows 595 ms (the same table size).
__device__ __forceinline__ uint2 load_pair_rec(const IndexView &ix, uint32_t c, uint32_t j) {
    const uint2 *p = ix.prec + (size_t)c * ix.pnblk + j;
    uint2 v;
    asm("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}
// Pairs c in rows [0, p), r the record of c for the block of p.
__device__ __forceinline__ uint32_t pair_rank(const uint2 &r, uint32_t p) {
    return r.x + __popc(r.y & low_mask(p % kPairRows));
}

// C, G and T among the first t symbols (t in [0, 32]) of one 64-bit word, in 32-bit steps:
// the lo/hi bit planes of the two 16-symbol halves are masked to the prefix and interleaved
// into one 32-bit word each, so three popcounts count 32 symbols.
__device__ __forceinline__ void count_word32(uint64_t w, uint32_t t, uint32_t &c, uint32_t &g,
                                             uint32_t &tt) {
    const uint32_t m55 = 0x55555555u;
    const uint32_t w0 = (uint32_t)w, w1 = (uint32_t)(w >> 32);
    const uint32_t t0 = t < 16u ? t : 16u;
    const uint32_t m0 = low_mask(2u * t0) & m55;
    const uint32_t m1 = low_mask(2u * (t - t0)) & m55;
    const uint32_t L = (w0 & m0) | ((w1 & m1) << 1);
    const uint32_t H = ((w0 >> 1) & m0) | (((w1 >> 1) & m1) << 1);
    const uint32_t both = __popc(L & H);
    tt += both;
    c += __popc(L) - both;
    g += __popc(H) - both;
}

// rank(c, p) for c = A,C,G,T given the loaded block of p (block index j = p / I).
template <int I>
__device__ __forceinline__ void rank4_in(const Blk<I> &B, uint32_t j, uint32_t p, uint32_t dollar,
                                         uint32_t r[4]) {
    const uint32_t o = p - j * (uint32_t)I;
    uint32_t c = 0, g = 0, t = 0;
#pragma unroll
    for (int wi = 0; wi < I / 32; ++wi) {
        const int32_t left = (int32_t)o - 32 * wi;
        const uint32_t n = left <= 0 ? 0u : (left >= 32 ? 32u : (uint32_t)left);
        count_word32(B.w[wi], n, c, g, t);
    }
    uint32_t a = o - c - g - t;
    const uint32_t base = j * (uint32_t)I;
    a -= (dollar >= base && dollar < p) ? 1u : 0u;
    r[0] = B.cnt.x + a;
    r[1] = B.cnt.y + c;
    r[2] = B.cnt.z + g;
    r[3] = B.cnt.w + t;
}

// Occurrences of symbol b among the first t symbols (t in [0, 32]) of one 64-bit word, in
// 32-bit steps: XOR with b's pattern turns b's pairs into 00; a pair is 00 when neither bit is
// set; the two 16-symbol halves are interleaved into one word for a single popcount.
__device__ __forceinline__ uint32_t count_sym(uint64_t w, uint32_t t, uint32_t b) {
    const uint32_t m55 = 0x55555555u;
    const uint32_t pat = m55 * b;
    const uint32_t x0 = (uint32_t)w ^ pat, x1 = (uint32_t)(w >> 32) ^ pat;
    const uint32_t t0 = t < 16u ? t : 16u;
    const uint32_t y0 = ~(x0 | (x0 >> 1)) & (low_mask(2u * t0) & m55);
    const uint32_t y1 = ~(x1 | (x1 >> 1)) & (low_mask(2u * (t - t0)) & m55);
    return __popc(y0 | (y1 << 1));
}

// rank(b, p) for one symbol b given the loaded block of p.
template <int I>
__device__ __forceinline__ uint32_t rank1_in(const Blk<I> &B, uint32_t j, uint32_t p,
                                             uint32_t dollar, uint32_t b) {
    const uint32_t o = p - j * (uint32_t)I;
    uint32_t r = 0;
#pragma unroll
    for (int wi = 0; wi < I / 32; ++wi) {
        const int32_t left = (int32_t)o - 32 * wi;
        const uint32_t n = left <= 0 ? 0u : (left >= 32 ? 32u : (uint32_t)left);
        r += count_sym(B.w[wi], n, b);
    }
    const uint32_t base = j * (uint32_t)I;
    if (b == 0u) r -= (dollar >= base && dollar < p) ? 1u : 0u;   // $ is stored as A
    const uint32_t cnt = b == 0 ? B.cnt.x : (b == 1 ? B.cnt.y : (b == 2 ? B.cnt.z : B.cnt.w));
    return cnt + r;
}

// BWT symbol at row p of the loaded block j (the $ row reads as A).
template <int I>
__device__ __forceinline__ uint32_t sym_in(const Blk<I> &B, uint32_t j, uint32_t p) {
    const uint32_t o = p - j * (uint32_t)I;
    const uint32_t sel = o >> 5;
    uint64_t w = 0;   // masked OR, not an indexed read: keeps the block in registers
#pragma unroll
    for (int t = 0; t < I / 32; ++t) w |= B.w[t] & (0ull - (uint64_t)(sel == (uint32_t)t));
    return (uint32_t)(w >> (2 * (o & 31))) & 3u;
}

}  // namespace fm
