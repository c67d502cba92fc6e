// Inexact search (Listing 2, InexRecur) with the D lower bound, on the device.
//
// A search node is one call of InexRecur: (query q, position i, differences left z, indel
// columns used g, interval [k, l]), packed in 16 bytes.  Expanding a node costs one eight-Occ
// step (rank(c, k) and rank(c, l+1) for c in ACGT, from one or two checkpoint blocks) and
// yields up to nine children, per Listing 2 with these readings:
//   insertion  (i-1, z-1, g+1, k, l)            when z >= 1 and g < max_gaps
//   deletion   (i,   z-1, g+1, k'_b, l'_b)      for each b with k'_b <= l'_b, z >= 1, g < max_gaps
//   match      (i-1, z,   g,   k'_b, l'_b)      for b = W[i], k'_b <= l'_b
//   mismatch   (i-1, z-1, g,   k'_b, l'_b)      for b != W[i], k'_b <= l'_b, z >= 1
// and, with an end restriction e > 0 (an option after BWA, not in the paper), an indel column
// only where at least e read symbols lie on each side of it: an insertion of W[i] when
// e <= i <= m-1-e, a deletion at i (between W[i] and W[i+1]) when e-1 <= i <= m-1-e.
// with k'_b = C[b] + rank(b, k) + 1 and l'_b = C[b] + rank(b, l+1) computed from the node's
// own interval.  A child at position i' >= 0 survives only when its z' >= D(i'); a child at
// i' = -1 is a leaf: its interval is a result unless k = 0 (no reference symbol read).
//
// Two schedulers of the same node expansion:
//   * plain: one thread per query, depth-first with an explicit stack in device memory
//     (interleaved across threads so that neighbouring lanes touch neighbouring words);
//   * persistent: a grid of resident warps.  Each warp keeps a pool of nodes of any queries
//     in shared memory, pops up to 32 of them per step (one per lane), expands them, and
//     pushes the surviving children back with a warp-ballot/shuffle prefix sum.  When its pool
//     runs low the warp takes the next chunk of queries from a device work queue (an atomic
//     counter) and stages each of them in a shared-memory slot (the query's 2-bit symbols,
//     oriented for its strand, its D breakpoints and length), so that no expansion reads
//     query data from device memory; when the pool would overflow it spills to a per-warp
//     region of device memory.  A warp leaves when the queue is drained and its pool and spill
//     are empty.
// Leaves are appended to a raw result buffer (warp-aggregated atomics).  The raw results are
// then grouped by query, sorted and deduplicated (canonical sets, Listing 2's set union), and
// compacted into the caller's counts/offsets/pairs.
#include <string.h>

#include "fm_internal.cuh"

namespace fm {
namespace {

constexpr uint32_t FULL = 0xffffffffu;

struct SearchCfg {
    IndexView ix;
    const uint8_t *reads;
    const uint4 *qmeta;          // plain kernel: one uint4 per query; persistent: kStageU4
    uint32_t nq;
    uint32_t z, max_gaps;
    uint32_t chunk;
    uint32_t *next_q;
    uint4 *raw;
    unsigned long long *raw_count;
    uint64_t raw_cap;
    unsigned long long *stats;   // nodes, blocks, raw
    uint32_t *err;
    uint32_t canon;              // enumerate canonical alignments only (see expand)
    uint32_t end_skip;           // indel columns need this many read symbols on each side
    uint32_t refill;             // persistent: take queries when the pools hold fewer nodes
    uint32_t chain2_min;         // persistent: step second exact chains when this many are live
    unsigned long long *fill;    // persistent: step-fill counters (kFillCounters), or null
};

// The canonical rewrites move indel columns across read positions, so under an end
// restriction the search enumerates every alignment of Listing 2 instead.
inline uint32_t search_canon(const Tuning &tu, const fm_search_params *sp) {
    return sp->indel_end_skip ? 0u : tu.canon;
}

__device__ __forceinline__ uint32_t d_at(const uint4 &mt, int i) {
    if (i < 0) return 0u;
    const uint32_t ib = (uint32_t)i * 0x01010101u;
    return __popc(__vcmpleu4(mt.x, ib) & 0x01010101u) + __popc(__vcmpleu4(mt.y, ib) & 0x01010101u);
}

__device__ __forceinline__ uint32_t w_at(const uint8_t *reads, const uint4 &mt, uint32_t i) {
    const uint32_t m = mt.w & 255u;
    if ((mt.w >> 8) & 1u) return 3u - reads[mt.z + m - 1u - i];   // bit 8: the strand
    return reads[mt.z + i];
}

// A query as the node expansion sees it: W[i] (oriented for the query's strand), D(i) and the
// length m.  GQuery reads the concatenated reads in device memory and the query's metadata
// word (plain kernel); SQuery reads the query's shared-memory slot (persistent kernel).
struct GQuery {
    const uint8_t *reads;
    uint4 mt;
    __device__ __forceinline__ uint32_t w(uint32_t i) const { return w_at(reads, mt, i); }
    __device__ __forceinline__ uint32_t d(int i) const { return d_at(mt, i); }
    __device__ __forceinline__ uint32_t len() const { return mt.w & 255u; }
    __device__ __forceinline__ uint32_t z0() const { return (mt.w >> 16) & 15u; }
    __device__ __forceinline__ uint32_t gaps() const { return (mt.w >> 20) & 15u; }
};

// An exact chain's query without staging: base is the index in reads of W[0] (the read's first
// symbol, or its last for the reverse complement), md the query's metadata word; then
// W[i] = reads[base + i], or 3 - reads[base - i] = reads[base - i] ^ 3 on the reverse strand.
struct CQuery {
    const uint8_t *reads;
    uint32_t base, md;
    __device__ __forceinline__ uint32_t w(uint32_t i) const {
        const uint32_t rc = (md >> 8) & 1u;
        return (uint32_t)reads[rc ? base - i : base + i] ^ (rc * 3u);
    }
    __device__ __forceinline__ uint32_t z0() const { return (md >> 16) & 15u; }
};
__device__ __forceinline__ uint2 chain_base(const uint4 &mt) {
    return make_uint2(((mt.w >> 8) & 1u) ? mt.z + (mt.w & 255u) - 1u : mt.z, mt.w);
}

// Shared-memory query slots of the persistent kernel (with staging): kSlots per warp, in
// kGroups groups of kGroupSlots, kSlotWords words each: words 0-15 the query's symbols, W[i]
// at bits 2(i%16) of word i/16; words 16-17 its D breakpoints; word 18 its length m (bits
// 0-7) and its search mode (bits 16-19 the differences allowed, 20-23 the indel columns
// allowed); word 19 the query number.  A node carries its query's slot in bits 25-29 of its
// state word.  The 80-byte stride keeps each slot 16-byte aligned and spreads the slots of 8
// lanes over distinct banks.
constexpr int kGroupSlots = 4;
constexpr int kGroups = 4;
constexpr int kSlots = kGroups * kGroupSlots;
constexpr int kSlotWords = 20;
constexpr uint32_t kSlotShift = 25u;
constexpr uint32_t kSlotBits = 31u << kSlotShift;
constexpr int kFillCounters = 8;
static_assert(kSlots <= 32, "a node holds a 5-bit slot");
__device__ __forceinline__ uint32_t slot_of(const uint4 &nd) { return (nd.y >> kSlotShift) & 31u; }

struct SQuery {
    const uint32_t *s;
    __device__ __forceinline__ uint32_t w(uint32_t i) const { return (s[i >> 4] >> (2u * (i & 15u))) & 3u; }
    __device__ __forceinline__ uint32_t d(int i) const { return d_at(make_uint4(s[16], s[17], 0u, 0u), i); }
    __device__ __forceinline__ uint32_t len() const { return s[18] & 255u; }
    __device__ __forceinline__ uint32_t z0() const { return (s[18] >> 16) & 15u; }
    __device__ __forceinline__ uint32_t gaps() const { return (s[18] >> 20) & 15u; }
    __device__ __forceinline__ uint32_t q() const { return s[19]; }
};

// The node pools of one warp: stk entries.  Without staging a node is one uint4 (query number,
// state word, k, l); with staging the query number lives in the node's slot and the pools keep
// three 32-bit arrays (state word, k, l), 12 bytes per node, so that the pools and the slots
// of a warp together take the 16-byte pools' shared memory.
template <bool STAGE>
struct Pool;
template <>
struct Pool<false> {
    uint4 *e;
    __device__ __forceinline__ uint4 get(int t) const { return e[t]; }
    __device__ __forceinline__ void put(int t, const uint4 &v) const { e[t] = v; }
    static constexpr int kWords = 4;   // per entry
};
template <>
struct Pool<true> {
    uint32_t *y, *k, *l;
    __device__ __forceinline__ uint4 get(int t) const { return make_uint4(0u, y[t], k[t], l[t]); }
    __device__ __forceinline__ void put(int t, const uint4 &v) const {
        y[t] = v.y;
        k[t] = v.z;
        l[t] = v.w;
    }
    static constexpr int kWords = 3;
};

// 32-bit words of shared memory per warp of the persistent kernel
__host__ __device__ constexpr int warp_smem_words(int stk, bool stage, bool fill) {
    return stk * (stage ? 3 : 4) + (stage ? kSlots * kSlotWords : 0) + (fill ? kFillCounters : 0);
}

// Node word y: bits 0-7 i, 8-11 z left, 12-15 indel columns used, 16-17 the operation that
// created the node (kOpMatch also for a root), 18-19 its reference symbol (mismatch, deletion),
// 20-23 the length d of the node's reference string X and bit 24 (kShallow) set while
// d < the interval-table depth.  A shallow node holds code(X) in z (w unused) instead of X's
// interval: its children come from the tables' occurrence bits, and at the table depth from
// one 32-byte sector of intervals, with no checkpoint block read.
constexpr uint32_t kOpMatch = 0u, kOpMis = 1u, kOpIns = 2u, kOpDel = 3u;
constexpr uint32_t kShallow = 1u << 24;
constexpr uint32_t kDepthBits = 15u << 20;
// step cost word of expand / exact_step: checkpoint blocks read in bits 0-15, interval-table
// sectors read in bits 16-31; accumulated per thread as blocks + (sectors << 32)
constexpr uint32_t kTabRead = 1u << 16;
__device__ __forceinline__ unsigned long long step_cost(uint32_t nb) {
    return (unsigned long long)(nb & 0xffffu) + ((unsigned long long)(nb >> 16) << 32);
}

// One expansion: the eight-Occ step of Listing 2 (rank(c, k) and rank(c, l+1) for c in ACGT
// from one or two checkpoint blocks), then the children.  Every lane runs the same code, so
// the block gathers of the whole warp are issued together.  Outputs the four child intervals
// and two 9-bit masks: bit 0 insertion, bits 1..4 deletion with b = 0..3, bits 5..8
// match/mismatch with b = 0..3; push: child kept as a node; leaf: child is a result.
//
// With c.canon set, only canonical alignments are enumerated.  Two alignments that differ by
// where an indel sits next to a mismatch, or by which copy of a repeated base an indel takes,
// spell the same reference string, and their search states coincide (or one has fewer
// differences left and is dominated).  Each rewrite below keeps the spelled string, never
// raises the cost or the indel count, and moves an indel one read position towards W[0] (or
// lowers the cost), so rewriting ends, and every alignment within the bounds has a canonical
// one spelling the same string.  Since a path to a result is never cut by the D bound (D(i)
// bounds the differences any alignment of W[0..i] needs), the reported intervals are those of
// Listing 2; only repeated subtrees go.  Forbidden, in processing order (i decreasing):
//   insertion of W[i+1], then match of W[i] = W[i+1]   (same as match, then insertion)
//   insertion, then mismatch or deletion               (mismatch/match first; or one mismatch)
//   deletion b at i >= 1, then match of W[i] = b        (match, then deletion at i-1)
//   deletion at i >= 1, then mismatch                  (mismatch/match, then deletion at i-1)
//   deletion, then insertion                           (one mismatch or match)
//   mismatch b at W[i+1], then insertion of W[i] = b   (insertion, then match: one less)
//   mismatch at W[i+1], then deletion of b = W[i+1]    (deletion, then match: one less)
// A node none of whose Occ children is allowed takes no Occ step and is not counted; a child
// that could take no step at all is not created.  The rewrites move indel columns, so they
// are not applied together with an end restriction (the host clears canon).
template <int I, class Q>
__device__ __forceinline__ void expand(const SearchCfg &c, const uint4 &nd, const Q &qv,
                                       uint32_t k2[4], uint32_t l2[4], uint32_t &push,
                                       uint32_t &leaf, uint32_t &nblocks, uint32_t &counted,
                                       uint32_t &wi_out) {
    const int i = (int)(nd.y & 255u);
    const uint32_t z = (nd.y >> 8) & 15u;
    const uint32_t g = (nd.y >> 12) & 15u;
    const uint32_t k = nd.z, l = nd.w;
    const uint32_t wi = qv.w((uint32_t)i);
    wi_out = wi;
    bool ins_r = true, mis_r = true, del_r = true, match_r = true;
    uint32_t del_keep = 0xfu;
    uint32_t wp = 4u;   // W[i-1] when the rules need it, else a value no symbol has
    if (c.canon) {
        const uint32_t op = (nd.y >> 16) & 3u, pb = (nd.y >> 18) & 3u;
        if (op == kOpIns || op == kOpMis) {
            const uint32_t wn = qv.w((uint32_t)i + 1u);
            if (op == kOpIns) {
                del_r = false;
                mis_r = false;
                match_r = wi != wn;
            } else {
                ins_r = pb != wi;
                del_keep = 0xfu & ~(1u << wn);
            }
        } else if (op == kOpDel) {
            ins_r = false;
            if (i >= 1) {
                mis_r = false;
                match_r = wi != pb;
            }
        }
        if (i >= 1) wp = qv.w((uint32_t)i - 1u);
    }
    if (c.end_skip) {
        const uint32_t m = qv.len(), e = c.end_skip;
        if ((uint32_t)i < e || (uint32_t)i + e >= m) ins_r = false;
        if ((uint32_t)i + 1u < e || (uint32_t)i + e >= m) del_r = false;
    }
    const uint32_t max_gaps = qv.gaps();
    const bool gap_ok = z >= 1u && g < max_gaps;
    const bool need = (gap_ok && del_r) || (z >= 1u && mis_r) || match_r;
    // a new indel child can take another indel only with a gap and a difference to spare
    const bool more_gaps = g + 1u < max_gaps && z >= 2u;
    const bool shallow = (nd.y & kShallow) != 0u;
    const uint32_t d = (nd.y >> 20) & 15u;
    uint32_t alive = 0;   // bit b: the child string bX occurs
    nblocks = 0;
    counted = need ? 1u : 0u;
    if (need && shallow) {
        // k holds code(X); the children's codes are 4 code(X) + b
        alive = kt_occ4(c.ix, d + 1u, k);
        if (d + 1u < c.ix.kdepth) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                k2[b] = 4u * k + (uint32_t)b;
                l2[b] = 0u;
            }
        } else {
            kt_get4(c.ix, d + 1u, k, k2, l2);
            nblocks = kTabRead;
        }
    } else if (need) {
        const uint32_t pk = k, pl = l + 1u;
        const uint32_t jk = pk / I, jl = pl / I;
        const uint32_t ok = pk - jk * I, ol = pl - jl * I;
        // every lane runs the same counting code on (Bk, Bl), Bl a copy when they share a block
        Blk<I> Bk, Bl;
        if (jk == jl) {
            load_block<I>(c.ix.blocks, jk, ok > ol ? ok : ol, Bk);
            Bl = Bk;
            nblocks = 1;
        } else {
            load_block<I>(c.ix.blocks, jk, ok, Bk);
            load_block<I>(c.ix.blocks, jl, ol, Bl);
            nblocks = 2;
        }
        uint32_t rk[4], rl[4];
        rank4_in<I>(Bk, jk, pk, c.ix.dollar, rk);
        rank4_in<I>(Bl, jl, pl, c.ix.dollar, rl);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            k2[b] = c.ix.C[b] + rk[b] + 1u;
            l2[b] = c.ix.C[b] + rl[b];
            alive |= (k2[b] <= l2[b] ? 1u : 0u) << b;
        }
    }
    const uint32_t d_here = qv.d(i);
    const uint32_t d_next = qv.d(i - 1);
    const bool del_ok = gap_ok && del_r && z - 1u >= d_here;
    const bool last = i == 0;
    push = 0;
    leaf = 0;
    // insertion: W[i] against no reference symbol, interval unchanged; the child at i-1 can
    // only insert again when W[i-1] = W[i] (rules on)
    if (gap_ok && ins_r) {
        if (last) {
            if (shallow ? d >= 1u : k >= 1u) leaf |= 1u;   // X non-empty
        } else if (z - 1u >= d_next && (wp != wi || more_gaps)) {
            push |= 1u;
        }
    }
    const bool mm_ok = z >= 1u && mis_r && (last || z - 1u >= d_next);   // a mismatch child survives
    const bool ma_ok = match_r && (last || z >= d_next);                 // the match child survives
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const bool ne = (alive >> b) & 1u;
        const bool keep = (uint32_t)b == wi ? ma_ok : mm_ok;
        const uint32_t mm = (ne && keep) ? (32u << b) : 0u;
        if (last) leaf |= mm; else push |= mm;
    }
    if (del_ok) {
        // deletion of each b with a non-empty interval; at i >= 1 the child deleting b = W[i]
        // can only delete again (rules on)
        uint32_t dm = alive & del_keep;
        if (c.canon && !last && !more_gaps) dm &= ~(1u << wi);
        push |= dm << 1;
    }
}

// One call of InexRecur with no difference left (z = 0): only the match b = W[i] can continue,
// so the eight-Occ step reduces to rank(W[i], k) and rank(W[i], l+1), i.e. one step of
// Listing 1.  The single child replaces the node (out), or the interval is a result (leaf at
// i = 0), or the branch ends (empty interval).  The child needs no D test: every node is
// created with z >= D(i), D never decreases with i, so here D(i-1) <= D(i) = 0.  Only the
// query's symbols are used.
//
// A shallow node (its string X shorter than the table depth L) runs all of its steps inside the
// tables at once: the symbols it will prepend are W[i], W[i-1], ..., so after t steps its
// string is W[i-t+1..i] X, of code code(X) 4^t + sum_s W[i-s] 4^(t-1-s).  With
// tmax = min(L - d, i + 1) steps left in the tables, the string after tmax steps is tested
// first: its table entry, whose k <= l says it occurs (an empty string's entry holds its
// insertion point, k = l + 1); otherwise the longest occurring prefix length t is found by
// bisection over occurrence bits (longer strings occur only if their shorter suffixes do, and
// the code after t steps is the code after tmax steps shifted right by 2 (tmax - t)).  The
// chain then ends after t + 1 steps, or after tmax steps becomes a result (i reaches -1) or an
// interval node at depth L.  nn counts the steps, as the one-step walk would count its nodes.
template <int I, class Q>
__device__ __forceinline__ void exact_step(const SearchCfg &c, const uint4 &nd, const Q &qv,
                                           uint4 &out, bool &survive, bool &is_leaf,
                                           uint32_t &nblocks, uint32_t &nn) {
    const uint32_t i = nd.y & 255u;
    const uint32_t k = nd.z, l = nd.w;
    const uint32_t ybits = nd.y & (0xf000u | kSlotBits);   // z = 0, created by a match
    if (nd.y & kShallow) {
        const uint32_t d = (nd.y >> 20) & 15u;
        const uint32_t left = c.ix.kdepth - d;
        const uint32_t tmax = left < i + 1u ? left : i + 1u;
        uint32_t code = k;
        for (uint32_t s = 0; s < tmax; ++s) code = 4u * code + qv.w(i - s);
        const uint2 kl = kt_get(c.ix, d + tmax, code);
        nblocks = kTabRead;
        if (kl.x > kl.y) {
            uint32_t lo = 0, hi = tmax - 1u;   // X itself occurs (the node exists)
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1u) >> 1;
                if (kt_occ1(c.ix, d + mid, code >> (2u * (tmax - mid)))) lo = mid; else hi = mid - 1u;
            }
            nn = lo + 1u;
            survive = false;
            is_leaf = false;
            out = nd;
            return;
        }
        nn = tmax;
        is_leaf = tmax == i + 1u;
        survive = !is_leaf;
        out = make_uint4(nd.x, (i - tmax) | ybits, kl.x, kl.y);
        return;
    }
    const uint32_t b = qv.w(i);
    const uint32_t pk = k, pl = l + 1u;
    const uint32_t jk = pk / I, jl = pl / I;
    const uint32_t ok = pk - jk * I, ol = pl - jl * I;
    // C[b] by select: a runtime index into the parameter struct would copy it to local memory
    const uint32_t cb = b == 0 ? c.ix.C[0] : (b == 1 ? c.ix.C[1] : (b == 2 ? c.ix.C[2] : c.ix.C[3]));
    Blk<I> Bk, Bl;
    if (jk == jl) {
        load_block<I>(c.ix.blocks, jk, ok > ol ? ok : ol, Bk);
        Bl = Bk;
        nblocks = 1;
    } else {
        load_block<I>(c.ix.blocks, jk, ok, Bk);
        load_block<I>(c.ix.blocks, jl, ol, Bl);
        nblocks = 2;
    }
    const uint32_t k2 = cb + rank1_in<I>(Bk, jk, pk, c.ix.dollar, b) + 1u;
    const uint32_t l2 = cb + rank1_in<I>(Bl, jl, pl, c.ix.dollar, b);
    const bool alive = k2 <= l2;
    nn = 1u;
    is_leaf = alive && i == 0u;
    survive = alive && i > 0u;
    out = make_uint4(nd.x, (i - 1u) | ybits, k2, l2);
}

// One exact continuation over two symbols: the interval of W[i-1] W[i] X from that of X through
// the pair table, for interval (not shallow) nodes with i >= 1.  When non-empty it is the
// interval of two single steps, both of whose nodes are counted (nn = 2); when empty the
// branch ends either way and only this node is counted (the middle one may or may not have
// been non-empty).  Sectors read go to the table-sector field of nblocks.
template <int I, class Q>
__device__ __forceinline__ void pair_step(const SearchCfg &c, const uint4 &nd, const Q &qv,
                                          uint4 &out, bool &survive, bool &is_leaf,
                                          uint32_t &nblocks, uint32_t &nn) {
    const uint32_t i = nd.y & 255u;
    const uint32_t b2 = qv.w(i), b1 = qv.w(i - 1u);
    const uint32_t pc = 4u * b1 + b2, pk = nd.z, pl = nd.w + 1u;
    const uint32_t jk = pk / kPairRows, jl = pl / kPairRows;
    const uint32_t c2 = __ldg(c.ix.pc2 + pc);
    const uint2 Rk = load_pair_rec(c.ix, pc, jk);   // one record when k and l+1 share a block
    const uint2 Rl = jl == jk ? Rk : load_pair_rec(c.ix, pc, jl);
    const uint32_t k2 = c2 + pair_rank(Rk, pk);
    const uint32_t l2 = c2 + pair_rank(Rl, pl) - 1u;
    const bool alive = k2 <= l2;
    nblocks = (jl == jk ? 1u : 2u) * kTabRead;
    nn = alive ? 2u : 1u;
    is_leaf = alive && i == 1u;
    survive = alive && i >= 2u;
    out = make_uint4(nd.x, (i - 2u) | (nd.y & (0xf000u | kSlotBits)), k2, l2);
}

// an exact continuation: two symbols from the pair table where it applies, else one
template <int I, class Q>
__device__ __forceinline__ void chain_step(const SearchCfg &c, const uint4 &nd, const Q &qv,
                                           uint4 &out, bool &survive, bool &is_leaf,
                                           uint32_t &nblocks, uint32_t &nn) {
    if (c.ix.pairs && !(nd.y & kShallow) && (nd.y & 255u) >= 1u) {
        pair_step<I>(c, nd, qv, out, survive, is_leaf, nblocks, nn);
    } else {
        exact_step<I>(c, nd, qv, out, survive, is_leaf, nblocks, nn);
    }
}

__device__ __forceinline__ uint32_t pick4(const uint32_t v[4], uint32_t b) {
    return b == 0 ? v[0] : (b == 1 ? v[1] : (b == 2 ? v[2] : v[3]));
}

// child number t (0 insertion, 1..4 deletion, 5..8 match/mismatch) of node nd
__device__ __forceinline__ uint4 make_child(const uint4 &nd, int t, const uint32_t k2[4],
                                            const uint32_t l2[4], uint32_t wi, uint32_t kdepth) {
    const uint32_t i = nd.y & 255u;
    const uint32_t z = (nd.y >> 8) & 15u;
    const uint32_t g = (nd.y >> 12) & 15u;
    const uint32_t d = (nd.y >> 20) & 15u;
    // a child one symbol longer stays shallow below the table depth
    const uint32_t sh = (((nd.y & kShallow) && d + 1u < kdepth) ? (kShallow | ((d + 1u) << 20)) : 0u) |
                        (nd.y & kSlotBits);
    uint4 ch;
    ch.x = nd.x;
    if (t == 0) {
        ch.y = (i - 1u) | ((z - 1u) << 8) | ((g + 1u) << 12) | (kOpIns << 16) |
               (nd.y & (kShallow | kDepthBits | kSlotBits));
        ch.z = nd.z;
        ch.w = nd.w;
    } else if (t <= 4) {
        const uint32_t b = (uint32_t)(t - 1);
        ch.y = i | ((z - 1u) << 8) | ((g + 1u) << 12) | (kOpDel << 16) | (b << 18) | sh;
        ch.z = pick4(k2, b);
        ch.w = pick4(l2, b);
    } else {
        const uint32_t b = (uint32_t)(t - 5);
        const uint32_t zc = b == wi ? z : z - 1u;
        ch.y = (i - 1u) | (zc << 8) | (g << 12) | (b == wi ? 0u : (kOpMis << 16) | (b << 18)) | sh;
        ch.z = pick4(k2, b);
        ch.w = pick4(l2, b);
    }
    return ch;
}

// interval of leaf child t (0 insertion, 5..8 match/mismatch) of node nd
__device__ __forceinline__ uint2 leaf_of(const SearchCfg &c, const uint4 &nd, int t,
                                         const uint32_t k2[4], const uint32_t l2[4]) {
    const bool sh = (nd.y & kShallow) != 0u;
    const uint32_t d = (nd.y >> 20) & 15u;
    if (t == 0) return sh ? kt_get(c.ix, d, nd.z) : make_uint2(nd.z, nd.w);
    const uint32_t b = (uint32_t)(t - 1) & 3u;
    if (sh && d + 1u < c.ix.kdepth) return kt_get(c.ix, d + 1u, pick4(k2, b));
    return make_uint2(pick4(k2, b), pick4(l2, b));
}

__device__ __forceinline__ uint4 root_of(const SearchCfg &c, uint32_t q, const uint4 &mt,
                                         bool &ok) {
    const uint32_t m = mt.w & 255u;
    const uint32_t z0 = (mt.w >> 16) & 15u;   // the query's differences allowed
    ok = m >= 1u && z0 >= d_at(mt, (int)m - 1);
    if (c.ix.kdepth) return make_uint4(q, (m - 1u) | (z0 << 8) | kShallow, 0u, 0u);   // X empty
    return make_uint4(q, (m - 1u) | (z0 << 8), 0u, c.ix.n);
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// append this warp's leaves to the raw buffer: (query, k, l, differences used); z0 is the
// query's differences allowed, q its number
__device__ __forceinline__ void emit_leaves(const SearchCfg &c, int lane, bool act,
                                            const uint4 &nd, uint32_t leaf, const uint32_t k2[4],
                                            const uint32_t l2[4], uint32_t wi, uint32_t z0,
                                            uint32_t q) {
    if (!__any_sync(FULL, act && leaf != 0u)) return;
    const int lc = act ? __popc(leaf) : 0;
    const int incl = warp_incl_scan(lc, lane);
    const int tot = __shfl_sync(FULL, incl, 31);
    if (tot == 0) return;
    unsigned long long base = 0;
    if (lane == 31) base = atomicAdd(c.raw_count, (unsigned long long)tot);
    base = __shfl_sync(FULL, base, 31);
    uint64_t pos = base + (uint64_t)(incl - lc);
    uint32_t mset = act ? leaf : 0u;
    while (mset) {
        const int t = __ffs(mset) - 1;
        mset &= mset - 1;
        if (pos < c.raw_cap) {
            const uint2 kl = leaf_of(c, nd, t, k2, l2);
            // z left after the leaf column: the match keeps z, insertion and mismatch spend one
            const uint32_t zl = ((nd.y >> 8) & 15u) - ((t >= 5 && (uint32_t)(t - 5) == wi) ? 0u : 1u);
            c.raw[pos] = make_uint4(q, kl.x, kl.y, z0 - zl);
        }
        ++pos;
    }
}

// ------------------------------------------------------------------------------------------
// persistent kernel
// ------------------------------------------------------------------------------------------
// Each warp keeps two node pools in one shared-memory array of stk entries: G (nodes with
// z >= 1, growing up from entry 0) and E (nodes with z = 0, growing down from entry stk-1).
// E nodes are exact continuations (one cheap step each, the child replacing the node); G nodes
// take the full eight-value expansion.  Policy per step:
//   * E holds >= 32 nodes, or only E has work: exact steps (below) until E runs dry;
//   * else a G step: up to min(32, (stk - |E|) / 9) G nodes expanded, so that their children
//     (at most 9 each) always fit beside E once G is out of the way; children with z' = 0 go
//     to E, the others to G (two warp prefix sums); if they would not fit, G is first moved to
//     the warp's spill region in device memory (E holds < 32 nodes at a G step);
//   * G empty but spilled nodes waiting: reload a batch;
//   * pools below the refill level: take up to `chunk` queries from the work queue and push
//     their roots (with STAGE, no more queries than the free slot groups hold, each staged in
//     a slot).
// A warp leaves when the queue is drained and both pools and its spill are empty.
//
// STAGE: every query a warp works on is staged in one of its shared-memory slots (its 2-bit
// symbols oriented for its strand, D breakpoints, length, search mode and number), so that no
// expansion or exact step reads query data from device memory.  Slots are taken and freed in
// groups of kGroupSlots.  The warp keeps, in registers, the number of live nodes of each
// group's queries (nodes in the pools, in the spill region or held by a lane): a G step adds,
// per group, the children of its nodes minus the nodes (one warp reduction per group), and the
// exact chains that end during an exact phase are counted per lane and subtracted when the
// phase ends (or every kFlushSteps steps).  A count can only lag behind, never run ahead, so a
// group is freed only when no node of its queries is left.  Every group a warp holds has a
// live node, so the warp never waits for a slot.  Without STAGE the query data is read through
// L1 from the staging records in device memory.
constexpr int kFlushSteps = 512;   // exact steps between two flushes of the ended-chain counts
constexpr int kPoolEntries = 320;  // node pool entries per warp

// PROF: the instantiation that counts the step fill (c.fill); the counting is compiled out of
// the others, where its live state alone cost 6% of the search time under the 64-register cap.
template <int I, bool STAGE, bool PROF>
__global__ void __launch_bounds__(256, I <= 128 ? 4 : 2) k_inexact_persistent(SearchCfg c, int stk, uint4 *spill_all,
                                                            uint32_t spill_cap) {
    extern __shared__ uint4 smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    constexpr bool prof = PROF;
    uint32_t *wbase = reinterpret_cast<uint32_t *>(smem) + (size_t)wib * warp_smem_words(stk, STAGE, prof);
    Pool<STAGE> st;
    if constexpr (STAGE) {
        st.y = wbase;
        st.k = wbase + stk;
        st.l = wbase + 2 * stk;
    } else {
        st.e = reinterpret_cast<uint4 *>(wbase);
    }
    uint32_t *slots = wbase + Pool<STAGE>::kWords * stk;                // kSlots x kSlotWords
    uint32_t *fillc = slots + (STAGE ? kSlots * kSlotWords : 0);         // step-fill counters
    const uint64_t gw = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    uint4 *spill = spill_all + gw * spill_cap;
    const uint32_t lt_mask = (1u << lane) - 1u;
    int gtop = 0;         // G: entries [0, gtop)
    int etop = 0;         // E: entries [stk - etop, stk), top at stk - etop
    uint32_t stop = 0;    // spilled G nodes (warp-uniform)
    bool qdone = false;
    uint32_t fgroups = (1u << kGroups) - 1u;   // free slot groups (warp-uniform)
    int gcount[kGroups];                       // live nodes per slot group (warp-uniform)
#pragma unroll
    for (int g = 0; g < kGroups; ++g) gcount[g] = 0;
    // this lane's nodes, checkpoint blocks and table sectors (32 bits: a lane expands well
    // under 2^32 nodes in one launch)
    uint32_t my_nodes = 0, my_blocks = 0, my_sects = 0;
    if (prof && lane < kFillCounters) fillc[lane] = 0u;
    __syncwarp();
    // metadata records: with STAGE the staging records (kStageU4 uint4 per query, the query's
    // symbols after its metadata word), else one uint4 per query
    constexpr uint32_t QS = STAGE ? kStageU4 : 1u;
    // the query data of node nd (with q, its number without STAGE)
    auto query = [&](const uint4 &nd) {
        if constexpr (STAGE) return SQuery{slots + slot_of(nd) * kSlotWords};
        else return GQuery{c.reads, c.qmeta[nd.x]};
    };
    // group counts: add the per-lane changes delta of the lanes holding a node of group g
    auto count_groups = [&](bool has, uint32_t grp, int delta) {
#pragma unroll
        for (int g = 0; g < kGroups; ++g) {
            gcount[g] += __reduce_add_sync(FULL, (has && grp == (uint32_t)g) ? delta : 0);
            if (gcount[g] == 0) fgroups |= 1u << g;
        }
    };

    for (;;) {
        if (gtop + etop < (int)c.refill && stop == 0 && !qdone && (!STAGE || fgroups != 0u)) {
            const uint32_t room = STAGE ? (uint32_t)(__popc(fgroups) * kGroupSlots) : 32u;
            const uint32_t take = c.chunk < room ? c.chunk : room;
            uint32_t q0 = 0;
            if (lane == 0) q0 = atomicAdd(c.next_q, take);
            q0 = __shfl_sync(FULL, q0, 0);
            if (q0 >= c.nq) {
                qdone = true;
            } else {
                const uint32_t q = q0 + lane;
                bool ok = false;
                uint4 nd = make_uint4(0, 0, 0, 0);
                uint32_t grp = 0;
                if ((uint32_t)lane < take && q < c.nq) {
                    const uint4 *src = c.qmeta + (size_t)q * QS;
                    const uint4 mt = src[0];
                    const uint32_t m = mt.w & 255u, z0 = (mt.w >> 16) & 15u;
                    ok = m >= 1u && z0 >= d_at(mt, (int)m - 1);
                    uint32_t sb = 0;
                    if constexpr (STAGE) {
                        uint32_t fg = fgroups;   // lanes 4j..4j+3 take the j-th free group
                        for (int t = 0; t < lane / kGroupSlots; ++t) fg &= fg - 1u;
                        grp = (uint32_t)__ffs(fg) - 1u;
                        const uint32_t sl = grp * kGroupSlots + (uint32_t)(lane % kGroupSlots);
                        uint4 *dst = reinterpret_cast<uint4 *>(slots + sl * kSlotWords);
                        dst[0] = src[1];
                        dst[1] = src[2];
                        dst[2] = src[3];
                        dst[3] = src[4];
                        dst[4] = make_uint4(mt.x, mt.y, m | (mt.w & 0x00ff0000u), q);
                        sb = sl << kSlotShift;
                    }
                    nd = c.ix.kdepth ? make_uint4(q, (m - 1u) | (z0 << 8) | kShallow | sb, 0u, 0u)
                                     : make_uint4(q, (m - 1u) | (z0 << 8) | sb, 0u, c.ix.n);
                }
                if constexpr (STAGE) {
                    // groups that received a root are taken (the rest stay free)
                    count_groups(ok, grp, 1);
                    fgroups &= ~__reduce_or_sync(FULL, ok ? 1u << grp : 0u);
                }
                // roots with no difference allowed are exact continuations (E), the rest G
                const bool ex = ok && ((nd.y >> 8) & 15u) == 0u;
                const uint32_t bale = __ballot_sync(FULL, ex), balg = __ballot_sync(FULL, ok && !ex);
                if (ex) st.put(stk - 1 - (etop + __popc(bale & lt_mask)), nd);
                if (ok && !ex) st.put(gtop + __popc(balg & lt_mask), nd);
                etop += __popc(bale);
                gtop += __popc(balg);
                if (prof && lane == 0) {
                    fillc[5] += 1u;
                    fillc[6] += __popc(bale | balg);
                }
                __syncwarp();
            }
        }
        if (etop >= 32 || (etop > 0 && gtop == 0 && stop == 0)) {
            // Exact steps: each lane holds up to two chains (n0, n1).  A chain stays in its lane
            // from step to step; a lane whose first chain ended moves its second one up, and
            // free chain places are refilled from E.  Second chains are stepped only while at
            // least chain2_min lanes hold one (otherwise they wait for a first place, so that
            // a sparse second pass does not run with most lanes idle).  The phase ends when
            // fewer than 32 chains are live and E is empty (unless nothing else is left to
            // do), and the survivors go back to E (fewer than 32, so E stays below 32 for the
            // next G step).
            uint4 n0 = make_uint4(0, 0, 0, 0), n1 = make_uint4(0, 0, 0, 0);
            uint2 r0 = make_uint2(0, 0), r1 = make_uint2(0, 0);   // without STAGE: chain_base
            bool a0 = false, a1 = false;
            uint32_t ended01 = 0, ended23 = 0;   // STAGE: ended chains of groups 0..3, 16-bit fields
            int since_flush = 0;
            auto flush = [&]() {
                if constexpr (STAGE) {
#pragma unroll
                    for (int g = 0; g < kGroups; ++g) {
                        const uint32_t w = g < 2 ? ended01 : ended23;
                        gcount[g] -= __reduce_add_sync(FULL, (int)((w >> (16 * (g & 1))) & 0xffffu));
                        if (gcount[g] == 0) fgroups |= 1u << g;
                    }
                    ended01 = ended23 = 0;
                }
            };
            for (;;) {
                if (!a0 && a1) {
                    n0 = n1;
                    r0 = r1;
                    a0 = true;
                    a1 = false;
                }
                // refill free chain places from E (first places first)
                {
                    const uint32_t f0 = __ballot_sync(FULL, !a0), f1 = __ballot_sync(FULL, !a1);
                    const int nf0 = __popc(f0);
                    const int t0 = nf0 < etop ? nf0 : etop;
                    const int p0 = __popc(f0 & lt_mask);
                    if (!a0 && p0 < t0) {
                        n0 = st.get(stk - etop + p0);
                        if constexpr (!STAGE) {
                            r0 = chain_base(c.qmeta[n0.x]);
                        }
                        a0 = true;
                    }
                    const int rest = etop - t0;
                    const int t1 = __popc(f1) < rest ? __popc(f1) : rest;
                    const int p1 = __popc(f1 & lt_mask);
                    if (!a1 && p1 < t1) {
                        n1 = st.get(stk - etop + t0 + p1);
                        if constexpr (!STAGE) {
                            r1 = chain_base(c.qmeta[n1.x]);
                        }
                        a1 = true;
                    }
                    etop -= t0 + t1;
                    __syncwarp();
                }
                const int live1 = __popc(__ballot_sync(FULL, a1));
                const bool step1 = a1 && live1 >= (int)c.chain2_min;
                uint4 c0 = make_uint4(0, 0, 0, 0), c1 = make_uint4(0, 0, 0, 0);
                bool s0 = false, s1 = false, e0 = false, e1 = false;
                uint32_t b0 = 0, b1 = 0, x0 = 0, x1 = 0;
                auto cq = [&](const uint4 &n, const uint2 &r) {
                    if constexpr (STAGE) return SQuery{slots + slot_of(n) * kSlotWords};
                    else return CQuery{c.reads, r.x, r.y};
                };
                if (a0) {
                    chain_step<I>(c, n0, cq(n0, r0), c0, s0, e0, b0, x0);
                    my_nodes += x0;
                    my_blocks += b0 & 0xffffu;
                    my_sects += b0 >> 16;
                }
                if (step1) {
                    chain_step<I>(c, n1, cq(n1, r1), c1, s1, e1, b1, x1);
                    my_nodes += x1;
                    my_blocks += b1 & 0xffffu;
                    my_sects += b1 >> 16;
                }
                if (prof) {   // warp-uniform
                    const int live0 = __popc(__ballot_sync(FULL, a0));
                    if (lane == 0) {
                        fillc[0] += 1u;
                        fillc[1] += (uint32_t)live0;
                        fillc[2] += live1 >= (int)c.chain2_min ? (uint32_t)live1 : 0u;
                        fillc[7] += (live1 > 0 && live1 < (int)c.chain2_min) ? 1u : 0u;
                    }
                }
                const uint32_t lb0 = __ballot_sync(FULL, e0), lb1 = __ballot_sync(FULL, e1);
                if (lb0 | lb1) {
                    unsigned long long base = 0;
                    if (lane == 0)
                        base = atomicAdd(c.raw_count, (unsigned long long)(__popc(lb0) + __popc(lb1)));
                    base = __shfl_sync(FULL, base, 0);
                    const uint64_t q0 = base + __popc(lb0 & lt_mask);
                    const uint64_t q1 = base + __popc(lb0) + __popc(lb1 & lt_mask);
                    // a z = 0 leaf used all of its query's differences
                    if constexpr (STAGE) {
                        if (e0 && q0 < c.raw_cap) {
                            const SQuery qv = cq(n0, r0);
                            c.raw[q0] = make_uint4(qv.q(), c0.z, c0.w, qv.z0());
                        }
                        if (e1 && q1 < c.raw_cap) {
                            const SQuery qv = cq(n1, r1);
                            c.raw[q1] = make_uint4(qv.q(), c1.z, c1.w, qv.z0());
                        }
                    } else {
                        if (e0 && q0 < c.raw_cap) c.raw[q0] = make_uint4(n0.x, c0.z, c0.w, cq(n0, r0).z0());
                        if (e1 && q1 < c.raw_cap) c.raw[q1] = make_uint4(n1.x, c1.z, c1.w, cq(n1, r1).z0());
                    }
                }
                if constexpr (STAGE) {   // an ended chain: one node less for its group
                    if (a0 && !s0) {
                        const uint32_t g = slot_of(n0) / kGroupSlots;
                        (g < 2 ? ended01 : ended23) += 1u << (16u * (g & 1u));
                    }
                    if (step1 && !s1) {
                        const uint32_t g = slot_of(n1) / kGroupSlots;
                        (g < 2 ? ended01 : ended23) += 1u << (16u * (g & 1u));
                    }
                    if (++since_flush == kFlushSteps) {
                        flush();
                        since_flush = 0;
                    }
                }
                if (s0) n0 = c0;
                if (s1) n1 = c1;
                a0 = s0;
                if (step1) a1 = s1;
                const int live = __popc(__ballot_sync(FULL, a0)) + __popc(__ballot_sync(FULL, a1));
                if (live == 0 && etop == 0) break;
                if (live < 32 && etop == 0 && !(gtop == 0 && stop == 0 && qdone)) {
                    // survivors back to E
                    const uint32_t v0 = __ballot_sync(FULL, a0), v1 = __ballot_sync(FULL, a1);
                    if (a0) st.put(stk - 1 - (etop + __popc(v0 & lt_mask)), n0);
                    if (a1) st.put(stk - 1 - (etop + __popc(v0) + __popc(v1 & lt_mask)), n1);
                    etop += __popc(v0) + __popc(v1);
                    __syncwarp();
                    break;
                }
            }
            flush();
            continue;
        }
        // nodes one G step may take: their children (at most 9 each) fit beside E
        const int cap_take = min(32, (stk - etop) / 9);
        if (gtop == 0 && stop > 0) {
            // reload spilled G nodes: one G step takes cap_take of them and pushes at most
            // 9 cap_take children, so stk - |E| - 8 cap_take (>= cap_take) fit without a spill
            const int room = stk - etop - 8 * cap_take;
            const uint32_t nmove = stop < (uint32_t)room ? stop : (uint32_t)room;
            for (uint32_t t = lane; t < nmove; t += 32) st.put((int)t, spill[stop - nmove + t]);
            stop -= nmove;
            gtop = (int)nmove;
            __syncwarp();
            continue;
        }
        if (gtop == 0) {
            if (etop == 0 && stop == 0) {
                if (qdone) break;
                if constexpr (STAGE) {
                    // the warp holds no node: every slot group is empty (this also frees the
                    // groups of nodes dropped on a spill overflow, whose pass is rerun)
                    fgroups = (1u << kGroups) - 1u;
#pragma unroll
                    for (int g = 0; g < kGroups; ++g) gcount[g] = 0;
                }
            }
            continue;
        }
        // general step on up to cap_take G nodes
        const int take = gtop < cap_take ? gtop : cap_take;
        const bool act = lane < take;
        uint4 nd = make_uint4(0, 0, 0, 0);
        if (act) nd = st.get(gtop - 1 - lane);
        gtop -= take;
        __syncwarp();
        uint32_t k2[4] = {0, 0, 0, 0}, l2[4] = {0, 0, 0, 0}, push = 0, leaf = 0, nb = 0, wi = 0;
        uint32_t z0 = 0, qn = nd.x;   // the query's differences allowed, and its number
        if (act) {
            const auto qv = query(nd);
            uint32_t cn = 0;
            expand<I>(c, nd, qv, k2, l2, push, leaf, nb, cn, wi);
            z0 = qv.z0();
            if constexpr (STAGE) qn = qv.q();
            my_nodes += cn;
            my_blocks += nb & 0xffffu;
            my_sects += nb >> 16;
        }
        if (prof && lane == 0) {
            fillc[3] += 1u;
            fillc[4] += (uint32_t)take;
        }
        // children with z' = 0 (every child but the match of a z = 1 node) go to E
        const uint32_t z = (nd.y >> 8) & 15u;
        const uint32_t emask = z == 1u ? (push & ~(32u << wi)) : 0u;
        const uint32_t gmask = push & ~emask;
        const int gc = __popc(gmask), ec = __popc(emask);
        const int gincl = warp_incl_scan(gc, lane);
        const int eincl = warp_incl_scan(ec, lane);
        const int gtot = __shfl_sync(FULL, gincl, 31);
        const int etot = __shfl_sync(FULL, eincl, 31);
        if (gtop + gtot + etop + etot > stk) {
            // pools full: move G to the spill region
            if (stop + (uint32_t)gtop > spill_cap) {
                if (lane == 0) atomicOr(c.err, kErrSpill);
                gtop = 0;   // work dropped: the host grows the spill region and reruns
            } else {
                for (int t = lane; t < gtop; t += 32) spill[stop + t] = st.get(t);
                stop += (uint32_t)gtop;
                gtop = 0;
            }
            __syncwarp();
        }
        {
            int gpos = gtop + gincl - gc;
            int epos = etop + eincl - ec;
            uint32_t mset = push;
            while (mset) {
                const int t = __ffs(mset) - 1;
                mset &= mset - 1;
                const uint4 chd = make_child(nd, t, k2, l2, wi, c.ix.kdepth);
                if ((emask >> t) & 1u) st.put(stk - 1 - (epos++), chd);
                else st.put(gpos++, chd);
            }
        }
        gtop += gtot;
        etop += etot;
        // live nodes per slot group: the children replace the expanded node
        if constexpr (STAGE) count_groups(act, slot_of(nd) / kGroupSlots, gc + ec - 1);
        emit_leaves(c, lane, act, nd, leaf, k2, l2, wi, z0, qn);
        __syncwarp();
    }
    if (c.stats) {
        unsigned long long tn = my_nodes, tb = my_blocks, ts = my_sects;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tn += __shfl_down_sync(FULL, tn, o);
            tb += __shfl_down_sync(FULL, tb, o);
            ts += __shfl_down_sync(FULL, ts, o);
        }
        if (lane == 0) {
            atomicAdd(c.stats + 0, tn);
            atomicAdd(c.stats + 1, tb);
            atomicAdd(c.stats + 3, ts);
        }
    }
    if (prof) {
        __syncwarp();
        if (lane < kFillCounters) atomicAdd(c.fill + lane, (unsigned long long)fillc[lane]);
    }
}

// ------------------------------------------------------------------------------------------
// plain kernel: one thread per query, depth-first
// ------------------------------------------------------------------------------------------
template <int I>
__global__ void __launch_bounds__(256) k_inexact_plain(SearchCfg c, uint4 *stacks, uint32_t cap,
                                                       uint32_t T) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= T) return;   // T is a multiple of 32: whole warps leave
    const int lane = threadIdx.x & 31;
    unsigned long long my_nodes = 0, my_blocks = 0;
    // every lane of a warp iterates until the whole warp is done (warp-synchronous leaves)
    uint32_t q = tid;
    uint32_t sp = 0;
    bool have = false;
    // a node with z = 0 is continued in place (one Listing 1 step per loop iteration) instead of
    // being pushed and popped
    bool cur = false;
    uint4 curnd = make_uint4(0, 0, 0, 0);
    for (;;) {
        // fetch the next query when the stack is empty
        while (!have && q < c.nq) {
            bool ok;
            uint4 mt = c.qmeta[q];
            uint4 r = root_of(c, q, mt, ok);
            if (ok) {
                stacks[(size_t)tid] = r;
                sp = 1;
                have = true;
            }
            q += T;
        }
        const bool act = have;
        if (!__any_sync(FULL, act)) break;
        uint4 nd = make_uint4(0, 0, 0, 0);
        uint32_t k2[4] = {0, 0, 0, 0}, l2[4] = {0, 0, 0, 0}, push = 0, leaf = 0, nb = 0, wi = 0;
        uint32_t counted = 1;   // an exact step is always a counted node
        uint32_t z0 = 0;        // the query's differences allowed
        bool ex_leaf = false;
        uint4 ex_out = make_uint4(0, 0, 0, 0);
        if (act) {
            if (cur) {
                nd = curnd;
            } else {
                nd = stacks[(size_t)(sp - 1) * T + tid];
                --sp;
            }
            cur = false;
            const GQuery qv{c.reads, c.qmeta[nd.x]};
            z0 = qv.z0();
            if (((nd.y >> 8) & 15u) == 0u) {
                bool survive = false;
                chain_step<I>(c, nd, qv, ex_out, survive, ex_leaf, nb, counted);
                if (survive) {
                    curnd = ex_out;
                    cur = true;
                }
            } else {
                expand<I>(c, nd, qv, k2, l2, push, leaf, nb, counted, wi);
                uint32_t mset = push;
                while (mset) {
                    const int t = __ffs(mset) - 1;
                    mset &= mset - 1;
                    if (sp < cap) {
                        stacks[(size_t)sp * T + tid] = make_child(nd, t, k2, l2, wi, c.ix.kdepth);
                        ++sp;
                    } else {
                        atomicOr(c.err, kErrStack);
                    }
                }
            }
            my_nodes += counted;
            my_blocks += step_cost(nb);
            if (sp == 0 && !cur) have = false;
        }
        emit_leaves(c, lane, act, nd, leaf, k2, l2, wi, z0, nd.x);
        const uint32_t lb = __ballot_sync(FULL, ex_leaf);
        if (lb) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(c.raw_count, (unsigned long long)__popc(lb));
            base = __shfl_sync(FULL, base, 0);
            const uint64_t pos = base + __popc(lb & ((1u << lane) - 1u));
            if (ex_leaf && pos < c.raw_cap) c.raw[pos] = make_uint4(nd.x, ex_out.z, ex_out.w, z0);
        }
    }
    if (c.stats) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            my_nodes += __shfl_down_sync(FULL, my_nodes, o);
            my_blocks += __shfl_down_sync(FULL, my_blocks, o);
        }
        if (lane == 0) {
            atomicAdd(c.stats + 0, my_nodes);
            atomicAdd(c.stats + 1, my_blocks & 0xffffffffull);
            atomicAdd(c.stats + 3, my_blocks >> 32);
        }
    }
}

// ------------------------------------------------------------------------------------------
// canonical result sets
// ------------------------------------------------------------------------------------------
// raw results: R = min(*d_R, cap) read on the device, so the launch needs no host sync
__global__ void k_hist(const uint4 *__restrict__ raw, const unsigned long long *__restrict__ d_R,
                       uint64_t cap, uint32_t *__restrict__ cnt) {
    const uint64_t R = *d_R < cap ? *d_R : cap;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < R;
         e += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + raw[e].x, 1u);
}

// raw results grouped by query: each goes to start[q] + its arrival order, as (k << 32) | l
__global__ void k_scatter(const uint4 *__restrict__ raw, const unsigned long long *__restrict__ d_R,
                          uint64_t cap, const uint64_t *__restrict__ start,
                          uint32_t *__restrict__ cursor, uint64_t *__restrict__ grouped) {
    const uint64_t R = *d_R < cap ? *d_R : cap;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < R;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 v = raw[e];
        const uint32_t at = atomicAdd(cursor + v.x, 1u);
        grouped[start[v.x] + at] = ((uint64_t)v.y << 32) | v.z;
    }
}

// warp per query: segments of up to 32 sorted in registers (bitonic over shuffles) and
// deduplicated with a ballot; larger segments are listed for the CTA kernel
__global__ void k_sort_small(uint32_t nq, const uint32_t *__restrict__ cnt,
                             const uint64_t *__restrict__ start, uint64_t *__restrict__ grouped,
                             uint32_t *__restrict__ ucnt, uint32_t *__restrict__ large,
                             uint32_t *__restrict__ nlarge) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nq; q += warps) {
        const uint32_t n = cnt[q];
        if (n > 32) {
            if (lane == 0) large[atomicAdd(nlarge, 1u)] = q;
            continue;
        }
        uint64_t *seg = grouped + start[q];
        uint64_t key = (uint32_t)lane < n ? seg[lane] : ~0ull;
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const uint64_t o = __shfl_xor_sync(FULL, key, j);
                const bool up = (lane & k) == 0;
                const bool low = (lane & j) == 0;
                key = (low == up) ? (key < o ? key : o) : (key > o ? key : o);
            }
        }
        const uint64_t prev = __shfl_up_sync(FULL, key, 1);
        const bool keep = (uint32_t)lane < n && (lane == 0 || key != prev);
        const uint32_t bal = __ballot_sync(FULL, keep);
        if (keep) seg[__popc(bal & ((1u << lane) - 1u))] = key;
        if (lane == 0) ucnt[q] = __popc(bal);
    }
}

// bitonic sort of P keys (a power of two, P <= 8192) in shared memory, by the whole CTA
__device__ __forceinline__ void cta_bitonic(uint64_t *sk, uint32_t P) {
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t t = threadIdx.x; t < P; t += blockDim.x) {
                const uint32_t o = t ^ j;
                if (o > t) {
                    const bool up = (t & k) == 0;
                    const uint64_t a = sk[t], b = sk[o];
                    if ((a > b) == up) {
                        sk[t] = b;
                        sk[o] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// CTA per large segment: bitonic sort in shared memory up to 8192 keys; above that, tiles of
// 8192 sorted in shared memory, then pairwise merges of sorted runs between the segment and
// tmp (each key's place: its index in its run plus its rank in the other run, by binary
// search; keys of the left run go before equal keys of the right run).
__global__ void k_sort_large(const uint32_t *__restrict__ large, const uint32_t *__restrict__ nlarge,
                             const uint32_t *__restrict__ cnt, const uint64_t *__restrict__ start,
                             uint64_t *__restrict__ grouped, uint64_t *__restrict__ tmp,
                             uint32_t *__restrict__ ucnt) {
    extern __shared__ uint64_t sk[];
    __shared__ uint32_t s_wsum[32];
    const uint32_t L = *nlarge;
    for (uint32_t li = blockIdx.x; li < L; li += gridDim.x) {
        const uint32_t q = large[li];
        const uint32_t n = cnt[q];
        uint64_t *seg = grouped + start[q];
        if (n <= 8192) {
            uint32_t P = 64;
            while (P < n) P <<= 1;
            for (uint32_t t = threadIdx.x; t < P; t += blockDim.x) sk[t] = t < n ? seg[t] : ~0ull;
            __syncthreads();
            cta_bitonic(sk, P);
            for (uint32_t t = threadIdx.x; t < n; t += blockDim.x) seg[t] = sk[t];
            __syncthreads();
        } else {
            for (uint32_t base = 0; base < n; base += 8192) {
                const uint32_t m = n - base < 8192 ? n - base : 8192;
                for (uint32_t t = threadIdx.x; t < 8192; t += blockDim.x)
                    sk[t] = t < m ? seg[base + t] : ~0ull;
                __syncthreads();
                cta_bitonic(sk, 8192);
                for (uint32_t t = threadIdx.x; t < m; t += blockDim.x) seg[base + t] = sk[t];
                __syncthreads();
            }
            uint64_t *src = seg, *dst = tmp + start[q];
            for (uint32_t w = 8192; w < n; w <<= 1) {
                for (uint32_t a0 = 0; a0 < n; a0 += 2 * w) {
                    const uint32_t a1 = n - a0 > w ? a0 + w : n;
                    const uint32_t b1 = n - a1 > w ? a1 + w : n;
                    for (uint32_t x = a0 + threadIdx.x; x < b1; x += blockDim.x) {
                        const uint64_t v = src[x];
                        // rank of v in the other run: lower bound in the right run for a left
                        // key, upper bound in the left run for a right key
                        const bool left = x < a1;
                        uint32_t lo = left ? a1 : a0, hi = left ? b1 : a1;
                        while (lo < hi) {
                            const uint32_t mid = (lo + hi) >> 1;
                            const uint64_t u = src[mid];
                            if (left ? (u < v) : (u <= v)) lo = mid + 1; else hi = mid;
                        }
                        dst[left ? x + (lo - a1) : a0 + (x - a1) + (lo - a0)] = v;
                    }
                }
                __syncthreads();
                uint64_t *t = src;
                src = dst;
                dst = t;
            }
            if (src != seg)
                for (uint32_t t = threadIdx.x; t < n; t += blockDim.x) seg[t] = src[t];
            __syncthreads();
        }
        // deduplicate the sorted segment in place, in tiles of blockDim keys
        uint32_t written = 0;
        for (uint32_t base = 0; base < n; base += blockDim.x) {
            const uint32_t t = base + threadIdx.x;
            bool keep = false;
            uint64_t x = 0;
            if (t < n) {
                x = seg[t];
                keep = (t == 0) || seg[t - 1] != x;
            }
            __syncthreads();   // all reads of this tile precede the writes below
            const uint32_t bal = __ballot_sync(FULL, keep);
            const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
            if (ln == 0) s_wsum[w] = __popc(bal);
            __syncthreads();
            uint32_t before = 0, tile = 0;
            for (int v = 0; v < (int)(blockDim.x >> 5); ++v) {
                if (v < w) before += s_wsum[v];
                tile += s_wsum[v];
            }
            if (keep) seg[written + before + __popc(bal & ((1u << ln) - 1u))] = x;
            written += tile;
            __syncthreads();
        }
        if (threadIdx.x == 0) ucnt[q] = written;
        __syncthreads();
    }
}

// writes nothing unless the total (offsets[nq]) fits the caller's capacity
__global__ void k_compact(uint32_t nq, const uint32_t *__restrict__ ucnt,
                          const uint64_t *__restrict__ start, const uint64_t *__restrict__ offsets,
                          const uint64_t *__restrict__ grouped, uint32_t *__restrict__ pairs,
                          uint64_t capacity) {
    if (offsets[nq] > capacity) return;
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nq; q += warps) {
        const uint32_t u = ucnt[q];
        const uint64_t *seg = grouped + start[q];
        uint32_t *dst = pairs + 2 * offsets[q];
        for (uint32_t t = lane; t < u; t += 32) {
            const uint64_t x = seg[t];
            dst[2 * t] = (uint32_t)(x >> 32);
            dst[2 * t + 1] = (uint32_t)x;
        }
    }
}

// Fewest differences per reported interval: each raw result finds its interval in its query's
// sorted distinct list (binary search) and lowers that interval's cost (cost32 starts at ~0).
__global__ void k_mincost(const uint4 *__restrict__ raw, const unsigned long long *__restrict__ d_R,
                          uint64_t cap, const uint64_t *__restrict__ start,
                          const uint32_t *__restrict__ ucnt, const uint64_t *__restrict__ grouped,
                          const uint64_t *__restrict__ uoff, uint32_t *__restrict__ cost32) {
    const uint64_t R = *d_R < cap ? *d_R : cap;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < R;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 v = raw[e];
        const uint64_t key = ((uint64_t)v.y << 32) | v.z;
        const uint64_t *seg = grouped + start[v.x];
        uint32_t lo = 0, hi = ucnt[v.x];
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (seg[mid] < key) lo = mid + 1; else hi = mid;
        }
        if (lo < ucnt[v.x] && seg[lo] == key) atomicMin(cost32 + uoff[v.x] + lo, v.w);
    }
}

// costs of all distinct intervals, in output order (nothing unless they fit the capacity)
__global__ void k_cost_out(const uint64_t *__restrict__ total, const uint32_t *__restrict__ cost32,
                           uint8_t *__restrict__ costs, uint64_t capacity) {
    const uint64_t n = *total;
    if (n > capacity) return;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n;
         t += (uint64_t)gridDim.x * blockDim.x)
        costs[t] = (uint8_t)cost32[t];
}

// best hits, warp per query: the query's minimum cost and how many of its intervals have it
__global__ void k_best_count(uint32_t nq, const uint32_t *__restrict__ ucnt,
                             const uint64_t *__restrict__ uoff, const uint32_t *__restrict__ cost32,
                             uint32_t *__restrict__ bcnt, uint32_t *__restrict__ qmin) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nq; q += warps) {
        const uint32_t u = ucnt[q];
        const uint32_t *cs = cost32 + uoff[q];
        uint32_t mn = 0xffffffffu;
        for (uint32_t t = lane; t < u; t += 32) mn = min(mn, cs[t]);
        mn = __reduce_min_sync(FULL, mn);
        uint32_t k = 0;
        for (uint32_t t = lane; t < u; t += 32) k += cs[t] == mn ? 1u : 0u;
        k = __reduce_add_sync(FULL, k);
        if (lane == 0) {
            bcnt[q] = k;
            qmin[q] = mn;
        }
    }
}

// best hits, warp per query: its minimum-cost intervals (and costs) at boff[q], in order
__global__ void k_best_compact(uint32_t nq, const uint32_t *__restrict__ ucnt,
                               const uint64_t *__restrict__ start, const uint64_t *__restrict__ uoff,
                               const uint64_t *__restrict__ grouped, const uint32_t *__restrict__ cost32,
                               const uint32_t *__restrict__ qmin, const uint64_t *__restrict__ boff,
                               uint32_t *__restrict__ pairs, uint8_t *__restrict__ costs,
                               uint64_t capacity) {
    if (boff[nq] > capacity) return;
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nq; q += warps) {
        const uint32_t u = ucnt[q], mn = qmin[q];
        const uint64_t *seg = grouped + start[q];
        const uint32_t *cs = cost32 + uoff[q];
        uint64_t at = boff[q];
        for (uint32_t base = 0; base < u; base += 32) {
            const uint32_t t = base + lane;
            const bool keep = t < u && cs[t] == mn;
            const uint32_t bal = __ballot_sync(FULL, keep);
            if (keep) {
                const uint64_t o = at + __popc(bal & ((1u << lane) - 1u));
                const uint64_t x = seg[t];
                pairs[2 * o] = (uint32_t)(x >> 32);
                pairs[2 * o + 1] = (uint32_t)x;
                if (costs) costs[o] = (uint8_t)mn;
            }
            at += __popc(bal);
        }
    }
}

// adds this call's counters to the caller's, unless the pass overflowed (it is then rerun)
__global__ void k_add_stats(const unsigned long long *__restrict__ in,
                            const unsigned long long *__restrict__ raw,
                            unsigned long long *__restrict__ out, uint64_t raw_cap,
                            const uint32_t *__restrict__ err) {
    if (*raw > raw_cap || (*err & (kErrSpill | kErrStack))) return;
    if (threadIdx.x == 0) {
        out[0] += in[0];
        out[1] += in[1];
        out[2] += *raw;
        out[3] += in[3];
    }
}

// the scalars the host reads after a captured search: raw count, search and D error words,
// large segments and the interval total
__global__ void k_status(const unsigned long long *__restrict__ raw, const uint32_t *__restrict__ err,
                         const uint32_t *__restrict__ nlarge, const uint64_t *__restrict__ total,
                         unsigned long long *__restrict__ out) {
    if (threadIdx.x == 0) {
        out[0] = *raw;
        out[1] = err[kErrSearch];
        out[2] = err[kErrDcalc];
        out[3] = *nlarge;
        out[4] = *total;
    }
}

// the per-query distinct counts into the caller's counts
__global__ void k_copy_counts(uint32_t nq, const uint32_t *__restrict__ ucnt,
                              uint32_t *__restrict__ counts) {
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x)
        counts[q] = ucnt[q];
}

// exclusive scan uint32 -> uint64 of n values, out has n+1 entries (out[n] = total).
// Three passes: tile sums, scan of the tile sums in one CTA, tile-local scans.
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t *ws, uint64_t &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        uint64_t y = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t t = __shfl_up_sync(FULL, y, o);
            if (lane >= o) y += t;
        }
        ws[lane] = y;
    }
    __syncthreads();
    const uint64_t before = w > 0 ? ws[w - 1] : 0;
    total = ws[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

// pass 1: the sum of each tile of kScanTile values
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const uint32_t *__restrict__ in, uint64_t n,
                                                             uint64_t *__restrict__ tile_sum) {
    __shared__ uint64_t ws[32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    uint64_t s = 0;
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        const uint64_t i = base + (uint64_t)threadIdx.x * kScanItems + t;
        if (i < n) s += in[i];
    }
    uint64_t total;
    block_excl_scan(s, ws, total);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

// pass 2 (one CTA): exclusive scan of the tile sums in place; tile_sum[ntiles] = total
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(uint64_t *__restrict__ tile_sum, uint64_t ntiles) {
    __shared__ uint64_t ws[32];
    uint64_t carry = 0;
    for (uint64_t b = 0; b < ntiles; b += blockDim.x) {
        const uint64_t i = b + threadIdx.x;
        const uint64_t v = i < ntiles ? tile_sum[i] : 0;
        uint64_t total;
        const uint64_t ex = block_excl_scan(v, ws, total);
        if (i < ntiles) tile_sum[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) tile_sum[ntiles] = carry;
}

// pass 3: each tile's exclusive scan from its offset; the last tile writes out[n] = total
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t *__restrict__ in, uint64_t n,
                                                             const uint64_t *__restrict__ tile_off,
                                                             uint64_t *__restrict__ out) {
    __shared__ uint64_t ws[32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    uint32_t v[kScanItems];
    uint64_t s = 0;
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        const uint64_t i = base + (uint64_t)threadIdx.x * kScanItems + t;
        v[t] = i < n ? in[i] : 0u;
        s += v[t];
    }
    uint64_t total;
    uint64_t run = tile_off[blockIdx.x] + block_excl_scan(s, ws, total);
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        const uint64_t i = base + (uint64_t)threadIdx.x * kScanItems + t;
        if (i < n) out[i] = run;
        run += v[t];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        const uint64_t ntiles = gridDim.x;
        out[n] = tile_off[ntiles];
    }
}

int grid_cap(fm_index *h, uint64_t work, int block) {
    uint64_t g = (work + block - 1) / block;
    uint64_t cap = (uint64_t)h->sms * (2048 / block) * 2;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

// exclusive scan of n uint32 into out[0..n] (out[n] = total); tile_sum needs
// ceil(n / kScanTile) + 1 entries
static int scan_u32(fm_index *h, const uint32_t *in, uint64_t n, uint64_t *out, uint64_t *tile_sum,
                    cudaStream_t st) {
    const uint64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles == 0) {
        FM_CUDA_TRY(h, cudaMemsetAsync(out, 0, 8, st));
        return FM_OK;
    }
    k_scan_tiles<<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, n, tile_sum);
    k_scan_sums<<<1, kScanThreads, 0, st>>>(tile_sum, ntiles);
    k_scan_apply<<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, n, tile_sum, out);
    FM_CUDA_TRY(h, cudaGetLastError());
    return FM_OK;
}

uint64_t scratch_total(const fm_index *h) {
    return h->s_qmeta.bytes + h->s_raw.bytes + h->s_spill.bytes + h->s_group.bytes +
           h->s_scan.bytes + h->s_plain.bytes + h->s_misc.bytes;
}

int ensure_scratch(fm_index *h, Scratch &s, size_t bytes) {
    if (s.bytes >= bytes && s.ptr) return FM_OK;
    if (h->scratch_budget) {
        const size_t want = bytes < 256 ? 256 : bytes;
        const uint64_t total = scratch_total(h) - s.bytes + want;
        if (total > h->scratch_budget)
            return set_error(h, FM_ENOMEM, "search scratch of " + std::to_string(total) +
                                               " bytes would exceed its budget of " +
                                               std::to_string(h->scratch_budget));
    }
    if (s.ptr) {
        cudaFree(s.ptr);
        s.ptr = nullptr;
        s.bytes = 0;
    }
    size_t want = bytes < 256 ? 256 : bytes;
    cudaError_t e = cudaMalloc(&s.ptr, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(h, FM_ENOMEM, "device allocation of " + std::to_string(want) +
                                           " bytes of search scratch failed");
    }
    s.bytes = want;
    return FM_OK;
}

// shared memory of one persistent CTA: per warp, stk pool entries plus its query slots and
// step-fill counters (without staging, the counters only when they are collected: the
// carveout, and so the L1 left beside it, follows the shared memory of the launch)
static size_t persistent_smem(int block, int stk, bool stage, bool fill = false) {
    return (size_t)(block / 32) * (size_t)warp_smem_words(stk, stage, fill) * 4;
}

// node pool entries per warp.  Smaller pools would leave more of the SM's memory to L1, but a
// G step then expands fewer nodes at once (measured slower at every size below 320)
static int pool_entries(const Tuning &) { return kPoolEntries; }

// the tuning knobs of the persistent scheduler, into a search configuration
static void set_sched(SearchCfg &c, const Tuning &tu) {
    c.chunk = tu.chunk;
    // roots of one chunk (at most 32) always fit: the pools take queries below pool - 32
    c.refill = tu.refill + 32u <= (uint32_t)kPoolEntries ? tu.refill : (uint32_t)kPoolEntries - 32u;
    c.chain2_min = tu.chain2_min;
    c.fill = nullptr;
}

// step-fill counters of the persistent kernel: 8 x uint64 in s_misc at this offset (after the
// counters at 0-31, the search stats at 32-63 and the status words of a graph at 64-103)
constexpr size_t kMiscFill = 128;
static_assert(kMiscFill + 64 <= 256, "s_misc holds 256 bytes");

static void copy_fill(fm_profile *prof, const unsigned long long *v) {
    prof->exact_steps = v[0];
    prof->exact_lanes = v[1];
    prof->exact_lanes2 = v[2];
    prof->general_steps = v[3];
    prof->general_lanes = v[4];
    prof->admissions = v[5];
    prof->admitted = v[6];
    prof->parked = v[7];
}

template <int I>
static int launch_search(fm_index *h, const SearchCfg &c, uint32_t kernel, uint4 *spill,
                         uint32_t spill_cap, int grid, int block, int stk, uint4 *stacks,
                         uint32_t cap, uint32_t T, cudaStream_t st) {
    if (kernel == FM_KERNEL_PLAIN) {
        const int pb = (int)h->tune.plain_block;
        k_inexact_plain<I><<<(T + pb - 1) / pb, pb, 0, st>>>(c, stacks, cap, T);
    } else {
        const bool fill = c.fill != nullptr;
        const size_t sm = persistent_smem(block, stk, h->tune.stage != 0, fill);
        if (h->tune.stage) {
            if (fill) k_inexact_persistent<I, true, true><<<grid, block, sm, st>>>(c, stk, spill, spill_cap);
            else k_inexact_persistent<I, true, false><<<grid, block, sm, st>>>(c, stk, spill, spill_cap);
        } else {
            if (fill) k_inexact_persistent<I, false, true><<<grid, block, sm, st>>>(c, stk, spill, spill_cap);
            else k_inexact_persistent<I, false, false><<<grid, block, sm, st>>>(c, stk, spill, spill_cap);
        }
    }
    FM_CUDA_TRY(h, cudaGetLastError());
    return FM_OK;
}

template <int I>
static cudaError_t set_smem_attr(size_t smem, bool stage, bool fill) {
    const int v = (int)smem;
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (stage) return fill ? cudaFuncSetAttribute(k_inexact_persistent<I, true, true>, a, v)
                           : cudaFuncSetAttribute(k_inexact_persistent<I, true, false>, a, v);
    return fill ? cudaFuncSetAttribute(k_inexact_persistent<I, false, true>, a, v)
                : cudaFuncSetAttribute(k_inexact_persistent<I, false, false>, a, v);
}

template <int I>
static int occupancy_blocks(int block, size_t smem, bool stage, bool fill) {
    int nb = 0;
    if (stage) {
        if (fill) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_inexact_persistent<I, true, true>, block, smem);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_inexact_persistent<I, true, false>, block, smem);
    } else {
        if (fill) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_inexact_persistent<I, false, true>, block, smem);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_inexact_persistent<I, false, false>, block, smem);
    }
    return nb;
}

static cudaError_t set_smem_attr_any(uint32_t I, size_t smem, bool stage, bool fill) {
    return I == 32 ? set_smem_attr<32>(smem, stage, fill)
                   : (I == 64 ? set_smem_attr<64>(smem, stage, fill)
                              : (I == 128 ? set_smem_attr<128>(smem, stage, fill)
                                          : set_smem_attr<256>(smem, stage, fill)));
}

static int occupancy_any(uint32_t I, int block, size_t smem, bool stage, bool fill) {
    return I == 32 ? occupancy_blocks<32>(block, smem, stage, fill)
                   : (I == 64 ? occupancy_blocks<64>(block, smem, stage, fill)
                              : (I == 128 ? occupancy_blocks<128>(block, smem, stage, fill)
                                          : occupancy_blocks<256>(block, smem, stage, fill)));
}

// fills the profile from the phase events: ev[0] start, ev[1] before the (last) search pass,
// ev[2] after it, ev[3] end of the canonical sets
static int finish_profile(fm_index *h, fm_profile *prof, cudaEvent_t *ev, uint32_t launches,
                          cudaStream_t st, const unsigned long long *fill = nullptr) {
    if (!prof) return FM_OK;
    FM_CUDA_TRY(h, cudaEventRecord(ev[3], st));
    FM_CUDA_TRY(h, cudaEventSynchronize(ev[3]));
    if (fill) {
        unsigned long long fv[8];
        FM_CUDA_TRY(h, cudaMemcpyAsync(fv, fill, sizeof(fv), cudaMemcpyDeviceToHost, st));
        FM_CUDA_TRY(h, cudaStreamSynchronize(st));
        copy_fill(prof, fv);
        prof->fill_counters = 1;
    }
    float a = 0, b = 0, c = 0, d = 0;
    FM_CUDA_TRY(h, cudaEventElapsedTime(&a, ev[0], ev[4] ? ev[4] : ev[1]));
    FM_CUDA_TRY(h, cudaEventElapsedTime(&b, ev[1], ev[2]));
    FM_CUDA_TRY(h, cudaEventElapsedTime(&c, ev[2], ev[3]));
    FM_CUDA_TRY(h, cudaEventElapsedTime(&d, ev[0], ev[3]));
    prof->ms_dcalc = a;
    prof->ms_search = b;
    prof->ms_canon = c;
    prof->ms_total = d;
    prof->launches = launches;
    return FM_OK;
}

int fetch_inexact(fm_index *h, uint32_t *pairs, uint64_t pair_capacity, cudaStream_t st) {
    if (!h->last_valid) return set_error(h, FM_EINVAL, "no search results to fetch");
    if (h->last_total > pair_capacity)
        return set_error(h, FM_ETRUNC, "pair capacity below the intervals found");
    if (h->last_total == 0) return FM_OK;
    if (!pairs) return set_error(h, FM_EINVAL, "pairs is NULL");
    char *gb = (char *)h->s_group.ptr;
    const uint32_t nq = h->last_nq;
    k_compact<<<grid_cap(h, (uint64_t)nq * 32, 256), 256, 0, st>>>(
        nq, (const uint32_t *)(gb + h->last_off_ucnt), (const uint64_t *)(gb + h->last_off_start),
        (const uint64_t *)(gb + h->last_off_uoff), (const uint64_t *)(gb + h->last_off_grp), pairs,
        pair_capacity);
    FM_CUDA_TRY(h, cudaGetLastError());
    FM_CUDA_TRY(h, cudaStreamSynchronize(st));
    return FM_OK;
}

// Group scratch layout for up to R raw results.
struct GroupLayout {
    size_t cnt, cur, ucnt, large, start, uoff, tiles, grp, tmp, total;
    GroupLayout(uint32_t nq, uint64_t R) {
        const uint64_t ntiles = (nq + kScanTile - 1) / kScanTile + 2;
        cnt = 0;
        cur = cnt + (size_t)nq * 4;
        ucnt = cur + (size_t)nq * 4;
        large = ucnt + (size_t)nq * 4;
        start = (large + (size_t)nq * 4 + 15) / 16 * 16;
        uoff = start + ((size_t)nq + 1) * 8;
        tiles = uoff + ((size_t)nq + 1) * 8;
        grp = tiles + ntiles * 8;
        tmp = grp + (R ? R : 1) * 8;
        total = tmp + (R ? R : 1) * 8;
    }
};

// The persistent search of one call as a CUDA graph: D pass, search, grouping, sorting,
// deduplication and compaction, with every size the host used to read in between taken on the
// device (raw count, large segments, pair total), so the whole call is one graph launch and one
// status read.  The graph is captured on a private stream the first time a key is seen (same
// buffers, sizes and parameters) and replayed on the caller's stream afterwards.  It needs
// scratch already sized by an earlier eager call; when the replayed pass overflows the raw
// buffer or a spill region, *fallback is set and the eager path regrows and reruns.
static int run_inexact_graph(fm_index *h, const uint8_t *reads, const uint32_t *offs,
                             uint32_t n_reads, const fm_search_params *sp, uint32_t *counts,
                             uint64_t *offsets, uint32_t *pairs, uint64_t pair_capacity,
                             uint64_t *pairs_needed, cudaStream_t st, bool *fallback,
                             const uint8_t *modes) {
    *fallback = true;
    const uint32_t nq = n_reads * sp->strands;
    const uint32_t I = h->interval;
    const Tuning &tu = h->tune;
    const int block = (int)tu.warps_per_block * 32;
    const int stk = pool_entries(tu);
    fm_profile *prof = sp->profile;
    const bool want_fill = prof && prof->fill_counters;
    // the kernel's shared-memory attribute is the launch's own size: the driver sizes the
    // carveout (and so the L1 left beside it) from it
    const size_t smem = persistent_smem(block, stk, tu.stage != 0, want_fill);
    int bps = (int)tu.blocks_per_sm;
    const int occ = occupancy_any(I, block, smem, tu.stage != 0, want_fill);
    if (bps <= 0 || bps > occ) bps = occ;
    if (bps <= 0) return FM_OK;
    const int grid = h->sms * bps;
    const uint64_t nwarps = (uint64_t)grid * (block / 32);
    if (!h->s_raw.ptr || !h->s_spill.ptr || !h->s_misc.ptr) return FM_OK;   // not sized yet
    const uint64_t raw_cap = h->s_raw.bytes / sizeof(uint4);
    const uint32_t spill_cap = (uint32_t)(h->s_spill.bytes / sizeof(uint4) / nwarps);
    if (raw_cap < (uint64_t)nq * 4 || spill_cap < 4096) return FM_OK;
    int rc;
    const uint32_t qstride = tu.stage ? kStageU4 : 1u;
    if ((rc = ensure_scratch(h, h->s_qmeta, (size_t)nq * qstride * sizeof(uint4)))) return rc;
    const GroupLayout L(nq, raw_cap);
    if ((rc = ensure_scratch(h, h->s_group, L.total))) return rc;
    if (!h->cap_stream) FM_CUDA_TRY(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    if (prof && !h->gev[0])
        for (auto &e : h->gev) FM_CUDA_TRY(h, cudaEventCreate(&e));

    GraphKey key{};
    key.reads = reads; key.offs = offs; key.counts = counts; key.offsets = offsets;
    key.pairs = pairs; key.stats = sp->stats; key.qmeta = h->s_qmeta.ptr; key.raw = h->s_raw.ptr;
    key.spill = h->s_spill.ptr; key.group = h->s_group.ptr; key.misc = h->s_misc.ptr;
    key.pair_capacity = pair_capacity; key.raw_cap = raw_cap; key.n_reads = n_reads;
    key.strands = sp->strands; key.z = sp->z; key.max_gaps = sp->max_gaps; key.interval = I;
    key.grid = (uint32_t)grid; key.block = (uint32_t)block; key.chunk = tu.chunk;
    key.spill_cap = spill_cap; key.profile = prof ? (want_fill ? 2u : 1u) : 0u;
    key.canon = search_canon(tu, sp);
    key.end_skip = sp->indel_end_skip; key.refill = tu.refill; key.chain2 = tu.chain2_min;
    key.pool = (uint32_t)stk | (tu.stage << 16);
    key.kt = h->d_kt; key.kdepth = h->kt_depth | (view_fwd(h).pairs << 16); key.modes = modes;

    char *misc = (char *)h->s_misc.ptr;
    unsigned long long *d_raw_count = (unsigned long long *)misc;
    uint32_t *d_next_q = (uint32_t *)(misc + 8);
    uint32_t *d_nlarge = (uint32_t *)(misc + 12);
    unsigned long long *d_stats = (unsigned long long *)(misc + 32);
    unsigned long long *d_status = (unsigned long long *)(misc + 64);
    char *gb = (char *)h->s_group.ptr;
    uint32_t *cnt = (uint32_t *)(gb + L.cnt), *cursor = (uint32_t *)(gb + L.cur),
             *ucnt = (uint32_t *)(gb + L.ucnt), *large = (uint32_t *)(gb + L.large);
    uint64_t *start = (uint64_t *)(gb + L.start), *uoff = (uint64_t *)(gb + L.uoff),
             *tiles = (uint64_t *)(gb + L.tiles), *grouped = (uint64_t *)(gb + L.grp),
             *tmp = (uint64_t *)(gb + L.tmp);

    if (!(h->gexec && h->gkey == key)) {
        if (h->gexec) {
            cudaGraphExecDestroy(h->gexec);
            h->gexec = nullptr;
        }
        cudaError_t e = set_smem_attr_any(I, smem, tu.stage != 0, want_fill);
        if (e != cudaSuccess) return cuda_status(h, e, "cudaFuncSetAttribute");
        FM_CUDA_TRY(h, cudaFuncSetAttribute(k_sort_large, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)(8192 * sizeof(uint64_t))));
        cudaStream_t cs = h->cap_stream;
        FM_CUDA_TRY(h, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        uint32_t launches = 0;
        int crc = FM_OK;
        do {
            if (prof && cudaEventRecordWithFlags(h->gev[0], cs, cudaEventRecordExternal)) { crc = FM_ECUDA; break; }
            if (cudaMemsetAsync(h->d_err + kErrDcalc, 0, 8, cs)) { crc = FM_ECUDA; break; }
            if ((crc = launch_dcalc(h, reads, offs, n_reads, sp->strands, (uint4 *)h->s_qmeta.ptr, nullptr, cs, qstride,
                                    modes, sp->z | (sp->max_gaps << 4)))) break;
            ++launches;
            if (prof && cudaEventRecordWithFlags(h->gev[1], cs, cudaEventRecordExternal)) { crc = FM_ECUDA; break; }
            if (cudaMemsetAsync(misc, 0, kMiscFill + 64, cs)) { crc = FM_ECUDA; break; }
            SearchCfg c;
            c.ix = view_fwd(h);
            c.reads = reads;
            c.qmeta = (const uint4 *)h->s_qmeta.ptr;
            c.nq = nq;
            c.z = sp->z;
            c.max_gaps = sp->max_gaps;
            set_sched(c, tu);
            if (want_fill) c.fill = (unsigned long long *)(misc + kMiscFill);
            c.next_q = d_next_q;
            c.raw = (uint4 *)h->s_raw.ptr;
            c.raw_count = d_raw_count;
            c.raw_cap = raw_cap;
            c.stats = d_stats;
            c.err = h->d_err + kErrSearch;
            c.canon = search_canon(tu, sp);
            c.end_skip = sp->indel_end_skip;
            switch (I) {
                case 32: crc = launch_search<32>(h, c, FM_KERNEL_PERSISTENT, (uint4 *)h->s_spill.ptr, spill_cap, grid, block, stk, nullptr, 0, 0, cs); break;
                case 64: crc = launch_search<64>(h, c, FM_KERNEL_PERSISTENT, (uint4 *)h->s_spill.ptr, spill_cap, grid, block, stk, nullptr, 0, 0, cs); break;
                case 128: crc = launch_search<128>(h, c, FM_KERNEL_PERSISTENT, (uint4 *)h->s_spill.ptr, spill_cap, grid, block, stk, nullptr, 0, 0, cs); break;
                default: crc = launch_search<256>(h, c, FM_KERNEL_PERSISTENT, (uint4 *)h->s_spill.ptr, spill_cap, grid, block, stk, nullptr, 0, 0, cs); break;
            }
            if (crc) break;
            ++launches;
            if (prof && cudaEventRecordWithFlags(h->gev[2], cs, cudaEventRecordExternal)) { crc = FM_ECUDA; break; }
            if (cudaMemsetAsync(cnt, 0, (size_t)nq * 8, cs)) { crc = FM_ECUDA; break; }
            const uint4 *raw = (const uint4 *)h->s_raw.ptr;
            k_hist<<<grid_cap(h, raw_cap, 256), 256, 0, cs>>>(raw, d_raw_count, raw_cap, cnt);
            if ((crc = scan_u32(h, cnt, nq, start, tiles, cs))) break;
            k_scatter<<<grid_cap(h, raw_cap, 256), 256, 0, cs>>>(raw, d_raw_count, raw_cap, start, cursor, grouped);
            k_sort_small<<<grid_cap(h, (uint64_t)nq * 32, 256), 256, 0, cs>>>(nq, cnt, start, grouped, ucnt, large, d_nlarge);
            k_sort_large<<<(unsigned)h->sms * 4, 512, 8192 * sizeof(uint64_t), cs>>>(large, d_nlarge, cnt, start, grouped, tmp, ucnt);
            launches += 2 + 3 + 2;
            if ((crc = scan_u32(h, ucnt, nq, uoff, tiles, cs))) break;
            if (cudaMemcpyAsync(offsets, uoff, ((size_t)nq + 1) * 8, cudaMemcpyDeviceToDevice, cs)) { crc = FM_ECUDA; break; }
            k_copy_counts<<<grid_cap(h, nq, 256), 256, 0, cs>>>(nq, ucnt, counts);
            k_compact<<<grid_cap(h, (uint64_t)nq * 32, 256), 256, 0, cs>>>(nq, ucnt, start, uoff, grouped, pairs, pair_capacity);
            launches += 3 + 2;
            if (sp->stats) {
                k_add_stats<<<1, 32, 0, cs>>>(d_stats, d_raw_count, (unsigned long long *)sp->stats, raw_cap, h->d_err);
                ++launches;
            }
            k_status<<<1, 32, 0, cs>>>(d_raw_count, h->d_err, d_nlarge, uoff + nq, d_status);
            ++launches;
            if (prof && cudaEventRecordWithFlags(h->gev[3], cs, cudaEventRecordExternal)) { crc = FM_ECUDA; break; }
            if (cudaGetLastError() != cudaSuccess) crc = FM_ECUDA;
        } while (0);
        cudaGraph_t graph = nullptr;
        cudaError_t ee = cudaStreamEndCapture(cs, &graph);
        if (crc || ee != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return FM_OK;   // capture failed: the eager path runs the call
        }
        ee = cudaGraphInstantiate(&h->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ee != cudaSuccess) {
            h->gexec = nullptr;
            cudaGetLastError();
            return FM_OK;
        }
        h->gkey = key;
        h->glaunches = launches;
        h->graph_captures += 1;
    }
    {   // an eager call since the capture may have set another size: restore the graph's
        cudaError_t e = set_smem_attr_any(I, smem, tu.stage != 0, want_fill);
        if (e != cudaSuccess) return cuda_status(h, e, "cudaFuncSetAttribute");
    }
    FM_CUDA_TRY(h, cudaGraphLaunch(h->gexec, st));
    h->graph_replays += 1;
    unsigned long long status[5] = {0, 0, 0, 0, 0};
    FM_CUDA_TRY(h, cudaMemcpyAsync(status, d_status, sizeof(status), cudaMemcpyDeviceToHost, st));
    FM_CUDA_TRY(h, cudaStreamSynchronize(st));
    const uint64_t rawn = status[0], need = status[4];
    const uint32_t errs = (uint32_t)status[1], errd = (uint32_t)status[2];
    if (rawn > raw_cap || (errs & (kErrSpill | kErrStack))) return FM_OK;   // regrow eagerly
    *fallback = false;
    h->last_valid = false;
    if (errd & kErrReadLen) return set_error(h, FM_EINVAL, "a read is longer than 255 symbols");
    if (errd & kErrDomain) return set_error(h, FM_EINVAL, "a read holds a code above 3");
    h->last_nq = nq;
    h->last_total = need;
    h->last_off_ucnt = L.ucnt;
    h->last_off_start = L.start;
    h->last_off_uoff = L.uoff;
    h->last_off_grp = L.grp;
    h->last_valid = true;
    if (pairs_needed) *pairs_needed = need;
    if (prof) {
        unsigned long long fv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (want_fill) {
            FM_CUDA_TRY(h, cudaMemcpyAsync(fv, misc + kMiscFill, sizeof(fv), cudaMemcpyDeviceToHost, st));
            FM_CUDA_TRY(h, cudaStreamSynchronize(st));
        }
        memset(prof, 0, sizeof(*prof));
        copy_fill(prof, fv);
        prof->fill_counters = want_fill ? 1u : 0u;
        float a = 0, b = 0, cc = 0, d = 0;
        FM_CUDA_TRY(h, cudaEventElapsedTime(&a, h->gev[0], h->gev[1]));
        FM_CUDA_TRY(h, cudaEventElapsedTime(&b, h->gev[1], h->gev[2]));
        FM_CUDA_TRY(h, cudaEventElapsedTime(&cc, h->gev[2], h->gev[3]));
        FM_CUDA_TRY(h, cudaEventElapsedTime(&d, h->gev[0], h->gev[3]));
        prof->ms_dcalc = a;
        prof->ms_search = b;
        prof->ms_canon = cc;
        prof->ms_total = d;
        prof->launches = h->glaunches;
        prof->passes = 1;
        prof->graph = 1;
    }
    if (need > pair_capacity)
        return set_error(h, FM_ETRUNC, "pair capacity " + std::to_string(pair_capacity) +
                                           " below the " + std::to_string(need) + " intervals found");
    return FM_OK;
}

int reserve_search_scratch(fm_index *h, uint64_t nq) {
    // the sizes run_inexact starts from for nq queries of the persistent kernel
    const Tuning &tu = h->tune;
    const int block = (int)tu.warps_per_block * 32;
    const size_t smem = persistent_smem(block, kPoolEntries, tu.stage != 0);
    int bps = (int)tu.blocks_per_sm;
    const int occ = occupancy_any(h->interval, block, smem, tu.stage != 0, false);
    if (bps <= 0 || bps > occ) bps = occ;
    const uint64_t nwarps = (uint64_t)h->sms * (bps > 0 ? bps : 1) * (block / 32);
    const uint64_t raw_cap = nq * 4 + (1u << 20);
    int rc;
    if ((rc = ensure_scratch(h, h->s_misc, 256))) return rc;
    if ((rc = ensure_scratch(h, h->s_qmeta, (size_t)nq * (tu.stage ? kStageU4 : 1u) * sizeof(uint4)))) return rc;
    if ((rc = ensure_scratch(h, h->s_raw, raw_cap * sizeof(uint4)))) return rc;
    if ((rc = ensure_scratch(h, h->s_spill, nwarps * 4096 * sizeof(uint4)))) return rc;
    return ensure_scratch(h, h->s_group, GroupLayout((uint32_t)nq, raw_cap).total);
}

int run_inexact(fm_index *h, const uint8_t *reads, const uint32_t *offs, uint32_t n_reads,
                const fm_search_params *sp, uint32_t *counts, uint64_t *offsets, uint32_t *pairs,
                uint64_t pair_capacity, uint64_t *pairs_needed, cudaStream_t st,
                const uint8_t *modes) {
    if (int krc = ensure_kmer(h, st)) return krc;
    if (int prc = ensure_pairs(h, st)) return prc;
    const bool want_cost = sp->costs != nullptr || sp->best;   // eager path only
    if (h->use_graphs && sp->kernel != FM_KERNEL_PLAIN && n_reads > 0 && !want_cost) {
        bool fallback = true;
        const int grc = run_inexact_graph(h, reads, offs, n_reads, sp, counts, offsets, pairs,
                                          pair_capacity, pairs_needed, st, &fallback, modes);
        if (!fallback) return grc;
        if (grc) return grc;
    }
    h->last_valid = false;   // only this call's results may be fetched after it
    FM_CUDA_TRY(h, cudaMemsetAsync(h->d_err + kErrDcalc, 0, 8, st));   // D pass and search words
    const uint32_t strands = sp->strands;
    const uint64_t nq64 = (uint64_t)n_reads * strands;
    if (nq64 > 0xffffffffull) return set_error(h, FM_EINVAL, "too many queries");
    const uint32_t nq = (uint32_t)nq64;
    int rc;

    // scratch layout in s_misc: counters
    //   [0] raw_count (u64) [1] next_q (u32) [2] nlarge (u32) [3..] spare
    if ((rc = ensure_scratch(h, h->s_misc, 256))) return rc;
    unsigned long long *d_raw_count = (unsigned long long *)h->s_misc.ptr;
    uint32_t *d_next_q = (uint32_t *)((char *)h->s_misc.ptr + 8);
    uint32_t *d_nlarge = (uint32_t *)((char *)h->s_misc.ptr + 12);
    unsigned long long *d_stats = (unsigned long long *)((char *)h->s_misc.ptr + 32);

    if (nq == 0) {
        if (pairs_needed) *pairs_needed = 0;
        FM_CUDA_TRY(h, cudaMemsetAsync(offsets, 0, 8, st));
        FM_CUDA_TRY(h, cudaStreamSynchronize(st));
        return FM_OK;
    }

    // phase events on the call's stream (profile requested)
    fm_profile *prof = sp->profile;
    const bool want_fill = prof && prof->fill_counters && sp->kernel != FM_KERNEL_PLAIN;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() {
            for (int i = 0; i < 5; ++i)
                if (e[i]) cudaEventDestroy(e[i]);
        }
    } evg{ev};
    if (prof) {
        memset(prof, 0, sizeof(*prof));   // the fill_counters request was read above
        for (int i = 0; i < 5; ++i) FM_CUDA_TRY(h, cudaEventCreate(&ev[i]));
        FM_CUDA_TRY(h, cudaEventRecord(ev[0], st));
    }
    uint32_t launches = 0;

    // D lower bound and per-query metadata (the persistent kernel's staging records)
    const uint32_t qstride = (sp->kernel != FM_KERNEL_PLAIN && h->tune.stage) ? kStageU4 : 1u;
    if ((rc = ensure_scratch(h, h->s_qmeta, (size_t)nq * qstride * sizeof(uint4)))) return rc;
    uint4 *qmeta = (uint4 *)h->s_qmeta.ptr;
    if ((rc = launch_dcalc(h, reads, offs, n_reads, strands, qmeta, nullptr, st, qstride, modes,
                           sp->z | (sp->max_gaps << 4))))
        return rc;
    ++launches;
    if (prof) FM_CUDA_TRY(h, cudaEventRecord(ev[4], st));   // end of the D pass

    const uint32_t I = h->interval;
    const Tuning &tu = h->tune;
    const int block = (int)tu.warps_per_block * 32;
    const int stk = pool_entries(tu);   // pool entries per warp (see the kernel)
    // the attribute is the launch's own size (see the graph path)
    const size_t smem = persistent_smem(block, stk, tu.stage != 0, want_fill);
    cudaError_t e = set_smem_attr_any(I, smem, tu.stage != 0, want_fill);
    if (e != cudaSuccess) return cuda_status(h, e, "cudaFuncSetAttribute");
    int bps = (int)tu.blocks_per_sm;
    const int occ = occupancy_any(I, block, smem, tu.stage != 0, want_fill);
    if (bps <= 0 || bps > occ) bps = occ;
    if (bps <= 0) return set_error(h, FM_ECUDA, "persistent kernel does not fit on an SM");
    int grid = h->sms * bps;
    const uint64_t nwarps = (uint64_t)grid * (block / 32);

    // plain-kernel stacks: depth-first eager pushes keep at most 8 siblings per level over at
    // most (read length + z) levels
    const uint32_t cap = 8u * ((uint32_t)kMaxReadLen + sp->z) + 16u;
    uint32_t T = 0;
    if (sp->kernel == FM_KERNEL_PLAIN) {
        uint64_t tmax = (uint64_t)h->sms * 1024;
        T = (uint32_t)(nq < tmax ? nq : tmax);
        T = (T + 31) / 32 * 32;
        if ((rc = ensure_scratch(h, h->s_plain, (size_t)T * cap * sizeof(uint4)))) return rc;
    }

    // raw result buffer and spill region, grown on overflow (the search is then rerun)
    uint64_t raw_cap = h->s_raw.bytes / sizeof(uint4);
    if (raw_cap < (uint64_t)nq * 4 + (1u << 20)) raw_cap = (uint64_t)nq * 4 + (1u << 20);
    uint32_t spill_cap = (uint32_t)(h->s_spill.bytes / sizeof(uint4) / (nwarps ? nwarps : 1));
    if (spill_cap < 4096) spill_cap = 4096;

    for (int attempt = 0; attempt < 8; ++attempt) {
        if ((rc = ensure_scratch(h, h->s_raw, raw_cap * sizeof(uint4)))) return rc;
        if (sp->kernel != FM_KERNEL_PLAIN)
            if ((rc = ensure_scratch(h, h->s_spill, nwarps * spill_cap * sizeof(uint4)))) return rc;
        FM_CUDA_TRY(h, cudaMemsetAsync(h->s_misc.ptr, 0, kMiscFill + 64, st));
        FM_CUDA_TRY(h, cudaMemsetAsync(h->d_err + kErrSearch, 0, 4, st));
        SearchCfg c;
        c.ix = view_fwd(h);
        c.reads = reads;
        c.qmeta = qmeta;
        c.nq = nq;
        c.z = sp->z;
        c.max_gaps = sp->max_gaps;
        set_sched(c, tu);
        if (want_fill) c.fill = (unsigned long long *)((char *)h->s_misc.ptr + kMiscFill);
        c.next_q = d_next_q;
        c.raw = (uint4 *)h->s_raw.ptr;
        c.raw_count = d_raw_count;
        c.raw_cap = raw_cap;
        c.stats = d_stats;
        c.err = h->d_err + kErrSearch;
        c.canon = search_canon(tu, sp);
        c.end_skip = sp->indel_end_skip;
        if (prof) FM_CUDA_TRY(h, cudaEventRecord(ev[1], st));
        switch (I) {
            case 32: rc = launch_search<32>(h, c, sp->kernel, (uint4 *)h->s_spill.ptr, spill_cap, grid, block, stk, (uint4 *)h->s_plain.ptr, cap, T, st); break;
            case 64: rc = launch_search<64>(h, c, sp->kernel, (uint4 *)h->s_spill.ptr, spill_cap, grid, block, stk, (uint4 *)h->s_plain.ptr, cap, T, st); break;
            case 128: rc = launch_search<128>(h, c, sp->kernel, (uint4 *)h->s_spill.ptr, spill_cap, grid, block, stk, (uint4 *)h->s_plain.ptr, cap, T, st); break;
            default: rc = launch_search<256>(h, c, sp->kernel, (uint4 *)h->s_spill.ptr, spill_cap, grid, block, stk, (uint4 *)h->s_plain.ptr, cap, T, st); break;
        }
        if (rc) return rc;
        ++launches;
        if (prof) {
            FM_CUDA_TRY(h, cudaEventRecord(ev[2], st));
            prof->passes += 1;
        }
        unsigned long long rawn = 0;
        uint32_t errw = 0, derr = 0;
        FM_CUDA_TRY(h, cudaMemcpyAsync(&rawn, d_raw_count, 8, cudaMemcpyDeviceToHost, st));
        FM_CUDA_TRY(h, cudaMemcpyAsync(&errw, h->d_err + kErrSearch, 4, cudaMemcpyDeviceToHost, st));
        FM_CUDA_TRY(h, cudaMemcpyAsync(&derr, h->d_err + kErrDcalc, 4, cudaMemcpyDeviceToHost, st));
        FM_CUDA_TRY(h, cudaStreamSynchronize(st));
        // a bad read is reported before anything else (a truncation status would send the
        // caller to fm_inexact_fetch for the results of a failed call)
        if (derr & kErrReadLen) return set_error(h, FM_EINVAL, "a read is longer than 255 symbols");
        if (derr & kErrDomain) return set_error(h, FM_EINVAL, "a read holds a code above 3");
        if (errw & kErrStack) return set_error(h, FM_ENOMEM, "plain search stack overflow");
        bool again = false;
        if (errw & kErrSpill) {
            spill_cap *= 4;
            again = true;
        }
        if (rawn > raw_cap) {
            raw_cap = rawn + rawn / 4 + 1024;
            again = true;
        }
        if (!again) {
            // canonical sets
            const uint64_t R = rawn;
            // group scratch: cnt, cursor, ucnt, large (4 x nq u32), start and uoff (nq+1 u64
            // each), tile sums, grouped and tmp (R u64 each)
            const uint64_t ntiles = (nq + kScanTile - 1) / kScanTile + 2;
            const size_t off_cnt = 0, off_cur = off_cnt + (size_t)nq * 4,
                         off_ucnt = off_cur + (size_t)nq * 4, off_large = off_ucnt + (size_t)nq * 4,
                         off_start = (off_large + (size_t)nq * 4 + 15) / 16 * 16,
                         off_uoff = off_start + ((size_t)nq + 1) * 8,
                         off_tiles = off_uoff + ((size_t)nq + 1) * 8, off_grp = off_tiles + ntiles * 8,
                         off_tmp = off_grp + (R ? R : 1) * 8, off_cost = off_tmp + (R ? R : 1) * 8,
                         off_bcnt = off_cost + (R ? R : 1) * 4, off_qmin = off_bcnt + (size_t)nq * 4,
                         off_boff = (off_qmin + (size_t)nq * 4 + 15) / 16 * 16,
                         total = want_cost ? off_boff + ((size_t)nq + 1) * 8 : off_cost;
            h->last_valid = false;
            if ((rc = ensure_scratch(h, h->s_group, total))) return rc;
            char *gb = (char *)h->s_group.ptr;
            uint32_t *cnt = (uint32_t *)(gb + off_cnt), *cursor = (uint32_t *)(gb + off_cur),
                     *ucnt = (uint32_t *)(gb + off_ucnt), *large = (uint32_t *)(gb + off_large);
            uint64_t *start = (uint64_t *)(gb + off_start), *uoff = (uint64_t *)(gb + off_uoff),
                     *tiles = (uint64_t *)(gb + off_tiles), *grouped = (uint64_t *)(gb + off_grp),
                     *tmp = (uint64_t *)(gb + off_tmp);
            FM_CUDA_TRY(h, cudaMemsetAsync(cnt, 0, (size_t)nq * 8, st));   // cnt and cursor
            const uint4 *raw = (const uint4 *)h->s_raw.ptr;
            if (R) k_hist<<<grid_cap(h, R, 256), 256, 0, st>>>(raw, d_raw_count, raw_cap, cnt);
            if ((rc = scan_u32(h, cnt, nq, start, tiles, st))) return rc;
            if (R) k_scatter<<<grid_cap(h, R, 256), 256, 0, st>>>(raw, d_raw_count, raw_cap, start, cursor, grouped);
            k_sort_small<<<grid_cap(h, (uint64_t)nq * 32, 256), 256, 0, st>>>(nq, cnt, start, grouped, ucnt, large, d_nlarge);
            FM_CUDA_TRY(h, cudaGetLastError());
            launches += (R ? 2u : 0u) + 3u + 1u;
            uint32_t nlarge = 0;
            FM_CUDA_TRY(h, cudaMemcpyAsync(&nlarge, d_nlarge, 4, cudaMemcpyDeviceToHost, st));
            FM_CUDA_TRY(h, cudaStreamSynchronize(st));
            if (nlarge) {
                const size_t lsm = 8192 * sizeof(uint64_t);
                FM_CUDA_TRY(h, cudaFuncSetAttribute(k_sort_large, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm));
                unsigned lg = nlarge < (uint32_t)h->sms * 4 ? nlarge : (uint32_t)h->sms * 4;
                k_sort_large<<<lg, 512, lsm, st>>>(large, d_nlarge, cnt, start, grouped, tmp, ucnt);
                FM_CUDA_TRY(h, cudaGetLastError());
                ++launches;
            }
            if ((rc = scan_u32(h, ucnt, nq, uoff, tiles, st))) return rc;
            launches += 3u;
            // fewest differences per interval, and the best hits
            uint32_t *cost32 = (uint32_t *)(gb + off_cost), *bcnt = (uint32_t *)(gb + off_bcnt),
                     *qmin = (uint32_t *)(gb + off_qmin);
            uint64_t *boff = (uint64_t *)(gb + off_boff);
            if (want_cost) {
                FM_CUDA_TRY(h, cudaMemsetAsync(cost32, 0xff, (R ? R : 1) * 4, st));
                if (R) {
                    k_mincost<<<grid_cap(h, R, 256), 256, 0, st>>>(raw, d_raw_count, raw_cap, start, ucnt,
                                                                  grouped, uoff, cost32);
                    ++launches;
                }
                if (sp->best) {
                    k_best_count<<<grid_cap(h, (uint64_t)nq * 32, 256), 256, 0, st>>>(nq, ucnt, uoff, cost32,
                                                                                       bcnt, qmin);
                    FM_CUDA_TRY(h, cudaGetLastError());
                    if ((rc = scan_u32(h, bcnt, nq, boff, tiles, st))) return rc;
                    launches += 4u;
                }
            }
            const uint32_t *out_cnt = sp->best ? bcnt : ucnt;
            const uint64_t *out_off = sp->best ? boff : uoff;
            FM_CUDA_TRY(h, cudaMemcpyAsync(offsets, out_off, ((size_t)nq + 1) * 8, cudaMemcpyDeviceToDevice, st));
            k_copy_counts<<<grid_cap(h, nq, 256), 256, 0, st>>>(nq, out_cnt, counts);
            FM_CUDA_TRY(h, cudaGetLastError());
            launches += 1u;
            uint64_t need = 0;
            FM_CUDA_TRY(h, cudaMemcpyAsync(&need, out_off + nq, 8, cudaMemcpyDeviceToHost, st));
            FM_CUDA_TRY(h, cudaStreamSynchronize(st));
            if (pairs_needed) *pairs_needed = need;
            h->last_nq = nq;
            h->last_total = need;
            h->last_off_ucnt = off_ucnt;
            h->last_off_start = off_start;
            h->last_off_uoff = off_uoff;
            h->last_off_grp = off_grp;
            h->last_valid = !want_cost;   // fm_inexact_fetch serves plain interval sets only
            if (sp->stats) {
                k_add_stats<<<1, 32, 0, st>>>(d_stats, d_raw_count, (unsigned long long *)sp->stats,
                                              raw_cap, h->d_err);
                FM_CUDA_TRY(h, cudaGetLastError());
                ++launches;
            }
            const unsigned long long *fillp =
                want_fill ? (const unsigned long long *)((char *)h->s_misc.ptr + kMiscFill) : nullptr;
            if (need > pair_capacity) {
                if ((rc = finish_profile(h, prof, ev, launches, st, fillp))) return rc;
                return set_error(h, FM_ETRUNC, "pair capacity " + std::to_string(pair_capacity) +
                                                   " below the " + std::to_string(need) + " intervals found");
            }
            if (need) {
                if (sp->best) {
                    k_best_compact<<<grid_cap(h, (uint64_t)nq * 32, 256), 256, 0, st>>>(
                        nq, ucnt, start, uoff, grouped, cost32, qmin, boff, pairs, sp->costs,
                        pair_capacity);
                } else {
                    k_compact<<<grid_cap(h, (uint64_t)nq * 32, 256), 256, 0, st>>>(nq, ucnt, start, uoff, grouped, pairs,
                                                                                    pair_capacity);
                    if (sp->costs)
                        k_cost_out<<<grid_cap(h, need ? need : 1, 256), 256, 0, st>>>(uoff + nq, cost32, sp->costs,
                                                                                     pair_capacity);
                }
                FM_CUDA_TRY(h, cudaGetLastError());
                launches += sp->costs && !sp->best ? 2u : 1u;
            }
            if ((rc = finish_profile(h, prof, ev, launches, st, fillp))) return rc;
            return FM_OK;
        }
    }
    return set_error(h, FM_ENOMEM, "search scratch did not converge after 8 regrowths");
}

}  // namespace fm

// ============================================================================================
// Allocation-free inexact search.
//
// fm_inexact grows its scratch (query metadata, raw intervals, frontier spill, grouping
// buffers) with cudaMalloc on demand.  fm_inexact_noalloc runs the same search with all of
// that scratch carved out of one fixed, file-scope device array, so a call allocates nothing.
// The array is 64 MiB; every device that loads this library holds it until the process exits.
// It runs the depth-first kernel (k_inexact_plain), whose per-thread stack has a proven bound
// (at most 8 siblings wait per level over at most read length + z levels), on a fixed number
// of threads, so the search itself cannot run out of space.  Limits that follow from the
// array's size: at most kNoAllocMaxQueries queries (reads x strands) per call and at most
// kNoAllocMaxRaw intervals before deduplication; a call beyond them returns an error instead
// of growing anything.  All calls share the one array: calls that overlap on the GPU (from any
// thread, stream or index handle) race on it and must not be issued.
// ============================================================================================
#include <mutex>

namespace fm {
namespace {

constexpr uint32_t kNoAllocMaxQueries = 32768;
constexpr uint64_t kNoAllocMaxRaw = 8ull * kNoAllocMaxQueries;
constexpr uint32_t kNoAllocThreads = 1536;                           // multiple of 32
constexpr uint32_t kNoAllocStackCap = 8u * ((uint32_t)kMaxReadLen + (uint32_t)kMaxZ) + 16u;

constexpr size_t na_align(size_t x) { return (x + 255) / 256 * 256; }
// byte offsets inside the array
constexpr size_t kNaMisc = 0;                                            // counters, 256 B
constexpr size_t kNaQmeta = kNaMisc + 256;                               // uint4 per query
constexpr size_t kNaRaw = na_align(kNaQmeta + (size_t)kNoAllocMaxQueries * 16);
constexpr size_t kNaStacks = na_align(kNaRaw + kNoAllocMaxRaw * 16);
constexpr size_t kNaCnt = na_align(kNaStacks + (size_t)kNoAllocThreads * kNoAllocStackCap * 16);
constexpr size_t kNaCursor = kNaCnt + (size_t)kNoAllocMaxQueries * 4;    // contiguous with cnt
constexpr size_t kNaUcnt = na_align(kNaCursor + (size_t)kNoAllocMaxQueries * 4);
constexpr size_t kNaLarge = na_align(kNaUcnt + (size_t)kNoAllocMaxQueries * 4);
constexpr size_t kNaStart = na_align(kNaLarge + (size_t)kNoAllocMaxQueries * 4);
constexpr size_t kNaUoff = na_align(kNaStart + ((size_t)kNoAllocMaxQueries + 1) * 8);
constexpr size_t kNaTiles = na_align(kNaUoff + ((size_t)kNoAllocMaxQueries + 1) * 8);
constexpr size_t kNaGrouped = na_align(kNaTiles + ((size_t)kNoAllocMaxQueries / kScanTile + 4) * 8);
constexpr size_t kNaTmp = na_align(kNaGrouped + kNoAllocMaxRaw * 8);
constexpr size_t kNaEnd = na_align(kNaTmp + kNoAllocMaxRaw * 8);
constexpr size_t kNoAllocBytes = (size_t)64 << 20;
static_assert(kNaEnd <= kNoAllocBytes, "no-alloc scratch layout exceeds its array");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device.  In host code the array's name is only a
// host-side stand-in, so its device address is taken once per device, with that device
// current, by cudaGetSymbolAddress.
std::mutex g_na_mu;
constexpr int kNaMaxDevices = 64;
unsigned char *g_na_base[kNaMaxDevices] = {};

int noalloc_base(fm_index *h, unsigned char **out) {
    if (h->device < 0 || h->device >= kNaMaxDevices)
        return set_error(h, FM_EINVAL, "device ordinal out of range for the static scratch");
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_base[h->device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(h, e, "cudaGetSymbolAddress(static scratch)");
        g_na_base[h->device] = (unsigned char *)p;
    }
    *out = g_na_base[h->device];
    return FM_OK;
}

template <int I>
int noalloc_launch(fm_index *h, const SearchCfg &c, uint4 *stacks, cudaStream_t st) {
    const int pb = 128;
    k_inexact_plain<I><<<(kNoAllocThreads + pb - 1) / pb, pb, 0, st>>>(c, stacks, kNoAllocStackCap,
                                                                        kNoAllocThreads);
    FM_CUDA_TRY(h, cudaGetLastError());
    return FM_OK;
}

int run_inexact_noalloc(fm_index *h, const uint8_t *reads, const uint32_t *offs,
                        uint32_t n_reads, const fm_search_params *sp, uint32_t *counts,
                        uint64_t *offsets, uint32_t *pairs, uint64_t pair_capacity,
                        uint64_t *pairs_needed, cudaStream_t st) {
    // its results live in the static array, not in the handle's scratch: fm_inexact_fetch
    // must not serve an earlier fm_inexact call's intervals in their place
    h->last_valid = false;
    if (sp->costs || sp->best)
        return set_error(h, FM_EINVAL, "fm_inexact_noalloc reports interval sets only (no costs, no best)");
    const uint64_t nq64 = (uint64_t)n_reads * sp->strands;
    if (nq64 > kNoAllocMaxQueries)
        return set_error(h, FM_EINVAL, "fm_inexact_noalloc: " + std::to_string(nq64) +
                                           " queries exceed the static scratch limit of " +
                                           std::to_string(kNoAllocMaxQueries));
    const uint32_t nq = (uint32_t)nq64;
    int rc;
    unsigned char *base = nullptr;
    if ((rc = noalloc_base(h, &base))) return rc;
    unsigned long long *d_raw_count = (unsigned long long *)(base + kNaMisc);
    uint32_t *d_next_q = (uint32_t *)(base + kNaMisc + 8);
    uint32_t *d_nlarge = (uint32_t *)(base + kNaMisc + 12);
    unsigned long long *d_stats = (unsigned long long *)(base + kNaMisc + 32);
    uint4 *qmeta = (uint4 *)(base + kNaQmeta);
    uint4 *raw = (uint4 *)(base + kNaRaw);
    uint4 *stacks = (uint4 *)(base + kNaStacks);
    uint32_t *cnt = (uint32_t *)(base + kNaCnt), *cursor = (uint32_t *)(base + kNaCursor);
    uint32_t *ucnt = (uint32_t *)(base + kNaUcnt), *large = (uint32_t *)(base + kNaLarge);
    uint64_t *start = (uint64_t *)(base + kNaStart), *uoff = (uint64_t *)(base + kNaUoff);
    uint64_t *tiles = (uint64_t *)(base + kNaTiles), *grouped = (uint64_t *)(base + kNaGrouped);
    uint64_t *tmp = (uint64_t *)(base + kNaTmp);

    // the array keeps the previous call's contents: counters start from zero
    FM_CUDA_TRY(h, cudaMemsetAsync(base + kNaMisc, 0, 64, st));
    if (nq == 0) {
        FM_CUDA_TRY(h, cudaMemsetAsync(offsets, 0, 8, st));
        FM_CUDA_TRY(h, cudaStreamSynchronize(st));
        if (pairs_needed) *pairs_needed = 0;
        return FM_OK;
    }
    FM_CUDA_TRY(h, cudaMemsetAsync(h->d_err + kErrSearch, 0, 4, st));
    if ((rc = launch_dcalc(h, reads, offs, n_reads, sp->strands, qmeta, nullptr, st, 1, nullptr,
                           sp->z | (sp->max_gaps << 4))))
        return rc;

    SearchCfg c;
    c.ix = view_fwd(h);
    c.reads = reads;
    c.qmeta = qmeta;
    c.nq = nq;
    c.z = sp->z;
    c.max_gaps = sp->max_gaps;
    set_sched(c, h->tune);
    c.next_q = d_next_q;
    c.raw = raw;
    c.raw_count = d_raw_count;
    c.raw_cap = kNoAllocMaxRaw;
    c.stats = d_stats;
    c.err = h->d_err + kErrSearch;
    c.canon = search_canon(h->tune, sp);
    c.end_skip = sp->indel_end_skip;
    switch (h->interval) {
        case 32: rc = noalloc_launch<32>(h, c, stacks, st); break;
        case 64: rc = noalloc_launch<64>(h, c, stacks, st); break;
        case 128: rc = noalloc_launch<128>(h, c, stacks, st); break;
        default: rc = noalloc_launch<256>(h, c, stacks, st); break;
    }
    if (rc) return rc;
    unsigned long long rawn = 0;
    uint32_t errw = 0, derr = 0;
    FM_CUDA_TRY(h, cudaMemcpyAsync(&rawn, d_raw_count, 8, cudaMemcpyDeviceToHost, st));
    FM_CUDA_TRY(h, cudaMemcpyAsync(&errw, h->d_err + kErrSearch, 4, cudaMemcpyDeviceToHost, st));
    FM_CUDA_TRY(h, cudaMemcpyAsync(&derr, h->d_err + kErrDcalc, 4, cudaMemcpyDeviceToHost, st));
    FM_CUDA_TRY(h, cudaStreamSynchronize(st));
    if (derr & kErrReadLen) return set_error(h, FM_EINVAL, "a read is longer than 255 symbols");
    if (derr & kErrDomain) return set_error(h, FM_EINVAL, "a read holds a code above 3");
    if (errw & kErrStack)   // cannot happen: the stack capacity is the proven bound
        return set_error(h, FM_ENOMEM, "fm_inexact_noalloc: depth-first stack overflow");
    if (rawn > kNoAllocMaxRaw)
        return set_error(h, FM_ENOMEM, "fm_inexact_noalloc: " + std::to_string(rawn) +
                                           " intervals before deduplication exceed the static "
                                           "limit of " + std::to_string(kNoAllocMaxRaw));
    const uint64_t R = rawn;
    FM_CUDA_TRY(h, cudaMemsetAsync(cnt, 0, (size_t)nq * 4, st));
    FM_CUDA_TRY(h, cudaMemsetAsync(cursor, 0, (size_t)nq * 4, st));
    if (R) k_hist<<<grid_cap(h, R, 256), 256, 0, st>>>(raw, d_raw_count, kNoAllocMaxRaw, cnt);
    if ((rc = scan_u32(h, cnt, nq, start, tiles, st))) return rc;
    if (R) k_scatter<<<grid_cap(h, R, 256), 256, 0, st>>>(raw, d_raw_count, kNoAllocMaxRaw, start, cursor, grouped);
    k_sort_small<<<grid_cap(h, (uint64_t)nq * 32, 256), 256, 0, st>>>(nq, cnt, start, grouped,
                                                                       ucnt, large, d_nlarge);
    FM_CUDA_TRY(h, cudaGetLastError());
    uint32_t nlarge = 0;
    FM_CUDA_TRY(h, cudaMemcpyAsync(&nlarge, d_nlarge, 4, cudaMemcpyDeviceToHost, st));
    FM_CUDA_TRY(h, cudaStreamSynchronize(st));
    if (nlarge) {
        const size_t lsm = 8192 * sizeof(uint64_t);
        FM_CUDA_TRY(h, cudaFuncSetAttribute(k_sort_large,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm));
        unsigned lg = nlarge < (uint32_t)h->sms * 4 ? nlarge : (uint32_t)h->sms * 4;
        k_sort_large<<<lg, 512, lsm, st>>>(large, d_nlarge, cnt, start, grouped, tmp, ucnt);
        FM_CUDA_TRY(h, cudaGetLastError());
    }
    if ((rc = scan_u32(h, ucnt, nq, uoff, tiles, st))) return rc;
    FM_CUDA_TRY(h, cudaMemcpyAsync(offsets, uoff, ((size_t)nq + 1) * 8, cudaMemcpyDeviceToDevice, st));
    k_copy_counts<<<grid_cap(h, nq, 256), 256, 0, st>>>(nq, ucnt, counts);
    FM_CUDA_TRY(h, cudaGetLastError());
    uint64_t need = 0;
    FM_CUDA_TRY(h, cudaMemcpyAsync(&need, uoff + nq, 8, cudaMemcpyDeviceToHost, st));
    FM_CUDA_TRY(h, cudaStreamSynchronize(st));
    if (pairs_needed) *pairs_needed = need;
    if (sp->stats) {
        k_add_stats<<<1, 32, 0, st>>>(d_stats, d_raw_count, (unsigned long long *)sp->stats,
                                      kNoAllocMaxRaw, h->d_err);
        FM_CUDA_TRY(h, cudaGetLastError());
    }
    if (need > pair_capacity) {
        FM_CUDA_TRY(h, cudaStreamSynchronize(st));
        return set_error(h, FM_ETRUNC, "pair capacity " + std::to_string(pair_capacity) +
                                           " below the " + std::to_string(need) + " intervals found");
    }
    if (need) {
        k_compact<<<grid_cap(h, (uint64_t)nq * 32, 256), 256, 0, st>>>(nq, ucnt, start, uoff,
                                                                        grouped, pairs, pair_capacity);
        FM_CUDA_TRY(h, cudaGetLastError());
    }
    FM_CUDA_TRY(h, cudaStreamSynchronize(st));
    return FM_OK;
}

}  // namespace
}  // namespace fm

extern "C" int fm_inexact_noalloc(fm_index *h, const uint8_t *reads, const uint32_t *offs,
                                  uint32_t n_reads, const fm_search_params *sp, uint32_t *counts,
                                  uint64_t *offsets, uint32_t *pairs, uint64_t pair_capacity,
                                  uint64_t *pairs_needed, void *stream) {
    using namespace fm;
    if (!h) return set_global_error(FM_EINVAL, "null index handle");
    if (!sp) return set_error(h, FM_EINVAL, "search params are NULL");
    if (!h->has_rev) return set_error(h, FM_EINVAL, "index built without reverse(R)");
    if (sp->z > (uint32_t)kMaxZ) return set_error(h, FM_EINVAL, "z must be at most 7");
    if (sp->max_gaps > (uint32_t)kMaxGaps) return set_error(h, FM_EINVAL, "max_gaps must be at most 7");
    if (sp->strands != 1 && sp->strands != 2) return set_error(h, FM_EINVAL, "strands must be 1 or 2");
    if (sp->indel_end_skip > 255) return set_error(h, FM_EINVAL, "indel_end_skip must be at most 255");
    if (!offsets || (n_reads && (!reads || !offs || !counts))) return set_error(h, FM_EINVAL, "null buffer");
    if (pair_capacity && !pairs) return set_error(h, FM_EINVAL, "pairs is NULL");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) {
        cudaGetLastError();
        prev = -1;
    }
    if (prev != h->device && cudaSetDevice(h->device) != cudaSuccess)
        return cuda_status(h, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = FM_OK;
    cudaError_t e = cudaMemsetAsync(h->d_err + kErrDcalc, 0, 8, st);
    if (e != cudaSuccess) rc = cuda_status(h, e, "cudaMemsetAsync(error words)");
    if (!rc)
        rc = run_inexact_noalloc(h, reads, offs, n_reads, sp, counts, offsets, pairs,
                                 pair_capacity, pairs_needed, st);
    if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
    return rc;
}
