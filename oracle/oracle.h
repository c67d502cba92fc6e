/*
 * Oracle for the FM-index search path of R. Snytsar, "Vectorized Character Counting for
 * Faster Pattern Matching" (arXiv 1811.06127).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow CPU restatement of what the search path
 * computes, used to check the CUDA library.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load it; the product path never calls it.  It shares no
 * code, header, table or helper with the CUDA library.
 *
 * Conventions (all integer arithmetic, no floating point anywhere):
 *   - A text R is n symbol codes A=0, C=1, G=2, T=3 (the 2-bit code of Fig. 2); the
 *     terminator $ is implicit at position n and is smaller than every symbol (Sec. 2).
 *   - Rows of the Burrows-Wheeler matrix run 0..n (n+1 rows); row 0 is the suffix "$".
 *   - In a BWT array, code 4 stands for $.
 *   - Occ(b,k) counts b in BWT[0..k] inclusive (Sec. 2), for k in [-1, n]; Occ(b,-1) = 0;
 *     $ is counted for no b.
 *   - C[b] counts the symbols of R smaller than b ($ excluded); C[4] = n (Fig. 1).
 *
 * Function pins (tests/test_oracle_*.py) and readings of the paper are listed per function.
 */
#ifndef FM_ORACLE_H
#define FM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Eq. 1: suffix array of R$ (n+1 entries, SA[0] = n) by plain comparison sort of suffixes.
 * Quadratic in the worst case: for small texts.  Returns 0. */
int or_sa_naive(const uint8_t *R, int64_t n, int64_t *SA);

/* Eq. 1: the same suffix array by SA-IS (Nong, Zhang and Chan, "Linear suffix array
 * construction by almost pure induced-sorting", DCC 2009), the "more sophisticated"
 * construction the paper allows in Sec. 2.  Returns 0, or -1 when out of memory. */
int or_sa_sais(const uint8_t *R, int64_t n, int64_t *SA);

/* Eq. 2: BWT[i] = R[SA[i]-1] when SA[i] > 0, else $ (code 4).  L has n+1 entries.
 * Returns the row holding $. */
int64_t or_bwt(const uint8_t *R, int64_t n, const int64_t *SA, uint8_t *L);

/* C array of Sec. 2 / Fig. 1: C[b] = number of symbols of R smaller than b, C[4] = n. */
void or_count(const uint8_t *R, int64_t n, int64_t C[5]);

/* Sec. 2: Occ(b,k) by a linear scan of BWT[0..k]; k in [-1, n]. */
int64_t or_occ_scan(const uint8_t *L, int64_t n, int b, int64_t k);

/* An oracle index: the text (borrowed), SA, BWT, C and a plain count-every-64-rows table
 * used to answer Occ by one checkpoint read plus a scan of at most 63 BWT symbols. */
typedef struct or_index or_index;

/* method 0: or_sa_naive, method 1: or_sa_sais.  NULL when out of memory. */
or_index *or_index_new(const uint8_t *R, int64_t n, int method);
void or_index_free(or_index *ix);
const int64_t *or_index_sa(const or_index *ix);
const uint8_t *or_index_bwt(const or_index *ix);
void or_index_c(const or_index *ix, int64_t C[5]);
int64_t or_index_dollar_row(const or_index *ix);

/* Occ(b,k) for b = A,C,G,T at once, k in [-1, n]. */
void or_occ4(const or_index *ix, int64_t k, int64_t occ[4]);

/* Sec. 2, "eight Occ values" per inexact step: for each query q,
 * out[8q..8q+3] = Occ(A..T, k[q]-1) and out[8q+4..8q+7] = Occ(A..T, l[q]),
 * for 0 <= k <= n+1 and 0 <= l <= n.  Returns 0, or -1 when a query is outside that domain.
 * threads <= 0 means one thread per online core. */
int or_occ8_batch(const or_index *ix, const uint32_t *k, const uint32_t *l, int64_t N,
                  uint32_t *out, int threads);

/* The same eight values by one sorted sweep over the BWT: all rank positions are sorted and
 * the BWT is streamed once with running counts.  Returns 0, -1 on domain error or no memory. */
int or_occ8_sweep(const uint8_t *L, int64_t n, const uint32_t *k, const uint32_t *l, int64_t N,
                  uint32_t *out);

/* Listing 1 (ExactRecur) from the whole range [0, n], without early exit: for i = m-1..0,
 * b = W[i], k <- C(b) + Occ(b,k-1) + 1, l <- C(b) + Occ(b,l).  An absent pattern ends with
 * k = l + 1.  Reads are concatenated codes with offs[nreads+1].  Returns 0, -1 on a bad code. */
int or_exact_batch(const or_index *ix, const uint8_t *codes, const uint32_t *offs, int64_t nreads,
                   uint32_t *k_out, uint32_t *l_out, int threads);

/* Closed form of the exact interval (no index): scans all n+1 suffixes of R$ and counts
 * less = #{suffixes smaller than W that do not start with W}, pre = #{suffixes starting with
 * W}; then k = less, l = less + pre - 1, and for every b
 *   occ[b]   = #{smaller suffixes p > 0 with R[p-1] = b}        = Occ(b, k-1)
 *   occ[4+b] = #{smaller-or-prefixed suffixes p > 0, R[p-1] = b} = Occ(b, l).
 * Batch over patterns (concatenated codes with offs), parallel over patterns.
 * out8 may be NULL.  Returns 0. */
int or_interval_naive_batch(const uint8_t *R, int64_t n, const uint8_t *codes,
                            const uint32_t *offs, int64_t npat, int64_t *k_out, int64_t *l_out,
                            int64_t *out8, int threads);

/* Lower bound D used to prune the inexact recursion (BWA; Li and Durbin 2009, cited in
 * Sec. 2 for Listing 2): greedily, z = 0, j = 0; for i = 0..m-1, if W[j..i] is not a
 * substring of R then z <- z+1 and j <- i+1; D[i] = z.  The substring test narrows an SA
 * interval by binary search, one symbol at a time.  D has m entries. */
void or_dcalc(const or_index *ix, const uint8_t *W, int64_t m, uint8_t *D);

/* Listing 2 (InexRecur), results as a set.  Readings applied:
 *   - every b uses fresh k', l' computed from the node's own (k, l);
 *   - the deletion, match and mismatch recursions all run only when k' <= l';
 *   - insertions and deletions are single-base columns, at most max_gaps of them in total
 *     (max_gaps = 0: mismatches only);
 *   - with prune & 1 a call returns nothing when z < D(i) (D(-1) = 0);
 *   - with prune & 2 the search enumerates canonical alignments only (test instrumentation,
 *     not in the paper; oracle.c states the rules): same results, fewer nodes;
 *   - a call with i < 0 and z >= 0 reports {k, l} unless k = 0 (no reference symbol used);
 *   - the top call is InexRecur(W, m-1, z, 0, n);
 *   - end_skip > 0 (an option after BWA, not in the paper): an indel column only where at
 *     least end_skip symbols of W lie on each side of it, i.e. inserting W[i] needs
 *     end_skip <= i <= m-1-end_skip, and a deletion between W[i] and W[i+1] needs
 *     end_skip - 1 <= i <= m-1-end_skip.  Not combined with prune & 2 (NULL).
 * Query q = r*strands + s searches read r (s = 0) or its reverse complement (s = 1).
 * Results per query are distinct intervals sorted by (k, l).  nodes counts calls that reach
 * the Occ loop (i >= 0 after the tests); blocks counts, per such call, the checkpoint blocks
 * of width `interval` holding rank positions k and l+1 (1 when the same block, else 2). */
typedef struct or_results {
    int64_t nq;
    uint32_t *counts;   /* [nq] intervals per query */
    uint64_t *offsets;  /* [nq+1] exclusive prefix sum of counts */
    uint32_t *pairs;    /* [2*total] k, l */
    uint8_t *costs;     /* [total] per interval, the fewest differences (mismatch and indel
                           columns) among the alignments that reached it */
    uint64_t *nodes;    /* [nq] */
    uint64_t *blocks;   /* [nq] */
    uint64_t total;
} or_results;

or_results *or_inexact_batch(const or_index *ix, const uint8_t *codes, const uint32_t *offs,
                             int64_t nreads, int strands, int z, int max_gaps, int prune,
                             int interval, int threads, int end_skip);
void or_results_free(or_results *res);

/* Textbook sliding window: #{p in [0, n-m] : Hamming(W, R[p..p+m-1]) <= z}. */
int64_t or_hamming_count(const uint8_t *R, int64_t n, const uint8_t *W, int64_t m, int z);

/* Number of threads the batch calls use for threads <= 0. */
int or_default_threads(void);

#ifdef __cplusplus
}
#endif
#endif
