/*
 * Oracle for the FM-index search path of R. Snytsar, "Vectorized Character Counting for
 * Faster Pattern Matching" (arXiv 1811.06127).  TEST INFRASTRUCTURE ONLY: loaded by the
 * tests, the smoke check and the benchmark's CPU-baseline leg, never by the product path.
 * Plain C: each function states the passage it follows; see oracle.h for the conventions.
 */
#define _GNU_SOURCE
#include "oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define SYM_DOLLAR 4

int or_default_threads(void) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c < 1 ? 1 : (int)c;
}

/* ------------------------------------------------------------------------------------------
 * tiny thread pool: run fn(arg, q) for q in [0, count) with a shared counter
 * ---------------------------------------------------------------------------------------- */
typedef void (*work_fn)(void *arg, int64_t q, int tid);
typedef struct {
    work_fn fn;
    void *arg;
    int64_t count;
    int64_t next;
    int64_t grain;
    pthread_mutex_t mu;
} pool_t;
typedef struct {
    pool_t *p;
    int tid;
} worker_t;

static void *pool_worker(void *a) {
    worker_t *w = (worker_t *)a;
    pool_t *p = w->p;
    for (;;) {
        pthread_mutex_lock(&p->mu);
        int64_t s = p->next;
        p->next += p->grain;
        pthread_mutex_unlock(&p->mu);
        if (s >= p->count) break;
        int64_t e = s + p->grain < p->count ? s + p->grain : p->count;
        for (int64_t q = s; q < e; ++q) p->fn(p->arg, q, w->tid);
    }
    return NULL;
}

static void run_parallel(work_fn fn, void *arg, int64_t count, int64_t grain, int threads) {
    if (threads <= 0) threads = or_default_threads();
    if (threads > count) threads = count > 0 ? (int)count : 1;
    pool_t p;
    p.fn = fn;
    p.arg = arg;
    p.count = count;
    p.next = 0;
    p.grain = grain < 1 ? 1 : grain;
    pthread_mutex_init(&p.mu, NULL);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * threads);
    worker_t *ws = (worker_t *)malloc(sizeof(worker_t) * threads);
    for (int t = 0; t < threads; ++t) {
        ws[t].p = &p;
        ws[t].tid = t;
    }
    for (int t = 1; t < threads; ++t) pthread_create(&th[t], NULL, pool_worker, &ws[t]);
    pool_worker(&ws[0]);
    for (int t = 1; t < threads; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&p.mu);
    free(th);
    free(ws);
}

/* ------------------------------------------------------------------------------------------
 * Eq. 1: suffix array, naive comparison sort.  Suffix p of R$ compared symbol by symbol;
 * position n holds $ (the smallest symbol).
 * ---------------------------------------------------------------------------------------- */
static const uint8_t *g_naive_R;
static int64_t g_naive_n;

static int sym_at(const uint8_t *R, int64_t n, int64_t p) {
    return p < n ? (int)R[p] + 1 : 0; /* $ = 0, A..T = 1..4 */
}

static int cmp_suffix(const void *pa, const void *pb) {
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    for (int64_t d = 0;; ++d) {
        int ca = sym_at(g_naive_R, g_naive_n, a + d);
        int cb = sym_at(g_naive_R, g_naive_n, b + d);
        if (ca != cb) return ca < cb ? -1 : 1;
        if (ca == 0) return 0; /* both reached $: same suffix */
    }
}

int or_sa_naive(const uint8_t *R, int64_t n, int64_t *SA) {
    static pthread_mutex_t mu = PTHREAD_MUTEX_INITIALIZER;
    for (int64_t i = 0; i <= n; ++i) SA[i] = i;
    pthread_mutex_lock(&mu);
    g_naive_R = R;
    g_naive_n = n;
    qsort(SA, (size_t)(n + 1), sizeof(int64_t), cmp_suffix);
    pthread_mutex_unlock(&mu);
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * Eq. 1 by SA-IS.  s[0..len) over [0, K), with s[len-1] = 0 the unique smallest sentinel.
 *   1. type each suffix S (smaller than its successor) or L; the sentinel is S;
 *   2. LMS positions: S-type with an L-type predecessor;
 *   3. put LMS positions at the ends of their buckets, induce L-types left to right and
 *      S-types right to left: the LMS substrings come out sorted;
 *   4. name the LMS substrings in that order (equal substrings share a name) and form the
 *      reduced string of names in text order; sort it recursively unless all names differ;
 *   5. put the LMS suffixes at their bucket ends in their sorted order and induce again.
 * ---------------------------------------------------------------------------------------- */
static void bucket_bounds(const int64_t *s, int64_t len, int64_t K, int64_t *bkt, int ends) {
    memset(bkt, 0, sizeof(int64_t) * K);
    for (int64_t i = 0; i < len; ++i) bkt[s[i]]++;
    int64_t sum = 0;
    for (int64_t c = 0; c < K; ++c) {
        sum += bkt[c];
        bkt[c] = ends ? sum : sum - bkt[c];
    }
}

static int is_lms(const uint8_t *t, int64_t i) { return i > 0 && t[i] && !t[i - 1]; }

static void induce(const int64_t *s, int64_t len, int64_t K, const uint8_t *t, int64_t *SA,
                   int64_t *bkt) {
    bucket_bounds(s, len, K, bkt, 0); /* L-types go to bucket heads, left to right */
    for (int64_t i = 0; i < len; ++i) {
        int64_t j = SA[i] - 1;
        if (SA[i] > 0 && !t[j]) SA[bkt[s[j]]++] = j;
    }
    bucket_bounds(s, len, K, bkt, 1); /* S-types go to bucket tails, right to left */
    for (int64_t i = len - 1; i >= 0; --i) {
        int64_t j = SA[i] - 1;
        if (SA[i] > 0 && t[j]) SA[--bkt[s[j]]] = j;
    }
}

static int lms_equal(const int64_t *s, const uint8_t *t, int64_t len, int64_t a, int64_t b) {
    for (int64_t d = 0;; ++d) {
        if (a + d >= len || b + d >= len) return 0;
        if (s[a + d] != s[b + d] || t[a + d] != t[b + d]) return 0;
        if (d > 0 && (is_lms(t, a + d) || is_lms(t, b + d)))
            return is_lms(t, a + d) && is_lms(t, b + d);
    }
}

static int sais_core(const int64_t *s, int64_t len, int64_t K, int64_t *SA) {
    if (len == 1) { /* the sentinel alone */
        SA[0] = 0;
        return 0;
    }
    uint8_t *t = (uint8_t *)malloc((size_t)len);
    int64_t *bkt = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    if (!t || !bkt) {
        free(t);
        free(bkt);
        return -1;
    }
    t[len - 1] = 1;
    for (int64_t i = len - 2; i >= 0; --i)
        t[i] = (s[i] < s[i + 1] || (s[i] == s[i + 1] && t[i + 1])) ? 1 : 0;

    /* step 3: LMS substrings sorted by induction */
    for (int64_t i = 0; i < len; ++i) SA[i] = -1;
    bucket_bounds(s, len, K, bkt, 1);
    for (int64_t i = 1; i < len; ++i)
        if (is_lms(t, i)) SA[--bkt[s[i]]] = i;
    induce(s, len, K, t, SA, bkt);

    /* step 4: names */
    int64_t n1 = 0;
    for (int64_t i = 0; i < len; ++i)
        if (SA[i] >= 0 && is_lms(t, SA[i])) SA[n1++] = SA[i];
    int64_t *name_at = (int64_t *)malloc(sizeof(int64_t) * (size_t)len);
    if (!name_at) {
        free(t);
        free(bkt);
        return -1;
    }
    for (int64_t i = 0; i < len; ++i) name_at[i] = -1;
    int64_t names = 0, prev = -1;
    for (int64_t i = 0; i < n1; ++i) {
        int64_t p = SA[i];
        if (prev < 0 || !lms_equal(s, t, len, prev, p)) names++;
        prev = p;
        name_at[p] = names - 1;
    }
    int64_t *s1 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n1 > 0 ? n1 : 1));
    int64_t *pos1 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n1 > 0 ? n1 : 1));
    int64_t *SA1 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n1 > 0 ? n1 : 1));
    if (!s1 || !pos1 || !SA1) {
        free(t); free(bkt); free(name_at); free(s1); free(pos1); free(SA1);
        return -1;
    }
    int64_t j = 0;
    for (int64_t i = 0; i < len; ++i)
        if (name_at[i] >= 0) {
            s1[j] = name_at[i];
            pos1[j] = i;
            ++j;
        }
    free(name_at);
    if (names < n1) {
        if (sais_core(s1, n1, names, SA1) != 0) {
            free(t); free(bkt); free(s1); free(pos1); free(SA1);
            return -1;
        }
    } else {
        for (int64_t i = 0; i < n1; ++i) SA1[s1[i]] = i;
    }

    /* step 5: sorted LMS suffixes to their bucket ends (largest first), induce */
    for (int64_t i = 0; i < len; ++i) SA[i] = -1;
    bucket_bounds(s, len, K, bkt, 1);
    for (int64_t i = n1 - 1; i >= 0; --i) {
        int64_t p = pos1[SA1[i]];
        SA[--bkt[s[p]]] = p;
    }
    induce(s, len, K, t, SA, bkt);
    free(t); free(bkt); free(s1); free(pos1); free(SA1);
    return 0;
}

int or_sa_sais(const uint8_t *R, int64_t n, int64_t *SA) {
    int64_t *s = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!s) return -1;
    for (int64_t i = 0; i < n; ++i) s[i] = (int64_t)R[i] + 1;
    s[n] = 0;
    int rc = sais_core(s, n + 1, 5, SA);
    free(s);
    return rc;
}

/* ------------------------------------------------------------------------------------------
 * Eq. 2, C and Occ (Sec. 2)
 * ---------------------------------------------------------------------------------------- */
int64_t or_bwt(const uint8_t *R, int64_t n, const int64_t *SA, uint8_t *L) {
    int64_t dollar = -1;
    for (int64_t i = 0; i <= n; ++i) {
        if (SA[i] > 0) {
            L[i] = R[SA[i] - 1];
        } else {
            L[i] = SYM_DOLLAR;
            dollar = i;
        }
    }
    return dollar;
}

void or_count(const uint8_t *R, int64_t n, int64_t C[5]) {
    int64_t cnt[4] = {0, 0, 0, 0};
    for (int64_t i = 0; i < n; ++i) cnt[R[i]]++;
    C[0] = 0;
    for (int b = 0; b < 4; ++b) C[b + 1] = C[b] + cnt[b];
}

int64_t or_occ_scan(const uint8_t *L, int64_t n, int b, int64_t k) {
    (void)n;
    int64_t c = 0;
    for (int64_t i = 0; i <= k; ++i) c += (L[i] == b);
    return c;
}

struct or_index {
    const uint8_t *R;
    int64_t n;
    int64_t *SA;
    uint8_t *L;
    int64_t C[5];
    int64_t dollar;
    int64_t *ck; /* ck[4j+b] = count of b in L[0, 64j) */
    int64_t nck;
};

#define CK_STEP 64

or_index *or_index_new(const uint8_t *R, int64_t n, int method) {
    or_index *ix = (or_index *)calloc(1, sizeof(or_index));
    if (!ix) return NULL;
    ix->R = R;
    ix->n = n;
    ix->SA = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    ix->L = (uint8_t *)malloc((size_t)(n + 1));
    ix->nck = (n + 1) / CK_STEP + 1;
    ix->ck = (int64_t *)malloc(sizeof(int64_t) * 4 * (size_t)ix->nck);
    if (!ix->SA || !ix->L || !ix->ck) {
        or_index_free(ix);
        return NULL;
    }
    int rc = method == 0 ? or_sa_naive(R, n, ix->SA) : or_sa_sais(R, n, ix->SA);
    if (rc != 0) {
        or_index_free(ix);
        return NULL;
    }
    ix->dollar = or_bwt(R, n, ix->SA, ix->L);
    or_count(R, n, ix->C);
    int64_t run[4] = {0, 0, 0, 0};
    for (int64_t i = 0; i <= n + 1; ++i) {
        if (i % CK_STEP == 0)
            for (int b = 0; b < 4; ++b) ix->ck[4 * (i / CK_STEP) + b] = run[b];
        if (i <= n && ix->L[i] < 4) run[ix->L[i]]++;
    }
    return ix;
}

void or_index_free(or_index *ix) {
    if (!ix) return;
    free(ix->SA);
    free(ix->L);
    free(ix->ck);
    free(ix);
}

const int64_t *or_index_sa(const or_index *ix) { return ix->SA; }
const uint8_t *or_index_bwt(const or_index *ix) { return ix->L; }
void or_index_c(const or_index *ix, int64_t C[5]) { memcpy(C, ix->C, sizeof(int64_t) * 5); }
int64_t or_index_dollar_row(const or_index *ix) { return ix->dollar; }

/* counts of each symbol in L[0, p), p in [0, n+1]: checkpoint plus a scan */
static void rank4(const or_index *ix, int64_t p, int64_t out[4]) {
    int64_t j = p / CK_STEP;
    for (int b = 0; b < 4; ++b) out[b] = ix->ck[4 * j + b];
    for (int64_t i = j * CK_STEP; i < p; ++i)
        if (ix->L[i] < 4) out[ix->L[i]]++;
}

void or_occ4(const or_index *ix, int64_t k, int64_t occ[4]) { rank4(ix, k + 1, occ); }

typedef struct {
    const or_index *ix;
    const uint32_t *k, *l;
    uint32_t *out;
    int bad;
} occ8_job;

static void occ8_one(void *a, int64_t q, int tid) {
    (void)tid;
    occ8_job *J = (occ8_job *)a;
    int64_t n = J->ix->n;
    int64_t k = J->k[q], l = J->l[q];
    if (k > n + 1 || l > n) {
        J->bad = 1;
        for (int c = 0; c < 8; ++c) J->out[8 * q + c] = 0;
        return;
    }
    int64_t o1[4], o2[4];
    or_occ4(J->ix, k - 1, o1);
    or_occ4(J->ix, l, o2);
    for (int b = 0; b < 4; ++b) {
        J->out[8 * q + b] = (uint32_t)o1[b];
        J->out[8 * q + 4 + b] = (uint32_t)o2[b];
    }
}

int or_occ8_batch(const or_index *ix, const uint32_t *k, const uint32_t *l, int64_t N,
                  uint32_t *out, int threads) {
    occ8_job J = {ix, k, l, out, 0};
    run_parallel(occ8_one, &J, N, 4096, threads);
    return J.bad ? -1 : 0;
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

int or_occ8_sweep(const uint8_t *L, int64_t n, const uint32_t *k, const uint32_t *l, int64_t N,
                  uint32_t *out) {
    /* rank position p of slot s: s = 2q -> k[q] (Occ(., k-1) = rank(., k)),
     * s = 2q+1 -> l[q]+1 (Occ(., l) = rank(., l+1)); key = p << 32 | s needs s < 2^32 */
    if (2 * N >= ((int64_t)1 << 32)) return -1;
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * N > 0 ? 2 * N : 1));
    if (!key) return -1;
    for (int64_t q = 0; q < N; ++q) {
        if ((int64_t)k[q] > n + 1 || (int64_t)l[q] > n) {
            free(key);
            return -1;
        }
        key[2 * q] = ((uint64_t)k[q] << 32) | (uint64_t)(2 * q);
        key[2 * q + 1] = ((uint64_t)l[q] + 1) << 32 | (uint64_t)(2 * q + 1);
    }
    qsort(key, (size_t)(2 * N), sizeof(uint64_t), cmp_u64);
    int64_t run[4] = {0, 0, 0, 0};
    int64_t at = 0; /* run = counts in L[0, at) */
    for (int64_t i = 0; i < 2 * N; ++i) {
        int64_t p = (int64_t)(key[i] >> 32);
        uint64_t s = key[i] & 0xFFFFFFFFu;
        while (at < p) {
            if (L[at] < 4) run[L[at]]++;
            ++at;
        }
        uint64_t q = s >> 1;
        int half = (int)(s & 1);
        for (int b = 0; b < 4; ++b) out[8 * q + 4 * half + b] = (uint32_t)run[b];
    }
    free(key);
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * Listing 1 (ExactRecur), iterative, from [0, n]
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    const or_index *ix;
    const uint8_t *codes;
    const uint32_t *offs;
    uint32_t *k_out, *l_out;
    int bad;
} exact_job;

static void exact_one(void *a, int64_t r, int tid) {
    (void)tid;
    exact_job *J = (exact_job *)a;
    const or_index *ix = J->ix;
    int64_t k = 0, l = ix->n;
    int64_t s = J->offs[r], e = J->offs[r + 1];
    for (int64_t i = e - 1; i >= s; --i) {
        int b = J->codes[i];
        if (b > 3) {
            J->bad = 1;
            break;
        }
        int64_t ok[4], ol[4];
        or_occ4(ix, k - 1, ok);
        or_occ4(ix, l, ol);
        k = ix->C[b] + ok[b] + 1;
        l = ix->C[b] + ol[b];
    }
    J->k_out[r] = (uint32_t)k;
    J->l_out[r] = (uint32_t)l;
}

int or_exact_batch(const or_index *ix, const uint8_t *codes, const uint32_t *offs, int64_t nreads,
                   uint32_t *k_out, uint32_t *l_out, int threads) {
    exact_job J = {ix, codes, offs, k_out, l_out, 0};
    run_parallel(exact_one, &J, nreads, 64, threads);
    return J.bad ? -1 : 0;
}

/* ------------------------------------------------------------------------------------------
 * closed form of the exact interval by scanning every suffix
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    const uint8_t *R;
    int64_t n;
    const uint8_t *codes;
    const uint32_t *offs;
    int64_t *k_out, *l_out, *out8;
} naive_job;

static void naive_one(void *a, int64_t q, int tid) {
    (void)tid;
    naive_job *J = (naive_job *)a;
    const uint8_t *R = J->R;
    int64_t n = J->n;
    const uint8_t *W = J->codes + J->offs[q];
    int64_t m = (int64_t)J->offs[q + 1] - (int64_t)J->offs[q];
    int64_t less = 0, pre = 0;
    int64_t oc_less[5] = {0, 0, 0, 0, 0}, oc_pre[5] = {0, 0, 0, 0, 0};
    for (int64_t p = 0; p <= n; ++p) {
        /* compare R[p..n)$ with W: -1 smaller (not prefixed), 0 prefixed, 1 larger */
        int rel = 0;
        for (int64_t d = 0; d < m; ++d) {
            if (p + d >= n) { /* suffix reaches $ first: smaller */
                rel = -1;
                break;
            }
            if (R[p + d] != W[d]) {
                rel = R[p + d] < W[d] ? -1 : 1;
                break;
            }
        }
        int before = p > 0 ? R[p - 1] : 4;
        if (rel < 0) {
            less++;
            oc_less[before]++;
        } else if (rel == 0) {
            pre++;
            oc_pre[before]++;
        }
    }
    J->k_out[q] = less;
    J->l_out[q] = less + pre - 1;
    if (J->out8)
        for (int b = 0; b < 4; ++b) {
            J->out8[8 * q + b] = oc_less[b];
            J->out8[8 * q + 4 + b] = oc_less[b] + oc_pre[b];
        }
}

int or_interval_naive_batch(const uint8_t *R, int64_t n, const uint8_t *codes,
                            const uint32_t *offs, int64_t npat, int64_t *k_out, int64_t *l_out,
                            int64_t *out8, int threads) {
    naive_job J = {R, n, codes, offs, k_out, l_out, out8};
    run_parallel(naive_one, &J, npat, 1, threads);
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * D lower bound: greedy non-substring windows, substring test on the SA
 * ---------------------------------------------------------------------------------------- */
/* symbol at offset d of the suffix in row r; -1 at or beyond $ */
static int row_sym(const or_index *ix, int64_t r, int64_t d) {
    int64_t p = ix->SA[r] + d;
    return p < ix->n ? (int)ix->R[p] : -1;
}

/* rows [lo,hi) share their first d symbols; keep those whose symbol at offset d is c */
static void narrow(const or_index *ix, int64_t *lo, int64_t *hi, int64_t d, int c) {
    int64_t a = *lo, b = *hi;
    while (a < b) { /* first row with symbol >= c */
        int64_t mid = a + (b - a) / 2;
        if (row_sym(ix, mid, d) < c) a = mid + 1; else b = mid;
    }
    int64_t first = a;
    b = *hi;
    while (a < b) { /* first row with symbol > c */
        int64_t mid = a + (b - a) / 2;
        if (row_sym(ix, mid, d) <= c) a = mid + 1; else b = mid;
    }
    *lo = first;
    *hi = a;
}

void or_dcalc(const or_index *ix, const uint8_t *W, int64_t m, uint8_t *D) {
    int64_t lo = 0, hi = ix->n + 1, d = 0;
    int z = 0;
    for (int64_t i = 0; i < m; ++i) {
        narrow(ix, &lo, &hi, d, W[i]);
        if (lo >= hi) { /* W[j..i] is not a substring */
            z++;
            lo = 0;
            hi = ix->n + 1;
            d = 0;
        } else {
            d++;
        }
        D[i] = (uint8_t)(z > 255 ? 255 : z);
    }
}

/* ------------------------------------------------------------------------------------------
 * The inexact search of Sec. 2 (Listing 2) with D pruning, set semantics
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    uint32_t *pairs; /* k, l, cost (differences the alignment used) */
    int64_t size, cap;
} pairvec;

static void pv_push(pairvec *v, uint32_t k, uint32_t l, uint32_t cost) {
    if (v->size == v->cap) {
        v->cap = v->cap ? 2 * v->cap : 64;
        v->pairs = (uint32_t *)realloc(v->pairs, sizeof(uint32_t) * 3 * (size_t)v->cap);
    }
    v->pairs[3 * v->size] = k;
    v->pairs[3 * v->size + 1] = l;
    v->pairs[3 * v->size + 2] = cost;
    v->size++;
}

typedef struct {
    const or_index *ix;
    const uint8_t *W;
    const uint8_t *D;
    int max_gaps, prune, interval;
    pairvec *out;
    uint64_t nodes, blocks;
    int z0; /* the differences allowed at the top call; a result's cost is z0 - z */
    int64_t m;        /* length of W */
    int64_t end_skip; /* an indel column needs at least this many symbols of W on each side */
} inex_ctx;

/* End restriction on indel columns (an option in the manner of BWA, Li and Durbin 2009, which
 * Listing 2 cites; not in the paper).  Reading: an indel column may be placed only where at
 * least end_skip symbols of W lie on each side of it.  Inserting W[i] leaves W[0..i-1] (i
 * symbols) on its left and W[i+1..m-1] (m-1-i) on its right; a deletion taken at position i
 * sits between W[i] and W[i+1], with i+1 symbols on its left and m-1-i on its right. */
static int ins_allowed(const inex_ctx *X, int64_t i) {
    return i >= X->end_skip && X->m - 1 - i >= X->end_skip;
}

static int del_allowed(const inex_ctx *X, int64_t i) {
    return i + 1 >= X->end_skip && X->m - 1 - i >= X->end_skip;
}

/* The search of Sec. 2 (Listing 2) as a worklist of alignment states.  A state is a partial
 * alignment built from the end of W: the columns placed so far spell a reference string X,
 * whose suffix-array interval is [k, l]; W[0..i] is still to be aligned, z differences are
 * left and gaps indel columns were used.  For the canonical enumeration a state also keeps
 * the column that created it (last: 0 match or the start, 1 mismatch, 2 insertion,
 * 3 deletion) and that column's reference symbol lb.  The next column to the left is one of:
 *   - W[i] against no reference symbol (an insertion): X and [k, l] unchanged, i - 1;
 *   - a reference symbol b against no symbol of W (a deletion): X becomes bX, i unchanged;
 *   - W[i] against b: X becomes bX, i - 1, one difference unless b = W[i].
 * An indel column costs a difference and a gap; prepending b needs bX to occur in R (its
 * interval non-empty).  A state with i < 0 has aligned all of W: X's interval is a result
 * (unless X is empty), with cost z0 - z.  A state is dropped when z < 0, or when z < D(i)
 * (the bound of or_dcalc) with pruning on.  The order in which states are taken does not
 * change the result set; this one is depth first. */
typedef struct {
    int64_t i, k, l;
    int z, gaps, last, lb;
} inex_state;

typedef struct {
    inex_state *a;
    int64_t n, cap;
} state_stack;

static void st_push(state_stack *S, int64_t i, int z, int gaps, int64_t k, int64_t l, int last,
                    int lb) {
    if (S->n == S->cap) {
        S->cap = S->cap ? 2 * S->cap : 256;
        S->a = (inex_state *)realloc(S->a, sizeof(inex_state) * (size_t)S->cap);
    }
    inex_state *t = &S->a[S->n++];
    t->i = i;
    t->z = z;
    t->gaps = gaps;
    t->k = k;
    t->l = l;
    t->last = last;
    t->lb = lb;
}

/* the interval of bX for every b, from the interval [k, l] of X: one backward step
 * (Eq. 3 and Listing 1) */
static void extend4(const or_index *ix, int64_t k, int64_t l, int64_t nk[4], int64_t nl[4]) {
    int64_t ok[4], ol[4];
    or_occ4(ix, k - 1, ok);
    or_occ4(ix, l, ol);
    for (int b = 0; b < 4; ++b) {
        nk[b] = ix->C[b] + ok[b] + 1;
        nl[b] = ix->C[b] + ol[b];
    }
}

/* canonical = 0: every alignment (the enumeration of Listing 2).  canonical = 1: the
 * canonical alignments only (test instrumentation, not part of the paper's method): a state
 * does not start a non-canonical pair of adjacent columns,
 *   after an insertion (of W[i+1]): no mismatch, no deletion, no match when W[i] = W[i+1];
 *   after a deletion of lb: no insertion; when i >= 1 also no mismatch and no match of lb;
 *   after a mismatch with lb at W[i+1]: no insertion when W[i] = lb, no deletion of W[i+1].
 * Each excluded pair spells the same reference string as a canonical pair of no higher cost,
 * so the results are unchanged.  A state counts as a node (nodes, blocks) when it reaches
 * the backward step: always with i >= 0 in the first enumeration; in the canonical one only
 * when a deletion, mismatch or match may follow (a state with none only passes its insertion
 * on).  The rules move indel columns, so they are not combined with an end restriction. */
static void inex_search(inex_ctx *X, int canonical) {
    const uint8_t *W = X->W;
    state_stack S = {NULL, 0, 0};
    st_push(&S, X->m - 1, X->z0, 0, 0, X->ix->n, 0, 0);
    while (S.n > 0) {
        const inex_state s = S.a[--S.n];
        if (s.z < 0) continue;
        if (X->prune && s.i >= 0 && s.z < X->D[s.i]) continue;
        if (s.i < 0) {
            if (s.k >= 1) pv_push(X->out, (uint32_t)s.k, (uint32_t)s.l, (uint32_t)(X->z0 - s.z));
            continue;
        }
        const int64_t i = s.i;
        /* the columns that may come next */
        int ins_ok = s.gaps < X->max_gaps && ins_allowed(X, i);
        int del_ok = s.gaps < X->max_gaps && del_allowed(X, i);
        int mis_ok = 1, match_ok = 1, no_del_sym = -1;
        if (canonical) {
            del_ok = del_ok && s.z >= 1;
            mis_ok = s.z >= 1;
            if (s.last == 2) {
                del_ok = 0;
                mis_ok = 0;
                if (W[i] == W[i + 1]) match_ok = 0;
            } else if (s.last == 3) {
                ins_ok = 0;
                if (i >= 1) {
                    mis_ok = 0;
                    if (W[i] == s.lb) match_ok = 0;
                }
            } else if (s.last == 1) {
                if (W[i] == s.lb) ins_ok = 0;
                no_del_sym = W[i + 1];
            }
        }
        if (ins_ok) st_push(&S, i - 1, s.z - 1, s.gaps + 1, s.k, s.l, 2, 0);
        if (canonical && !del_ok && !mis_ok && !match_ok) continue;
        X->nodes++;
        X->blocks += (s.k / X->interval == (s.l + 1) / X->interval) ? 1 : 2;
        int64_t nk[4], nl[4];
        extend4(X->ix, s.k, s.l, nk, nl);
        for (int b = 0; b < 4; ++b) {
            if (nk[b] > nl[b]) continue; /* bX does not occur */
            if (del_ok && b != no_del_sym) st_push(&S, i, s.z - 1, s.gaps + 1, nk[b], nl[b], 3, b);
            if (b == W[i]) {
                if (match_ok) st_push(&S, i - 1, s.z, s.gaps, nk[b], nl[b], 0, b);
            } else if (mis_ok) {
                st_push(&S, i - 1, s.z - 1, s.gaps, nk[b], nl[b], 1, b);
            }
        }
    }
    free(S.a);
}

/* order of (k, l, cost) triples; same_interval compares (k, l) only */
static int cmp_triple(const void *a, const void *b) {
    const uint32_t *x = (const uint32_t *)a, *y = (const uint32_t *)b;
    for (int t = 0; t < 3; ++t)
        if (x[t] != y[t]) return x[t] < y[t] ? -1 : 1;
    return 0;
}

static int same_interval(const uint32_t *x, const uint32_t *y) {
    return x[0] == y[0] && x[1] == y[1];
}

typedef struct {
    const or_index *ix;
    const uint8_t *codes;
    const uint32_t *offs;
    int strands, z, max_gaps, prune, interval, end_skip;
    pairvec *per_query;
    uint64_t *nodes, *blocks;
} inex_job;

static void inex_one(void *a, int64_t q, int tid) {
    (void)tid;
    inex_job *J = (inex_job *)a;
    int64_t r = q / J->strands;
    int strand = (int)(q % J->strands);
    int64_t s = J->offs[r];
    int64_t m = (int64_t)J->offs[r + 1] - s;
    uint8_t *W = (uint8_t *)malloc((size_t)(m > 0 ? m : 1));
    uint8_t *D = (uint8_t *)malloc((size_t)(m > 0 ? m : 1));
    for (int64_t i = 0; i < m; ++i)
        W[i] = strand ? (uint8_t)(3 - J->codes[s + m - 1 - i]) : J->codes[s + i];
    or_dcalc(J->ix, W, m, D);
    pairvec v = {NULL, 0, 0};
    inex_ctx X = {J->ix, W, D, J->max_gaps, J->prune & 1, J->interval, &v, 0, 0, J->z, m,
                  J->end_skip};
    inex_search(&X, (J->prune & 2) ? 1 : 0);
    if (v.size > 1) { /* sort and keep distinct intervals */
        /* each interval once, with the fewest differences any of its alignments used (the
         * first of its run after sorting by cost too) */
        qsort(v.pairs, (size_t)v.size, 3 * sizeof(uint32_t), cmp_triple);
        int64_t w = 1;
        for (int64_t i = 1; i < v.size; ++i)
            if (!same_interval(&v.pairs[3 * i], &v.pairs[3 * (w - 1)])) {
                v.pairs[3 * w] = v.pairs[3 * i];
                v.pairs[3 * w + 1] = v.pairs[3 * i + 1];
                v.pairs[3 * w + 2] = v.pairs[3 * i + 2];
                ++w;
            }
        v.size = w;
    }
    J->per_query[q] = v;
    J->nodes[q] = X.nodes;
    J->blocks[q] = X.blocks;
    free(W);
    free(D);
}

or_results *or_inexact_batch(const or_index *ix, const uint8_t *codes, const uint32_t *offs,
                             int64_t nreads, int strands, int z, int max_gaps, int prune,
                             int interval, int threads, int end_skip) {
    if (strands != 1 && strands != 2) return NULL;
    if (end_skip < 0 || (end_skip > 0 && (prune & 2))) return NULL;
    if (interval <= 0) interval = 64;
    int64_t nq = nreads * strands;
    or_results *res = (or_results *)calloc(1, sizeof(or_results));
    res->nq = nq;
    res->counts = (uint32_t *)calloc((size_t)(nq > 0 ? nq : 1), sizeof(uint32_t));
    res->offsets = (uint64_t *)calloc((size_t)nq + 1, sizeof(uint64_t));
    res->nodes = (uint64_t *)calloc((size_t)(nq > 0 ? nq : 1), sizeof(uint64_t));
    res->blocks = (uint64_t *)calloc((size_t)(nq > 0 ? nq : 1), sizeof(uint64_t));
    pairvec *pq = (pairvec *)calloc((size_t)(nq > 0 ? nq : 1), sizeof(pairvec));
    inex_job J = {ix, codes, offs, strands, z, max_gaps, prune, interval, end_skip, pq,
                  res->nodes, res->blocks};
    run_parallel(inex_one, &J, nq, 16, threads);
    uint64_t total = 0;
    for (int64_t q = 0; q < nq; ++q) {
        res->offsets[q] = total;
        res->counts[q] = (uint32_t)pq[q].size;
        total += (uint64_t)pq[q].size;
    }
    res->offsets[nq] = total;
    res->total = total;
    res->pairs = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (size_t)(total > 0 ? total : 1));
    res->costs = (uint8_t *)malloc((size_t)(total > 0 ? total : 1));
    for (int64_t q = 0; q < nq; ++q) {
        for (int64_t t = 0; t < pq[q].size; ++t) {
            const uint64_t o = res->offsets[q] + (uint64_t)t;
            res->pairs[2 * o] = pq[q].pairs[3 * t];
            res->pairs[2 * o + 1] = pq[q].pairs[3 * t + 1];
            res->costs[o] = (uint8_t)pq[q].pairs[3 * t + 2];
        }
        free(pq[q].pairs);
    }
    free(pq);
    return res;
}

void or_results_free(or_results *res) {
    if (!res) return;
    free(res->counts);
    free(res->offsets);
    free(res->pairs);
    free(res->costs);
    free(res->nodes);
    free(res->blocks);
    free(res);
}

/* ------------------------------------------------------------------------------------------
 * Hamming sliding window
 * ---------------------------------------------------------------------------------------- */
int64_t or_hamming_count(const uint8_t *R, int64_t n, const uint8_t *W, int64_t m, int z) {
    int64_t hits = 0;
    for (int64_t p = 0; p + m <= n; ++p) {
        int mm = 0;
        for (int64_t d = 0; d < m && mm <= z; ++d) mm += (R[p + d] != W[d]);
        if (mm <= z) hits++;
    }
    return hits;
}
