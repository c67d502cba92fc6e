// Hot-path kernels of the exact search: the eight-Occ query (Sec. 2 closing remarks, Sec. 3.3),
// Listing 1 (ExactRecur) and the D lower bound of the inexact search (forward extension on the
// index of reverse(R)).
//
// All three read the resident checkpoint blocks with 256-bit read-only gathers and count
// symbols with mask-and-popcount on the 2-bit words (fm_internal.cuh, rank4_in).  The role of
// the paper's half-byte lookup / SAD extraction (Sec. 3.1-3.2) is taken by that popcount:
// per 64-bit word, lo = w & 0x55.., hi = (w >> 1) & 0x55.., T = popc(lo & hi),
// C = popc(lo) - T, G = popc(hi) - T, and A is the remainder minus the $ correction.
#include "fm_internal.cuh"

#include <vector>

namespace fm {

IndexView view_fwd(const fm_index *h) {
    IndexView v;
    v.blocks = h->d_fwd;
    v.n = (uint32_t)h->n;
    v.dollar = (uint32_t)h->dollar;
    for (int i = 0; i < 5; ++i) v.C[i] = (uint32_t)h->C[i];
    v.kt = h->d_kt;
    v.kbits = h->d_kbits;
    v.kdepth = h->kt_depth;
    v.prec = h->d_prec;
    v.pc2 = h->d_pc2;
    v.pnblk = (uint32_t)((h->n + 1) / kPairRows + 1);
    v.pairs = h->pairs_built && h->tune.pairs ? 1u : 0u;
    return v;
}

IndexView view_rev(const fm_index *h) {
    IndexView v = view_fwd(h);
    v.blocks = h->d_rev;
    v.kt = h->d_kt_rev;
    v.kbits = h->d_kbits_rev;
    v.kdepth = h->d_kt_rev ? h->kt_depth : 0u;
    v.prec = h->d_prec_rev;
    v.pc2 = h->d_pc2_rev;
    v.pairs = h->pairs_built && h->tune.pairs && h->d_prec_rev ? 1u : 0u;
    v.dollar = (uint32_t)h->rev_dollar;
    return v;
}

namespace {

// -------------------------------------------------------------------------------------------
// eight Occ values per query
// -------------------------------------------------------------------------------------------
// Each thread takes Q queries (q, q + S, ..., S = grid size) and issues all their block loads
// before counting, so that 1..2*Q independent gathers per thread are in flight.
template <int I, int Q>
__global__ void __launch_bounds__(256) k_occ8(IndexView ix, const uint32_t *__restrict__ kq,
                                              const uint32_t *__restrict__ lq,
                                              uint32_t *__restrict__ out, uint64_t N,
                                              uint32_t *__restrict__ err) {
    const uint64_t S = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t q0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q0 < N; q0 += S * Q) {
        uint32_t p1[Q], p2[Q], j1[Q], j2[Q];
        bool ok[Q];
        Blk<I> B1[Q], B2[Q];
#pragma unroll
        for (int t = 0; t < Q; ++t) {
            uint64_t q = q0 + (uint64_t)t * S;
            ok[t] = false;
            p1[t] = p2[t] = 0;
            if (q < N) {
                uint32_t k = __ldcs(kq + q), l = __ldcs(lq + q);
                ok[t] = (k <= ix.n + 1u) && (l <= ix.n);
                if (ok[t]) {
                    p1[t] = k;       // Occ(c, k-1) = rank(c, k)
                    p2[t] = l + 1u;  // Occ(c, l)   = rank(c, l+1)
                }
            }
            j1[t] = p1[t] / I;
            j2[t] = p2[t] / I;
        }
#pragma unroll
        for (int t = 0; t < Q; ++t) {
            if (ok[t]) {
                uint32_t o1 = p1[t] - j1[t] * I, o2 = p2[t] - j2[t] * I;
                if (j1[t] == j2[t]) {
                    load_block<I>(ix.blocks, j1[t], o1 > o2 ? o1 : o2, B1[t]);
                    B2[t] = B1[t];
                } else {
                    load_block<I>(ix.blocks, j1[t], o1, B1[t]);
                    load_block<I>(ix.blocks, j2[t], o2, B2[t]);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < Q; ++t) {
            uint64_t q = q0 + (uint64_t)t * S;
            if (q >= N) continue;
            uint32_t a[4] = {0, 0, 0, 0}, b[4] = {0, 0, 0, 0};
            if (ok[t]) {
                rank4_in<I>(B1[t], j1[t], p1[t], ix.dollar, a);
                rank4_in<I>(B2[t], j2[t], p2[t], ix.dollar, b);
            } else {
                atomicOr(err, kErrDomain);
            }
            uint4 *o = reinterpret_cast<uint4 *>(out + 8 * q);
            __stcs(o, make_uint4(a[0], a[1], a[2], a[3]));
            __stcs(o + 1, make_uint4(b[0], b[1], b[2], b[3]));
        }
    }
}

// -------------------------------------------------------------------------------------------
// Listing 1, one thread per read
// -------------------------------------------------------------------------------------------
template <int I>
__global__ void __launch_bounds__(128) k_exact(IndexView ix, const uint8_t *__restrict__ reads,
                                               const uint32_t *__restrict__ offs, uint32_t nr,
                                               uint32_t *__restrict__ kout,
                                               uint32_t *__restrict__ lout,
                                               uint32_t *__restrict__ err) {
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += gridDim.x * blockDim.x) {
        const uint32_t s = offs[r], e = offs[r + 1];
        uint32_t k = 0, l = ix.n;
        // the last j0 symbols at once from the interval tables (their state is Listing 1's
        // after those j0 steps, insertion points included)
        const uint32_t j0 = e - s < ix.kdepth ? e - s : ix.kdepth;
        uint32_t code = 0, bad = 0;
        for (uint32_t t = 0; t < j0; ++t) {
            const uint32_t b = reads[e - j0 + t];
            bad |= b;
            code |= (b & 3u) << (2u * t);
        }
        if (bad > 3u) {
            atomicOr(err, kErrDomain);
            kout[r] = 0;
            lout[r] = ix.n;
            continue;
        }
        if (j0) {
            const uint2 kl = kt_get(ix, j0, code);
            k = kl.x;
            l = kl.y;
        }
        for (uint32_t i = e - j0; i > s; --i) {
            if (ix.pairs && i - s >= 2u) {
                // two symbols at once from the pair table (the same interval, insertion points
                // included, as two single steps)
                const uint32_t b2 = reads[i - 1], b1 = reads[i - 2];
                if ((b1 | b2) > 3u) {
                    atomicOr(err, kErrDomain);
                    k = 0;
                    l = ix.n;
                    break;
                }
                const uint32_t pc = 4u * b1 + b2, pk = k, pl = l + 1u;
                const uint2 Rk = load_pair_rec(ix, pc, pk / kPairRows);
                const uint2 Rl = pl / kPairRows == pk / kPairRows ? Rk : load_pair_rec(ix, pc, pl / kPairRows);
                const uint32_t c2 = __ldg(ix.pc2 + pc);
                k = c2 + pair_rank(Rk, pk);
                l = c2 + pair_rank(Rl, pl) - 1u;
                --i;
                continue;
            }
            const uint32_t b = reads[i - 1];
            if (b > 3u) {
                atomicOr(err, kErrDomain);
                k = 0;
                l = ix.n;
                break;
            }
            const uint32_t pk = k, pl = l + 1u;
            const uint32_t jk = pk / I, jl = pl / I;
            Blk<I> Bk, Bl;
            const uint32_t ok = pk - jk * I, ol = pl - jl * I;
            if (jk == jl) {
                load_block<I>(ix.blocks, jk, ok > ol ? ok : ol, Bk);
                Bl = Bk;
            } else {
                load_block<I>(ix.blocks, jk, ok, Bk);
                load_block<I>(ix.blocks, jl, ol, Bl);
            }
            const uint32_t rk = rank1_in<I>(Bk, jk, pk, ix.dollar, b);
            const uint32_t rl = rank1_in<I>(Bl, jl, pl, ix.dollar, b);
            const uint32_t cb = b == 0 ? ix.C[0] : (b == 1 ? ix.C[1] : (b == 2 ? ix.C[2] : ix.C[3]));
            k = cb + rk + 1u;
            l = cb + rl;
        }
        kout[r] = k;
        lout[r] = l;
    }
}

// -------------------------------------------------------------------------------------------
// D lower bound by forward extension on the index of reverse(R), one thread per query.
// qmeta[q * stride] = { D breakpoints 0..3, D breakpoints 4..7, read start,
// m | strand << 8 | mode << 16 }, mode = the query's search mode byte (differences allowed in
// bits 0-3, indel columns allowed in bits 4-7: modes[r] for read r, or defmode),
// with breakpoint j = first position i at which D(i) >= j+1 (255: never), so that
// D(i) = #{j : bp_j <= i}.  With stride kStageU4 (the staging record of the persistent search)
// the next four uint4 hold the query itself, oriented for its strand: W[i] at bits 2(i%16) of
// 32-bit word i/16 (words past the query's end are left as they were).
// -------------------------------------------------------------------------------------------
template <int I>
__global__ void __launch_bounds__(128) k_dcalc(IndexView rv, const uint8_t *__restrict__ reads,
                                               const uint32_t *__restrict__ offs, uint32_t nr,
                                               uint32_t strands, uint4 *__restrict__ qmeta,
                                               uint32_t stride, const uint8_t *__restrict__ modes,
                                               uint32_t defmode, uint8_t *__restrict__ D_out,
                                               uint32_t *__restrict__ err) {
    const uint32_t nq = nr * strands;
    const uint32_t L = rv.kdepth;   // interval tables of reverse(R) (0: none)
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        const uint32_t r = strands == 2 ? q >> 1 : q;
        const uint32_t strand = strands == 2 ? (q & 1u) : 0u;
        const uint32_t s = offs[r];
        const uint32_t m = offs[r + 1] - s;
        // breakpoint j = first i with D(i) >= j+1, 8 bits each, 255 = never
        uint32_t bp_lo = 0xffffffffu, bp_hi = 0xffffffffu;
        bool bad = m > (uint32_t)kMaxReadLen;
        if (bad) atomicOr(err, kErrReadLen);
        uint8_t *Dq = D_out ? D_out + (size_t)strands * s + (size_t)strand * m : nullptr;
        uint32_t *Wq = (qmeta && stride == kStageU4) ? (uint32_t *)(qmeta + (size_t)q * stride + 1) : nullptr;
        // W[i], oriented for the strand
        auto wsym = [&](uint32_t i) -> uint32_t {
            const uint32_t c = strand ? reads[s + m - 1 - i] : reads[s + i];
            return strand ? 3u - c : c;
        };
        // the codes are checked (and, for staging, packed 16 to a word) before the D bound
        {
            uint32_t wacc = 0;
            for (uint32_t i = 0; i < m && !bad; ++i) {
                const uint32_t c = strand ? reads[s + m - 1 - i] : reads[s + i];
                if (c > 3u) {
                    atomicOr(err, kErrDomain);
                    bad = true;
                    break;
                }
                if (Wq) {
                    wacc |= (strand ? 3u - c : c) << (2u * (i & 15u));
                    if ((i & 15u) == 15u || i + 1u == m) {
                        Wq[i >> 4] = wacc;
                        wacc = 0;
                    }
                }
            }
        }
        // a window W[j..i] that does not occur closes at i: the next breakpoint is i
        uint32_t z = 0;
        auto close_at = [&](uint32_t i) {
            if (z < 4) bp_lo = (bp_lo & ~(0xffu << (8 * z))) | (i << (8 * z));
            else if (z < 8) bp_hi = (bp_hi & ~(0xffu << (8 * (z - 4)))) | (i << (8 * (z - 4)));
            ++z;
        };
        uint32_t k = 0, l = rv.n;
        bool fresh = true;   // a window starts at i ([k, l] = [0, n])
        // Without a D array to fill, the pass stops once more windows have closed than the
        // query allows differences (zq): D only prunes, and every node at a position past that
        // breakpoint is pruned whatever the further breakpoints are.
        const uint32_t zq = (modes ? (uint32_t)modes[r] : defmode) & 15u;
        for (uint32_t i = 0; i < m && !bad && (Dq || z <= zq);) {
            if (L && fresh) {
                // The window's first dmax symbols from the tables of reverse(R): a window
                // W[i..i+d-1] occurs in R exactly when its reverse occurs in reverse(R), the
                // string whose code is P >> 2(L - d) with P holding W[i] in its highest symbol.
                // Prefixes of an occurring string occur, so the longest occurring d is found by
                // testing dmax first and else by bisection over the occurrence bits.
                const uint32_t dmax = m - i < L ? m - i : L;
                uint32_t P = 0;
                for (uint32_t t = 0; t < dmax; ++t) P = (P << 2) | wsym(i + t);
                P <<= 2u * (L - dmax);
                auto occurs = [&](uint32_t d) { return kt_occ1(rv, d, P >> (2u * (L - d))) != 0u; };
                uint32_t d = dmax;
                if (!occurs(dmax)) {
                    uint32_t lo = 0, hi = dmax - 1;   // occurs(lo), and d <= hi
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi + 1) / 2;
                        if (occurs(mid)) lo = mid; else hi = mid - 1;
                    }
                    d = lo;
                }
                if (Dq)
                    for (uint32_t t = 0; t < d; ++t) Dq[i + t] = (uint8_t)(z > 255 ? 255 : z);
                if (d < dmax) {   // W[i..i+d] does not occur: the window closes at i + d
                    close_at(i + d);
                    if (Dq) Dq[i + d] = (uint8_t)(z > 255 ? 255 : z);
                    i += d + 1;
                    continue;
                }
                i += dmax;
                if (i == m) break;
                const uint2 kl = kt_get(rv, L, P);   // dmax = L: continue from the table entry
                k = kl.x;
                l = kl.y;
                fresh = false;
                continue;
            }
            const uint32_t b = wsym(i);
            if (rv.pairs && i + 1u < m) {
                // W[i] and W[i+1] at once over the pair table of reverse(R) (prepended to the
                // reversed window in that order: pair code 4 W[i+1] + W[i]); a pair that does
                // not occur falls back to the single step below, which finds where the window
                // closes
                const uint32_t pc = 4u * wsym(i + 1u) + b, pk = k, pl = l + 1u;
                const uint2 Rk = load_pair_rec(rv, pc, pk / kPairRows);
                const uint2 Rl = pl / kPairRows == pk / kPairRows ? Rk : load_pair_rec(rv, pc, pl / kPairRows);
                const uint32_t c2 = __ldg(rv.pc2 + pc);
                const uint32_t k2 = c2 + pair_rank(Rk, pk), l2 = c2 + pair_rank(Rl, pl) - 1u;
                if (k2 <= l2) {
                    k = k2;
                    l = l2;
                    if (Dq) Dq[i] = Dq[i + 1] = (uint8_t)(z > 255 ? 255 : z);
                    i += 2;
                    continue;
                }
            }
            const uint32_t pk = k, pl = l + 1u;
            const uint32_t jk = pk / I, jl = pl / I;
            Blk<I> Bk, Bl;
            const uint32_t ok = pk - jk * I, ol = pl - jl * I;
            if (jk == jl) {
                load_block<I>(rv.blocks, jk, ok > ol ? ok : ol, Bk);
                Bl = Bk;
            } else {
                load_block<I>(rv.blocks, jk, ok, Bk);
                load_block<I>(rv.blocks, jl, ol, Bl);
            }
            const uint32_t cb = b == 0 ? rv.C[0] : (b == 1 ? rv.C[1] : (b == 2 ? rv.C[2] : rv.C[3]));
            const uint32_t k2 = cb + rank1_in<I>(Bk, jk, pk, rv.dollar, b) + 1u;
            const uint32_t l2 = cb + rank1_in<I>(Bl, jl, pl, rv.dollar, b);
            if (k2 > l2) {   // W[j..i] does not occur: close the window, restart after i
                close_at(i);
                k = 0;
                l = rv.n;
                fresh = true;
            } else {
                k = k2;
                l = l2;
            }
            if (Dq) Dq[i] = (uint8_t)(z > 255 ? 255 : z);
            ++i;
        }
        if (qmeta) {
            uint4 mt;
            mt.x = bp_lo;
            mt.y = bp_hi;
            mt.z = s;
            // a bad query is given length 0: the search then reports nothing for it
            mt.w = (bad ? 0u : m) | (strand << 8) | ((modes ? (uint32_t)modes[r] : defmode) << 16);
            qmeta[(size_t)q * stride] = mt;
        }
    }
}

// -------------------------------------------------------------------------------------------
// Locate (Sec. 2, Eq. 4-5): SA[row] from the rows sampled every `rate` (SA[j*rate] kept) by
// walking LF(i) = C[BWT[i]] + Occ(BWT[i], i), which moves to the row of the suffix one text
// position earlier, so SA[row] = SA[LF^j(row)] + j at the first sampled row.  The $ row holds
// suffix 0 (SA = 0) and ends a walk too.  One thread per row; every step is one block gather.
// -------------------------------------------------------------------------------------------
template <int I>
__global__ void __launch_bounds__(256) k_locate(IndexView ix, const uint32_t *__restrict__ sa_sample,
                                                uint32_t rate, const uint32_t *__restrict__ rows,
                                                uint64_t N, uint32_t *__restrict__ pos,
                                                unsigned long long *__restrict__ steps,
                                                uint32_t *__restrict__ err) {
    unsigned long long my_steps = 0;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < N;
         q += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t i = rows[q];
        if (i > ix.n) {
            atomicOr(err, kErrDomain);
            pos[q] = 0;
            continue;
        }
        uint32_t j = 0;
        for (;;) {
            if (i % rate == 0) {
                pos[q] = sa_sample[i / rate] + j;
                break;
            }
            if (i == ix.dollar) {
                pos[q] = j;
                break;
            }
            const uint32_t jb = i / I;
            Blk<I> B;
            load_block<I>(ix.blocks, jb, i - jb * I + 1u, B);
            const uint32_t b = sym_in<I>(B, jb, i);
            const uint32_t cb = b == 0 ? ix.C[0] : (b == 1 ? ix.C[1] : (b == 2 ? ix.C[2] : ix.C[3]));
            i = cb + rank1_in<I>(B, jb, i, ix.dollar, b) + 1u;   // Occ(b, i) = rank(b, i) + 1
            ++j;
        }
        my_steps += j;
    }
    if (steps) {
        for (int o = 16; o > 0; o >>= 1) my_steps += __shfl_down_sync(0xffffffffu, my_steps, o);
        if ((threadIdx.x & 31) == 0 && my_steps) atomicAdd(steps, my_steps);
    }
}

// -------------------------------------------------------------------------------------------
// Interval tables of short strings.  Level j+1 from level j: one eight-Occ step per string X of
// length j gives the four extensions bX (codes 4 code(X) + b), by Listing 1's formula whether or
// not X occurs, so every entry is Listing 1's state after reading its string.
// -------------------------------------------------------------------------------------------
template <int I>
__global__ void __launch_bounds__(256) k_kmer_level(IndexView ix, uint2 *__restrict__ kt, uint32_t j) {
    const uint32_t cnt = 1u << (2u * j);
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < cnt; c += gridDim.x * blockDim.x) {
        const uint2 kl = kt[cnt + c];
        const uint32_t pk = kl.x, pl = kl.y + 1u;
        const uint32_t jk = pk / I, jl = pl / I;
        Blk<I> Bk, Bl;
        load_block<I>(ix.blocks, jk, pk - jk * I, Bk);
        load_block<I>(ix.blocks, jl, pl - jl * I, Bl);
        uint32_t rk[4], rl[4];
        rank4_in<I>(Bk, jk, pk, ix.dollar, rk);
        rank4_in<I>(Bl, jl, pl, ix.dollar, rl);
        uint2 *out = kt + 4u * cnt + 4u * c;
#pragma unroll
        for (int b = 0; b < 4; ++b) out[b] = make_uint2(ix.C[b] + rk[b] + 1u, ix.C[b] + rl[b]);
    }
}

// occurrence bits: bit t (t in [4^j, 2 4^j), j <= L) = entry t is non-empty; other bits 0
__global__ void __launch_bounds__(256) k_kmer_bits(const uint2 *__restrict__ kt, uint32_t *__restrict__ bits,
                                                   uint32_t nwords, uint32_t L) {
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += gridDim.x * blockDim.x) {
        uint32_t word = 0;
        for (uint32_t u = 0; u < 32u; ++u) {
            const uint32_t t = 32u * w + u;
            if (t == 0u) continue;
            const uint32_t j = (31u - (uint32_t)__clz(t)) >> 1;
            if (j > L || t >= (2u << (2u * j))) continue;
            const uint2 kl = kt[t];
            if (kl.x <= kl.y) word |= 1u << u;
        }
        bits[w] = word;
    }
}

// -------------------------------------------------------------------------------------------
// Pair table.  Row i's pair is (BWT[LF(i)], BWT[i]) with LF(i) = C[b] + rank(b, i) + 1 for
// b = BWT[i] (Eq. 4-5): the two symbols before suffix SA[i].  Thread per 32-row block: the
// rows of each pair code among them, written into the sixteen records of the block (word 1).
// The $ row and the row whose LF is the $ row have no pair (row b recorded).
// -------------------------------------------------------------------------------------------
template <int I>
__global__ void __launch_bounds__(256) k_pair_sym(IndexView ix, uint2 *__restrict__ prec, uint64_t nblk,
                                                  uint64_t N, uint32_t *__restrict__ row_b) {
    const uint64_t nrows32 = (N + 31) / 32;   // 32-row blocks holding rows
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < nrows32;
         w += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t rows[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) rows[c] = 0u;
        for (uint32_t t = 0; t < 32u; ++t) {
            const uint64_t i64 = 32 * w + t;
            if (i64 >= N) break;
            const uint32_t i = (uint32_t)i64;
            if (i == ix.dollar) continue;
            const uint32_t jb = i / I;
            Blk<I> B;
            load_block<I>(ix.blocks, jb, i - jb * I + 1u, B);
            const uint32_t b = sym_in<I>(B, jb, i);
            const uint32_t cb = b == 0 ? ix.C[0] : (b == 1 ? ix.C[1] : (b == 2 ? ix.C[2] : ix.C[3]));
            const uint32_t lf = cb + rank1_in<I>(B, jb, i, ix.dollar, b) + 1u;
            if (lf == ix.dollar) {
                *row_b = i;
                continue;
            }
            const uint32_t jl = lf / I;
            Blk<I> L;
            load_block<I>(ix.blocks, jl, lf - jl * I + 1u, L);
            const uint32_t code = 4u * sym_in<I>(L, jl, lf) + b;
#pragma unroll
            for (int c = 0; c < 16; ++c) rows[c] |= (code == (uint32_t)c ? 1u : 0u) << t;
        }
#pragma unroll
        for (int c = 0; c < 16; ++c) prec[(size_t)c * nblk + w].y = rows[c];
    }
}

// Thread per (pair code c, run of kPairScanBlocks blocks): x of each record = pairs c in the
// run's rows before its block; the run's total goes to tot.
__global__ void __launch_bounds__(256) k_pair_counts(uint2 *__restrict__ prec, uint64_t nblk, uint64_t nrun,
                                                     uint32_t *__restrict__ tot) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < nrun * 16;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t c = t / nrun, run = t % nrun;
        uint2 *rec = prec + c * nblk;
        const uint64_t j0 = run * kPairScanBlocks;
        const uint64_t j1 = j0 + kPairScanBlocks < nblk ? j0 + kPairScanBlocks : nblk;
        uint32_t acc = 0;
        for (uint64_t j = j0; j < j1; ++j) {
            rec[j].x = acc;
            acc += __popc(rec[j].y);
        }
        tot[t] = acc;
    }
}

// Thread per record: add the pairs c before its run (base[c * nrun + run]).
__global__ void __launch_bounds__(256) k_pair_base(uint2 *__restrict__ prec, uint64_t nblk, uint64_t nrun,
                                                   const uint32_t *__restrict__ base) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < nblk * 16;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t c = t / nblk, j = t % nblk;
        prec[t].x += base[c * nrun + j / kPairScanBlocks];
    }
}

int grid_occ(fm_index *h, uint64_t work, int block) {
    uint64_t g = (work + block - 1) / block;
    uint64_t cap = (uint64_t)h->sms * (2048 / block) * 4;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

template <int Q>
static void occ8_q(fm_index *h, IndexView ix, const uint32_t *k, const uint32_t *l, uint32_t *out8,
                   uint64_t N, uint32_t *err, cudaStream_t st) {
    const int block = 256;
    int grid = grid_occ(h, (N + Q - 1) / Q, block);
    switch (h->interval) {
        case 32: k_occ8<32, Q><<<grid, block, 0, st>>>(ix, k, l, out8, N, err); break;
        case 64: k_occ8<64, Q><<<grid, block, 0, st>>>(ix, k, l, out8, N, err); break;
        case 128: k_occ8<128, Q><<<grid, block, 0, st>>>(ix, k, l, out8, N, err); break;
        default: k_occ8<256, Q><<<grid, block, 0, st>>>(ix, k, l, out8, N, err); break;
    }
}

int launch_occ8(fm_index *h, const uint32_t *k, const uint32_t *l, uint32_t *out8, uint64_t N,
                cudaStream_t st) {
    if (N == 0) return FM_OK;
    IndexView ix = view_fwd(h);
    uint32_t *err = h->d_err + kErrOcc;
    switch (h->tune.occ_q) {
        case 1: occ8_q<1>(h, ix, k, l, out8, N, err, st); break;
        case 4: occ8_q<4>(h, ix, k, l, out8, N, err, st); break;
        default: occ8_q<2>(h, ix, k, l, out8, N, err, st); break;
    }
    FM_CUDA_TRY(h, cudaGetLastError());
    return FM_OK;
}

int launch_locate(fm_index *h, const uint32_t *rows, uint64_t N, uint32_t *pos,
                  unsigned long long *steps, cudaStream_t st) {
    if (N == 0) return FM_OK;
    IndexView ix = view_fwd(h);
    uint32_t *err = h->d_err + kErrExact;
    const int block = 256;
    const int grid = grid_occ(h, N, block);
    const uint32_t rate = (uint32_t)h->sa_rate;
    switch (h->interval) {
        case 32: k_locate<32><<<grid, block, 0, st>>>(ix, h->d_sa_sample, rate, rows, N, pos, steps, err); break;
        case 64: k_locate<64><<<grid, block, 0, st>>>(ix, h->d_sa_sample, rate, rows, N, pos, steps, err); break;
        case 128: k_locate<128><<<grid, block, 0, st>>>(ix, h->d_sa_sample, rate, rows, N, pos, steps, err); break;
        default: k_locate<256><<<grid, block, 0, st>>>(ix, h->d_sa_sample, rate, rows, N, pos, steps, err); break;
    }
    FM_CUDA_TRY(h, cudaGetLastError());
    return FM_OK;
}

uint32_t kmer_depth_for(const fm_index *h) {
    const uint32_t set = h->tune.kmer;
    if (set == FM_KMER_OFF) return 0;
    if (set != FM_KMER_AUTO) return set < kMaxKmerDepth ? set : kMaxKmerDepth;
    uint32_t lg = 0;   // floor(log4(n + 1))
    while (lg < 31 && (1ull << (2 * (lg + 1))) <= h->n + 1) ++lg;
    // one level below the length at which a random string stops occurring: exact chains and
    // the D bound cross the whole table region in one lookup, so the deepest useful tables
    // pay (measured at 2 Gbp: depth 14 634 ms, 13 689 ms, 15 646 ms)
    const uint32_t d = lg > 1 ? lg - 1 : 0;
    return d < kMaxKmerDepth ? d : kMaxKmerDepth;
}

int ensure_kmer(fm_index *h, cudaStream_t st) {
    if (h->borrowed) return FM_OK;   // a search context uses its owner's tables as they are
    const uint32_t L = kmer_depth_for(h);
    if (L == h->kt_depth) return FM_OK;
    FM_CUDA_TRY(h, cudaStreamSynchronize(st));   // no kernel of this stream reads the old tables
    uint2 **kts[2] = {&h->d_kt, &h->d_kt_rev};
    uint32_t **kbs[2] = {&h->d_kbits, &h->d_kbits_rev};
    for (int v = 0; v < 2; ++v) {
        cudaFree(*kts[v]);
        cudaFree(*kbs[v]);
        *kts[v] = nullptr;
        *kbs[v] = nullptr;
    }
    h->kt_depth = 0;
    if (L == 0) return FM_OK;
    const uint64_t entries = 2ull << (2 * L);
    const uint64_t nwords = (entries + 31) / 32;
    // the forward index's tables (search) and, with the index of reverse(R), that index's own
    // (the D bound: windows of a query are looked up as strings of reverse(R))
    for (int v = 0; v < (h->has_rev ? 2 : 1); ++v) {
        if (cudaMalloc(kts[v], entries * sizeof(uint2)) != cudaSuccess ||
            cudaMalloc(kbs[v], nwords * sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            for (int u = 0; u < 2; ++u) {
                cudaFree(*kts[u]);
                cudaFree(*kbs[u]);
                *kts[u] = nullptr;
                *kbs[u] = nullptr;
            }
            return set_error(h, FM_ENOMEM, "interval tables: out of device memory");
        }
        const uint2 root = make_uint2(0u, (uint32_t)h->n);   // the empty string: [0, n]
        FM_CUDA_TRY(h, cudaMemcpyAsync(*kts[v] + 1, &root, sizeof(root), cudaMemcpyHostToDevice, st));
        IndexView ix = view_fwd(h);
        if (v == 1) {
            ix = view_rev(h);
            ix.kt = nullptr;   // the steps below read checkpoint blocks only
            ix.kbits = nullptr;
            ix.kdepth = 0;
        }
        for (uint32_t j = 0; j < L; ++j) {
            const int block = 256;
            const int grid = grid_occ(h, 1ull << (2 * j), block);
            switch (h->interval) {
                case 32: k_kmer_level<32><<<grid, block, 0, st>>>(ix, *kts[v], j); break;
                case 64: k_kmer_level<64><<<grid, block, 0, st>>>(ix, *kts[v], j); break;
                case 128: k_kmer_level<128><<<grid, block, 0, st>>>(ix, *kts[v], j); break;
                default: k_kmer_level<256><<<grid, block, 0, st>>>(ix, *kts[v], j); break;
            }
            FM_CUDA_TRY(h, cudaGetLastError());
        }
        k_kmer_bits<<<grid_occ(h, nwords, 256), 256, 0, st>>>(*kts[v], *kbs[v], (uint32_t)nwords, L);
        FM_CUDA_TRY(h, cudaGetLastError());
    }
    FM_CUDA_TRY(h, cudaStreamSynchronize(st));
    h->kt_depth = L;
    return FM_OK;
}

// The pair records and pc2 of the index ix views (blocks: its checkpoint blocks, whose first
// holds the symbol before its $ suffix, the text's last symbol).
static int build_pair_table(fm_index *h, const IndexView &ix, const uint8_t *blocks, uint2 **prec,
                            uint32_t **pc2_out, cudaStream_t st) {
    const uint64_t N = h->n + 1;                    // rows
    const uint64_t nblk = N / kPairRows + 1;        // rank positions 0..N
    const uint64_t nrun = (nblk + kPairScanBlocks - 1) / kPairScanBlocks;
    const uint32_t sentinel = 0xffffffffu;
    uint32_t *d_rowb = nullptr, *d_tot = nullptr;
    int rc = FM_OK;
    if (cudaMalloc(prec, nblk * 16 * sizeof(uint2)) != cudaSuccess ||
        cudaMalloc(pc2_out, 16 * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&d_tot, nrun * 16 * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&d_rowb, sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        rc = set_error(h, FM_ENOMEM, "pair table: out of device memory");
    }
    std::vector<uint32_t> tot, base;
    if (!rc) {
        FM_CUDA_TRY(h, cudaMemsetAsync(*prec, 0, nblk * 16 * sizeof(uint2), st));
        FM_CUDA_TRY(h, cudaMemcpyAsync(d_rowb, &sentinel, 4, cudaMemcpyHostToDevice, st));
        const int grid = grid_occ(h, (N + 7) / 8, 256);
        switch (h->interval) {
            case 32: k_pair_sym<32><<<grid, 256, 0, st>>>(ix, *prec, nblk, N, d_rowb); break;
            case 64: k_pair_sym<64><<<grid, 256, 0, st>>>(ix, *prec, nblk, N, d_rowb); break;
            case 128: k_pair_sym<128><<<grid, 256, 0, st>>>(ix, *prec, nblk, N, d_rowb); break;
            default: k_pair_sym<256><<<grid, 256, 0, st>>>(ix, *prec, nblk, N, d_rowb); break;
        }
        FM_CUDA_TRY(h, cudaGetLastError());
        uint32_t rowb = sentinel;
        FM_CUDA_TRY(h, cudaMemcpyAsync(&rowb, d_rowb, 4, cudaMemcpyDeviceToHost, st));
        FM_CUDA_TRY(h, cudaStreamSynchronize(st));
        if (rowb == sentinel) rc = set_error(h, FM_ECUDA, "pair table: no row precedes the $ row");
    }
    if (!rc) {
        k_pair_counts<<<grid_occ(h, nrun * 16, 256), 256, 0, st>>>(*prec, nblk, nrun, d_tot);
        FM_CUDA_TRY(h, cudaGetLastError());
        tot.resize(nrun * 16);
        FM_CUDA_TRY(h, cudaMemcpyAsync(tot.data(), d_tot, nrun * 16 * 4, cudaMemcpyDeviceToHost, st));
        // the symbol of row 0 (the $ suffix) is the text's last symbol: read it from the first
        // checkpoint block
        uint8_t b0[32];
        FM_CUDA_TRY(h, cudaMemcpyAsync(b0, blocks, 32, cudaMemcpyDeviceToHost, st));
        FM_CUDA_TRY(h, cudaStreamSynchronize(st));
        const uint32_t last = b0[16] & 3u;
        // run bases (exclusive scan per pair code), then pc2
        base.assign(nrun * 16, 0u);
        uint64_t run[16] = {0};
        for (int c = 0; c < 16; ++c)
            for (uint64_t r = 0; r < nrun; ++r) {
                base[c * nrun + r] = (uint32_t)run[c];
                run[c] += tot[c * nrun + r];
            }
        // rows before every string that starts with pair (b1, b2): the $ row, suffixes starting
        // with a symbol below b1, the suffix "b1 $" when the text ends with b1, and suffixes
        // starting with b1 then a symbol below b2 (C is the same for R and reverse(R))
        uint32_t pc2[16];
        for (uint32_t b1 = 0; b1 < 4; ++b1)
            for (uint32_t b2 = 0; b2 < 4; ++b2) {
                uint64_t v = 1 + h->C[b1] + (last == b1 ? 1 : 0);
                for (uint32_t y = 0; y < b2; ++y) v += run[4 * b1 + y];
                pc2[4 * b1 + b2] = (uint32_t)v;
            }
        FM_CUDA_TRY(h, cudaMemcpyAsync(d_tot, base.data(), base.size() * 4, cudaMemcpyHostToDevice, st));
        FM_CUDA_TRY(h, cudaMemcpyAsync(*pc2_out, pc2, sizeof(pc2), cudaMemcpyHostToDevice, st));
        k_pair_base<<<grid_occ(h, nblk * 16, 256), 256, 0, st>>>(*prec, nblk, nrun, d_tot);
        FM_CUDA_TRY(h, cudaGetLastError());
        FM_CUDA_TRY(h, cudaStreamSynchronize(st));
    }
    cudaFree(d_tot);
    cudaFree(d_rowb);
    if (rc) {
        cudaFree(*prec);
        cudaFree(*pc2_out);
        *prec = nullptr;
        *pc2_out = nullptr;
    }
    return rc;
}

// The pair tables: the forward index's (search steps) and, with the index of reverse(R), that
// index's own (two-symbol steps of the D pass).
int ensure_pairs(fm_index *h, cudaStream_t st) {
    if (!h->tune.pairs || h->pairs_built || h->borrowed) return FM_OK;
    FM_CUDA_TRY(h, cudaStreamSynchronize(st));
    int rc = build_pair_table(h, view_fwd(h), h->d_fwd, &h->d_prec, &h->d_pc2, st);
    if (!rc && h->has_rev) {
        IndexView rv = view_rev(h);
        rv.kt = nullptr;   // the builder's steps read checkpoint blocks only
        rv.kbits = nullptr;
        rv.kdepth = 0;
        rc = build_pair_table(h, rv, h->d_rev, &h->d_prec_rev, &h->d_pc2_rev, st);
    }
    if (rc) {
        cudaFree(h->d_prec);
        cudaFree(h->d_pc2);
        h->d_prec = nullptr;
        h->d_pc2 = nullptr;
        return rc;
    }
    h->pairs_built = true;
    return FM_OK;
}

int launch_exact(fm_index *h, const uint8_t *reads, const uint32_t *offs, uint32_t n_reads,
                 uint32_t *k_out, uint32_t *l_out, cudaStream_t st) {
    if (n_reads == 0) return FM_OK;
    if (int rc = ensure_kmer(h, st)) return rc;
    if (int rc = ensure_pairs(h, st)) return rc;
    IndexView ix = view_fwd(h);
    uint32_t *err = h->d_err + kErrExact;
    const int block = 128;
    int grid = grid_occ(h, n_reads, block);
    switch (h->interval) {
        case 32: k_exact<32><<<grid, block, 0, st>>>(ix, reads, offs, n_reads, k_out, l_out, err); break;
        case 64: k_exact<64><<<grid, block, 0, st>>>(ix, reads, offs, n_reads, k_out, l_out, err); break;
        case 128: k_exact<128><<<grid, block, 0, st>>>(ix, reads, offs, n_reads, k_out, l_out, err); break;
        default: k_exact<256><<<grid, block, 0, st>>>(ix, reads, offs, n_reads, k_out, l_out, err); break;
    }
    FM_CUDA_TRY(h, cudaGetLastError());
    return FM_OK;
}

int launch_dcalc(fm_index *h, const uint8_t *reads, const uint32_t *offs, uint32_t n_reads,
                 uint32_t strands, uint4 *qmeta, uint8_t *D_out, cudaStream_t st, uint32_t stride,
                 const uint8_t *modes, uint32_t defmode) {
    uint64_t nq = (uint64_t)n_reads * strands;
    if (nq == 0) return FM_OK;
    IndexView rv = view_rev(h);
    uint32_t *err = h->d_err + kErrDcalc;
    const int block = 128;
    int grid = grid_occ(h, nq, block);
    switch (h->interval) {
        case 32: k_dcalc<32><<<grid, block, 0, st>>>(rv, reads, offs, n_reads, strands, qmeta, stride, modes, defmode, D_out, err); break;
        case 64: k_dcalc<64><<<grid, block, 0, st>>>(rv, reads, offs, n_reads, strands, qmeta, stride, modes, defmode, D_out, err); break;
        case 128: k_dcalc<128><<<grid, block, 0, st>>>(rv, reads, offs, n_reads, strands, qmeta, stride, modes, defmode, D_out, err); break;
        default: k_dcalc<256><<<grid, block, 0, st>>>(rv, reads, offs, n_reads, strands, qmeta, stride, modes, defmode, D_out, err); break;
    }
    FM_CUDA_TRY(h, cudaGetLastError());
    return FM_OK;
}

}  // namespace fm
