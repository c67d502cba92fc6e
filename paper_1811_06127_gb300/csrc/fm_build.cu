// Index construction on the device (Sec. 2: Eq. 1 suffix array, Eq. 2 BWT, C, and the
// checkpointed occurrence table).  Runs once per index, off the search path.
//
// Suffix array by prefix doubling (Manber and Myers 1993), each pass one radix sort of the
// n+1 suffixes by a 64-bit key:
//   pass 0: the first 27 symbols of each suffix in base 5 ($ = 0 beyond the end, A..T =
//            1..4; 5^27 < 2^63), so most suffixes are told apart without any doubling;
//   pass r: key = (rank_h(i), rank_h(i+h) + 1) with rank_h the start of i's group after the
//            previous pass, h doubling from 27; a suffix whose first h symbols include $ is
//            already alone in its group.
// Passes stop when every group is a singleton.  The radix sort and scans of this build path
// are CUB's (header library shipped with the CUDA toolkit); the search path uses none.
#include <cub/cub.cuh>

#include "fm_internal.cuh"

namespace fm {
namespace {

// reverse(R), the text of the second index (the D bound extends forward on it)
__global__ void k_reverse(const uint8_t *__restrict__ in, uint64_t n, uint8_t *__restrict__ out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = in[n - 1 - i];
}

// pass-0 key of suffix i: its first 27 symbols in base 5 ($ = 0 past the end); val = i
__global__ void k_keys27(const uint8_t *__restrict__ codes, uint64_t n, uint64_t *__restrict__ key,
                         uint32_t *__restrict__ val) {
    const uint64_t N = n + 1;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t k = 0;
#pragma unroll
        for (int d = 0; d < 27; ++d) {
            uint64_t p = i + d;
            uint32_t s = p < n ? (uint32_t)codes[p] + 1u : 0u;
            k = k * 5u + s;
        }
        key[i] = k;
        val[i] = (uint32_t)i;
    }
}

// head[j] = j at the first element of each run of equal keys, 0 elsewhere; count the heads
__global__ void k_heads(const uint64_t *__restrict__ key, uint64_t N, uint32_t *__restrict__ head,
                        unsigned long long *__restrict__ nheads) {
    unsigned long long local = 0;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < N;
         j += (uint64_t)gridDim.x * blockDim.x) {
        bool h = (j == 0) || key[j] != key[j - 1];
        head[j] = h ? (uint32_t)j : 0u;
        local += h;
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(nheads, local);
}

// rank[suffix] = the start of its group, from the sorted order (val) and the group heads
__global__ void k_scatter_rank(const uint32_t *__restrict__ val, const uint32_t *__restrict__ grp,
                               uint64_t N, uint32_t *__restrict__ rank) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < N;
         j += (uint64_t)gridDim.x * blockDim.x)
        rank[val[j]] = grp[j];
}

// doubling key of suffix i: (rank_h(i), rank_h(i+h) + 1), 0 when i+h passes the end
__global__ void k_keys_double(const uint32_t *__restrict__ rank, uint64_t N, uint64_t h, int shift,
                              uint64_t *__restrict__ key, uint32_t *__restrict__ val) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t second = (i + h < N) ? (uint64_t)rank[i + h] + 1u : 0u;
        key[i] = ((uint64_t)rank[i] << shift) | second;
        val[i] = (uint32_t)i;
    }
}

// BWT (Eq. 2) as codes with $ stored as A, the $ row, and the SA samples
__global__ void k_bwt(const uint32_t *__restrict__ sa, const uint8_t *__restrict__ codes, uint64_t N,
                      uint64_t rate, uint8_t *__restrict__ bwt, uint32_t *__restrict__ sa_sample,
                      unsigned long long *__restrict__ dollar) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < N;
         j += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t s = sa[j];
        if (s == 0) {
            bwt[j] = 0;
            *dollar = j;
        } else {
            bwt[j] = codes[s - 1];
        }
        if (j % rate == 0) sa_sample[j / rate] = s;
    }
}

// per-block symbol counts of rows [j*I, min((j+1)*I, N)), $ row excluded
__global__ void k_block_counts(const uint8_t *__restrict__ bwt, uint64_t N, uint32_t I,
                               uint64_t nb, const unsigned long long *__restrict__ dollar,
                               uint4 *__restrict__ bc) {
    uint64_t drow = *dollar;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < nb;
         j += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t c[4] = {0, 0, 0, 0};
        uint64_t s = j * I, e = s + I < N ? s + I : N;
        for (uint64_t r = s; r < e; ++r) c[bwt[r]]++;
        if (drow >= s && drow < e) c[0]--;
        bc[j] = make_uint4(c[0], c[1], c[2], c[3]);
    }
}

struct AddU4 {
    __host__ __device__ uint4 operator()(const uint4 &a, const uint4 &b) const {
        return make_uint4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
    }
};

// one thread per 64-bit symbol word (32 rows); thread w < nb writes block w's counters
__global__ void k_pack(const uint8_t *__restrict__ bwt, uint64_t N, uint32_t I, uint32_t bbytes,
                       uint64_t nb, const uint4 *__restrict__ scan, uint8_t *__restrict__ blocks) {
    const uint32_t wpb = I / 32;
    const uint64_t nwords = nb * wpb;
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < nwords;
         w += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t j = w / wpb, slot = w % wpb;
        uint64_t r0 = w * 32;
        uint64_t word = 0;
        for (int t = 0; t < 32; ++t) {
            uint64_t r = r0 + t;
            uint64_t s = r < N ? (uint64_t)(bwt[r] & 3u) : 0u;
            word |= s << (2 * t);
        }
        uint8_t *bp = blocks + j * bbytes;
        reinterpret_cast<uint64_t *>(bp + 16)[slot] = word;
        if (slot == 0) *reinterpret_cast<uint4 *>(bp) = scan[j];
    }
}

int grid_for(uint64_t n, int sms) {
    uint64_t g = (n + 255) / 256;
    uint64_t cap = (uint64_t)sms * 32;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

int bits_for(uint64_t v) {
    int b = 1;
    while (b < 63 && ((1ull << b) <= v)) ++b;
    return b;
}

}  // namespace

// Build the checkpoint blocks of the text in d_codes (n codes 0..3, device); optionally of its
// reverse.  Temporaries are freed before returning.
int build_index(fm_index *h, const uint8_t *d_codes_in, uint64_t n, bool reverse,
                uint8_t **out_blocks, uint64_t *out_dollar, uint64_t C[5],
                uint32_t **out_sa_sample, cudaStream_t st) {
    const uint64_t N = n + 1;
    const uint32_t I = h->interval;
    const uint32_t bb = block_bytes(I);
    const uint64_t nb = N / I + 1;
    const int sms = h->sms;
    const int G = grid_for(N, sms);

    uint8_t *d_codes = const_cast<uint8_t *>(d_codes_in);
    uint8_t *d_revbuf = nullptr;
    uint64_t *key[2] = {nullptr, nullptr};
    uint32_t *val[2] = {nullptr, nullptr};
    uint32_t *rank = nullptr, *grp = nullptr;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    unsigned long long *d_cnt = nullptr;
    uint8_t *bwt = nullptr;
    uint4 *bc = nullptr;
    uint8_t *blocks = nullptr;
    uint32_t *sa_sample = nullptr;
    int rc = FM_OK;
    cudaError_t e = cudaSuccess;

#define BTRY(call)                                      \
    do {                                                \
        e = (call);                                     \
        if (e != cudaSuccess) {                         \
            rc = cuda_status(h, e, #call);              \
            goto done;                                  \
        }                                               \
    } while (0)

    {
        if (reverse) {
            BTRY(cudaMallocAsync((void **)&d_revbuf, n, st));
            k_reverse<<<grid_for(n, sms), 256, 0, st>>>(d_codes_in, n, d_revbuf);
            d_codes = d_revbuf;
        }
        BTRY(cudaMallocAsync((void **)&key[0], N * 8, st));
        BTRY(cudaMallocAsync((void **)&key[1], N * 8, st));
        BTRY(cudaMallocAsync((void **)&val[0], N * 4, st));
        BTRY(cudaMallocAsync((void **)&val[1], N * 4, st));
        BTRY(cudaMallocAsync((void **)&rank, N * 4, st));
        BTRY(cudaMallocAsync((void **)&grp, N * 4, st));
        BTRY(cudaMallocAsync((void **)&d_cnt, 16, st));

        k_keys27<<<G, 256, 0, st>>>(d_codes, n, key[0], val[0]);
        BTRY(cudaGetLastError());

        cub::DoubleBuffer<uint64_t> dk(key[0], key[1]);
        cub::DoubleBuffer<uint32_t> dv(val[0], val[1]);
        const int nbits = bits_for(N);        // ranks and second keys are <= N
        size_t need = 0;
        BTRY(cub::DeviceRadixSort::SortPairs(nullptr, need, dk, dv, (int)N, 0, 64, st));
        {
            size_t need2 = 0;
            BTRY(cub::DeviceScan::InclusiveScan(nullptr, need2, grp, grp, cuda::maximum<uint32_t>(),
                                                (int)N, st));
            if (need2 > need) need = need2;
            size_t need3 = 0;
            BTRY(cub::DeviceScan::ExclusiveScan(nullptr, need3, (uint4 *)nullptr, (uint4 *)nullptr,
                                                AddU4(), make_uint4(0, 0, 0, 0), (int)(nb + 1), st));
            if (need3 > need) need = need3;
        }
        tmp_bytes = need;
        BTRY(cudaMallocAsync(&tmp, tmp_bytes, st));

        int end_bit = 63;   // 5^27 < 2^63
        uint64_t hlen = 27;
        for (int pass = 0; pass < 64; ++pass) {
            size_t tb = tmp_bytes;
            BTRY(cub::DeviceRadixSort::SortPairs(tmp, tb, dk, dv, (int)N, 0, end_bit, st));
            BTRY(cudaMemsetAsync(d_cnt, 0, 8, st));
            k_heads<<<G, 256, 0, st>>>(dk.Current(), N, grp, d_cnt);
            BTRY(cudaGetLastError());
            tb = tmp_bytes;
            BTRY(cub::DeviceScan::InclusiveScan(tmp, tb, grp, grp, cuda::maximum<uint32_t>(), (int)N,
                                                st));
            unsigned long long heads = 0;
            BTRY(cudaMemcpyAsync(&heads, d_cnt, 8, cudaMemcpyDeviceToHost, st));
            BTRY(cudaStreamSynchronize(st));
            if (heads == N) break;   // every suffix alone: dv.Current() is the SA
            k_scatter_rank<<<G, 256, 0, st>>>(dv.Current(), grp, N, rank);
            BTRY(cudaGetLastError());
            // next pass: keys (rank(i), rank(i+h)+1) into the current key buffer
            k_keys_double<<<G, 256, 0, st>>>(rank, N, hlen, nbits, dk.Current(), dv.Current());
            BTRY(cudaGetLastError());
            end_bit = 2 * nbits;
            hlen *= 2;
            if (pass == 63) {
                rc = set_error(h, FM_ECUDA, "suffix sorting did not converge");
                goto done;
            }
        }
        const uint32_t *sa = dv.Current();

        // free the sort buffers not holding the SA before allocating the tables
        BTRY(cudaFreeAsync(key[0], st));
        key[0] = nullptr;
        BTRY(cudaFreeAsync(key[1], st));
        key[1] = nullptr;
        BTRY(cudaFreeAsync(rank, st));
        rank = nullptr;

        const uint64_t rate = h->sa_rate;
        const uint64_t nsamp = (N + rate - 1) / rate;
        BTRY(cudaMallocAsync((void **)&bwt, N, st));
        BTRY(cudaMallocAsync((void **)&sa_sample, nsamp * 4, st));
        BTRY(cudaMemsetAsync(d_cnt, 0, 16, st));
        k_bwt<<<G, 256, 0, st>>>(sa, d_codes, N, rate, bwt, sa_sample, d_cnt);
        BTRY(cudaGetLastError());

        // per-block counts, then an exclusive scan over nb+1 entries: entry j is
        // rank(., j*I) and entry nb holds the totals
        BTRY(cudaMallocAsync((void **)&bc, (nb + 1) * sizeof(uint4), st));
        BTRY(cudaMemsetAsync(bc + nb, 0, sizeof(uint4), st));
        k_block_counts<<<grid_for(nb, sms), 256, 0, st>>>(bwt, N, I, nb, d_cnt, bc);
        BTRY(cudaGetLastError());
        {
            size_t tb = tmp_bytes;
            BTRY(cub::DeviceScan::ExclusiveScan(tmp, tb, bc, bc, AddU4(), make_uint4(0, 0, 0, 0),
                                                (int)(nb + 1), st));
        }
        BTRY(cudaMallocAsync((void **)&blocks, nb * bb, st));
        BTRY(cudaMemsetAsync(blocks, 0, nb * bb, st));
        k_pack<<<grid_for(nb * (I / 32), sms), 256, 0, st>>>(bwt, N, I, bb, nb, bc, blocks);
        BTRY(cudaGetLastError());

        uint4 tot;
        unsigned long long drow = 0;
        BTRY(cudaMemcpyAsync(&tot, bc + nb, sizeof(uint4), cudaMemcpyDeviceToHost, st));
        BTRY(cudaMemcpyAsync(&drow, d_cnt, 8, cudaMemcpyDeviceToHost, st));
        BTRY(cudaStreamSynchronize(st));
        C[0] = 0;
        C[1] = tot.x;
        C[2] = C[1] + tot.y;
        C[3] = C[2] + tot.z;
        C[4] = C[3] + tot.w;
        *out_dollar = drow;
        *out_blocks = blocks;
        blocks = nullptr;
        if (out_sa_sample) {
            *out_sa_sample = sa_sample;
            sa_sample = nullptr;
        }
    }
done:
    if (d_revbuf) cudaFreeAsync(d_revbuf, st);
    if (key[0]) cudaFreeAsync(key[0], st);
    if (key[1]) cudaFreeAsync(key[1], st);
    if (val[0]) cudaFreeAsync(val[0], st);
    if (val[1]) cudaFreeAsync(val[1], st);
    if (rank) cudaFreeAsync(rank, st);
    if (grp) cudaFreeAsync(grp, st);
    if (tmp) cudaFreeAsync(tmp, st);
    if (d_cnt) cudaFreeAsync(d_cnt, st);
    if (bwt) cudaFreeAsync(bwt, st);
    if (bc) cudaFreeAsync(bc, st);
    if (blocks) cudaFreeAsync(blocks, st);
    if (sa_sample) cudaFreeAsync(sa_sample, st);
    cudaStreamSynchronize(st);
#undef BTRY
    return rc;
}

}  // namespace fm
