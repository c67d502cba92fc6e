// C ABI of the fmocc library (declarations and contracts in include/fmocc.h).
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "fm_internal.cuh"

namespace fm {

static thread_local std::string g_last_error;

int set_error(fm_index *h, int code, const std::string &msg) {
    if (h) h->err = msg;
    else g_last_error = msg;
    return code;
}

int set_global_error(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_status(fm_index *h, cudaError_t e, const char *what) {
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    int code = (e == cudaErrorMemoryAllocation) ? FM_ENOMEM : FM_ECUDA;
    cudaGetLastError();   // clear a sticky-free error so later calls can proceed
    return set_error(h, code, msg);
}

int device_sms(int device) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    return v;
}

namespace {

// Makes the index's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// T[n + i] = 3 - T[n - 1 - i] (the reverse complement after R, codes already checked)
__global__ void k_append_revcomp(uint8_t *__restrict__ t, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        t[n + i] = (uint8_t)(3u - t[n - 1 - i]);
}

// ACGTacgt (or codes 0..3) to codes 0..3 in place; any other symbol sets *err
__global__ void k_encode(uint8_t *__restrict__ t, uint64_t n, int ascii, uint32_t *__restrict__ err) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t c = t[i];
        uint32_t code;
        if (ascii) {
            switch (c | 0x20u) {   // case-insensitive
                case 'a': code = 0; break;
                case 'c': code = 1; break;
                case 'g': code = 2; break;
                case 't': code = 3; break;
                default: code = 255; break;
            }
        } else {
            code = c <= 3u ? c : 255u;
        }
        if (code == 255u) {
            atomicOr(err, kErrDomain);
            code = 0;
        }
        t[i] = (uint8_t)code;
    }
}

uint64_t fnv1a(uint64_t hsh, const void *p, size_t n) {
    const uint8_t *b = (const uint8_t *)p;
    for (size_t i = 0; i < n; ++i) {
        hsh ^= b[i];
        hsh *= 1099511628211ull;
    }
    return hsh;
}

constexpr uint64_t kFnvSeed = 1469598103934665603ull;
constexpr char kMagic[8] = {'F', 'M', 'O', 'C', 'C', '0', '0', '1'};

struct FileHeader {
    char magic[8];
    uint64_t n;
    uint32_t interval, bbytes;
    uint64_t n_blocks;
    uint64_t C[5];
    uint64_t dollar, rev_dollar;
    uint32_t has_rev, both_strands;
    uint64_t sa_rate, n_sa;
};

int alloc_common(fm_index *h) {
    cudaError_t e = cudaMalloc((void **)&h->d_err, kErrSlots * sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_status(h, e, "cudaMalloc(error words)");
    e = cudaMemset(h->d_err, 0, kErrSlots * sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_status(h, e, "cudaMemset(error words)");
    return FM_OK;
}

void release(fm_index *h) {
    if (!h) return;
    DeviceGuard g(h->device);
    cudaFree(h->d_fwd);
    cudaFree(h->d_rev);
    cudaFree(h->d_sa_sample);
    cudaFree(h->d_err);
    cudaFree(h->d_kt);
    cudaFree(h->d_kbits);
    cudaFree(h->d_kt_rev);
    cudaFree(h->d_kbits_rev);
    cudaFree(h->d_prec);
    cudaFree(h->d_pc2);
    cudaFree(h->d_prec_rev);
    cudaFree(h->d_pc2_rev);
    fm::Scratch *ss[] = {&h->s_qmeta, &h->s_raw, &h->s_spill, &h->s_group, &h->s_scan, &h->s_plain,
                         &h->s_misc};
    for (auto *s : ss) cudaFree(s->ptr);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (auto &e : h->gev)
        if (e) cudaEventDestroy(e);
    delete h;
}

}  // namespace

fm_index *new_search_context(fm_index *h) {
    fm_index *c = new fm_index(*h);
    c->borrowed = true;
    c->err.clear();
    fm::Scratch *ss[] = {&c->s_qmeta, &c->s_raw, &c->s_spill, &c->s_group, &c->s_scan, &c->s_plain,
                         &c->s_misc};
    for (auto *sc : ss) *sc = fm::Scratch{};
    c->scratch_budget = 0;
    c->d_err = nullptr;
    c->last_valid = false;
    c->cap_stream = nullptr;
    c->gexec = nullptr;
    c->gkey = fm::GraphKey{};
    for (auto &e : c->gev) e = nullptr;
    c->graph_replays = c->graph_captures = 0;
    DeviceGuard g(h->device);
    if (alloc_common(c) != FM_OK) {
        cudaFree(c->d_err);
        delete c;
        return nullptr;
    }
    return c;
}

void free_search_context(fm_index *c) {
    if (!c || !c->borrowed) return;
    DeviceGuard g(c->device);
    cudaFree(c->d_err);
    fm::Scratch *ss[] = {&c->s_qmeta, &c->s_raw, &c->s_spill, &c->s_group, &c->s_scan, &c->s_plain,
                         &c->s_misc};
    for (auto *sc : ss) cudaFree(sc->ptr);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (auto &e : c->gev)
        if (e) cudaEventDestroy(e);
    delete c;
}

namespace {

// the context's L2 fetch granularity, when the tuning asks for one
void apply_l2(fm_index *h) {
    if (h->tune.l2_fetch) {
        size_t cur = 0;
        cudaDeviceGetLimit(&cur, cudaLimitMaxL2FetchGranularity);
        if (cur != h->tune.l2_fetch) cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, h->tune.l2_fetch);
        cudaGetLastError();
    }
}

// reads the error word of a slot after synchronising the stream, and clears it
int take_err(fm_index *h, ErrSlot slot, cudaStream_t st, uint32_t *out) {
    FM_CUDA_TRY(h, cudaMemcpyAsync(out, h->d_err + slot, 4, cudaMemcpyDeviceToHost, st));
    FM_CUDA_TRY(h, cudaStreamSynchronize(st));
    return FM_OK;
}

int check_handle(const fm_index *h) {
    if (!h) return set_global_error(FM_EINVAL, "null index handle");
    return FM_OK;
}

}  // namespace
}  // namespace fm

using namespace fm;

extern "C" {

const char *fm_last_error(const fm_index *h) {
    return h ? h->err.c_str() : g_last_error.c_str();
}

int fm_build(const char *ref, uint64_t n, const fm_params *p, fm_index **out) {
    if (!out) return set_global_error(FM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!ref) return set_global_error(FM_EINVAL, "ref is NULL");
    if (n < 1 || n > 2147483646ull)
        return set_global_error(FM_EINVAL, "reference length must be in [1, 2147483646]");
    const bool both = p && (p->flags & FM_BUILD_BOTH_STRANDS);
    if (both && n > 1073741823ull)
        return set_global_error(FM_EINVAL, "with FM_BUILD_BOTH_STRANDS the reference length must be "
                                           "at most 1073741823");
    const uint64_t nt = both ? 2 * n : n;   // indexed text length
    uint32_t I = p && p->interval ? p->interval : 64;
    if (I != 32 && I != 64 && I != 128 && I != 256)
        return set_global_error(FM_EINVAL, "interval must be 32, 64, 128 or 256");
    uint32_t flags = p ? p->flags : 0;
    int dev = -1;
    if (p && p->device >= 0) dev = p->device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return set_global_error(FM_ECUDA, "no CUDA device");
    }
    DeviceGuard guard(dev);
    fm_index *h = new fm_index();
    h->device = dev;
    h->sms = device_sms(dev);
    h->n = nt;
    h->both_strands = both;
    h->interval = I;
    h->bbytes = block_bytes(I);
    h->n_blocks = (nt + 1) / I + 1;
    int rc = alloc_common(h);
    cudaStream_t st = nullptr;
    uint8_t *d_text = nullptr;
    uint32_t errw = 0;
    if (!rc && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        rc = cuda_status(h, cudaGetLastError(), "cudaStreamCreate");
    if (!rc) {
        cudaError_t e = cudaMalloc((void **)&d_text, nt);
        if (e != cudaSuccess) rc = cuda_status(h, e, "cudaMalloc(text)");
    }
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(d_text, ref, n, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) rc = cuda_status(h, e, "cudaMemcpy(text)");
    }
    if (!rc) {
        int grid = h->sms * 8;
        k_encode<<<grid, 256, 0, st>>>(d_text, n, (flags & FM_BUILD_CODES) ? 0 : 1,
                                       h->d_err + kErrBuild);
        rc = take_err(h, kErrBuild, st, &errw);
        if (!rc && errw) rc = set_error(h, FM_EINVAL, (flags & FM_BUILD_CODES)
                                                           ? "reference holds a code above 3"
                                                           : "reference holds a symbol outside ACGTacgt");
    }
    if (!rc && both) {
        k_append_revcomp<<<h->sms * 8, 256, 0, st>>>(d_text, n);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_status(h, e, "k_append_revcomp");
    }
    if (!rc) rc = build_index(h, d_text, nt, false, &h->d_fwd, &h->dollar, h->C, &h->d_sa_sample, st);
    if (!rc) h->n_sa_sample = (nt + 1 + h->sa_rate - 1) / h->sa_rate;
    if (!rc && !(flags & FM_BUILD_FORWARD_ONLY)) {
        uint64_t Crev[5];
        rc = build_index(h, d_text, nt, true, &h->d_rev, &h->rev_dollar, Crev, nullptr, st);
        if (!rc) {
            h->has_rev = true;
            for (int b = 0; b < 5; ++b)
                if (Crev[b] != h->C[b]) rc = set_error(h, FM_ECUDA, "reverse index C differs");
        }
    }
    if (d_text) cudaFree(d_text);
    if (st) cudaStreamDestroy(st);
    if (rc) {
        set_global_error(rc, h->err);
        release(h);
        return rc;
    }
    *out = h;
    return FM_OK;
}

void fm_free(fm_index *h) { release(h); }

int fm_info(const fm_index *h, fm_info_t *out) {
    if (int rc = check_handle(h)) return rc;
    if (!out) return set_global_error(FM_EINVAL, "out is NULL");
    memset(out, 0, sizeof(*out));
    out->n = h->n;
    out->interval = h->interval;
    out->block_bytes = h->bbytes;
    for (int b = 0; b < 5; ++b) out->C[b] = h->C[b];
    out->dollar_row = h->dollar;
    out->rev_dollar_row = h->rev_dollar;
    out->n_blocks = h->n_blocks;
    out->sa_sample_rate = h->sa_rate;
    out->bytes_device = h->n_blocks * h->bbytes * (h->has_rev ? 2 : 1) + h->n_sa_sample * 4;
    if (h->kt_depth)   // forward tables, and the reverse index's own with it
        out->bytes_device += (h->d_kt_rev ? 2 : 1) * (2ull << (2 * h->kt_depth)) * (8 + 1.0 / 8);
    if (h->pairs_built)   // forward pair table, and the reverse index's own with it
        out->bytes_device += (h->d_prec_rev ? 2 : 1) * (((h->n + 1) / fm::kPairRows + 1) * 16 * 8 + 64);
    out->has_reverse = h->has_rev ? 1 : 0;
    out->both_strands = h->both_strands ? 1 : 0;
    out->device = h->device;
    return FM_OK;
}

int fm_get_bwt(const fm_index *h_, int rev, uint8_t *bwt) {
    fm_index *h = const_cast<fm_index *>(h_);
    if (int rc = check_handle(h)) return rc;
    if (!bwt) return set_error(h, FM_EINVAL, "bwt is NULL");
    if (rev && !h->has_rev) return set_error(h, FM_EINVAL, "no reverse index");
    DeviceGuard g(h->device);
    std::vector<uint8_t> blk(h->n_blocks * h->bbytes);
    FM_CUDA_TRY(h, cudaMemcpy(blk.data(), rev ? h->d_rev : h->d_fwd, blk.size(), cudaMemcpyDeviceToHost));
    const uint64_t N = h->n + 1;
    const uint64_t drow = rev ? h->rev_dollar : h->dollar;
    for (uint64_t r = 0; r < N; ++r) {
        uint64_t j = r / h->interval, t = r % h->interval;
        const uint64_t *w = reinterpret_cast<const uint64_t *>(blk.data() + j * h->bbytes + 16);
        bwt[r] = (uint8_t)((w[t / 32] >> (2 * (t % 32))) & 3u);
    }
    bwt[drow] = 4;
    return FM_OK;
}

int fm_save(const fm_index *h_, const char *path) {
    fm_index *h = const_cast<fm_index *>(h_);
    if (int rc = check_handle(h)) return rc;
    if (!path) return set_error(h, FM_EINVAL, "path is NULL");
    DeviceGuard g(h->device);
    FILE *f = fopen(path, "wb");
    if (!f) return set_error(h, FM_EIO, std::string("cannot open ") + path);
    FileHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, kMagic, 8);
    hd.n = h->n;
    hd.interval = h->interval;
    hd.bbytes = h->bbytes;
    hd.n_blocks = h->n_blocks;
    for (int b = 0; b < 5; ++b) hd.C[b] = h->C[b];
    hd.dollar = h->dollar;
    hd.rev_dollar = h->rev_dollar;
    hd.has_rev = h->has_rev;
    hd.both_strands = h->both_strands ? 1u : 0u;
    hd.sa_rate = h->sa_rate;
    hd.n_sa = h->n_sa_sample;
    uint64_t sum = fnv1a(kFnvSeed, &hd, sizeof(hd));
    bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1;
    const size_t chunk = (size_t)256 << 20;
    std::vector<uint8_t> buf;
    auto dump = [&](const void *dptr, size_t bytes) {
        for (size_t o = 0; ok && o < bytes; o += chunk) {
            size_t b = bytes - o < chunk ? bytes - o : chunk;
            buf.resize(b);
            if (cudaMemcpy(buf.data(), (const char *)dptr + o, b, cudaMemcpyDeviceToHost) != cudaSuccess) {
                cudaGetLastError();
                ok = false;
                break;
            }
            sum = fnv1a(sum, buf.data(), b);
            ok = fwrite(buf.data(), 1, b, f) == b;
        }
    };
    dump(h->d_fwd, h->n_blocks * h->bbytes);
    if (h->has_rev) dump(h->d_rev, h->n_blocks * h->bbytes);
    dump(h->d_sa_sample, h->n_sa_sample * 4);
    if (ok) ok = fwrite(&sum, 8, 1, f) == 1;
    if (fclose(f) != 0) ok = false;
    if (!ok) return set_error(h, FM_EIO, std::string("write failed: ") + path);
    return FM_OK;
}

int fm_load(const char *path, const fm_params *p, fm_index **out) {
    if (!out || !path) return set_global_error(FM_EINVAL, "null argument");
    *out = nullptr;
    int dev = -1;
    if (p && p->device >= 0) dev = p->device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return set_global_error(FM_ECUDA, "no CUDA device");
    }
    DeviceGuard g(dev);
    FILE *f = fopen(path, "rb");
    if (!f) return set_global_error(FM_EIO, std::string("cannot open ") + path);
    FileHeader hd;
    if (fread(&hd, sizeof(hd), 1, f) != 1 || memcmp(hd.magic, kMagic, 8) != 0 ||
        (hd.interval != 32 && hd.interval != 64 && hd.interval != 128 && hd.interval != 256) ||
        hd.bbytes != block_bytes(hd.interval) || hd.n_blocks != (hd.n + 1) / hd.interval + 1) {
        fclose(f);
        return set_global_error(FM_EIO, "not an fmocc index file");
    }
    fm_index *h = new fm_index();
    h->device = dev;
    h->sms = device_sms(dev);
    h->n = hd.n;
    h->interval = hd.interval;
    h->bbytes = hd.bbytes;
    h->n_blocks = hd.n_blocks;
    for (int b = 0; b < 5; ++b) h->C[b] = hd.C[b];
    h->dollar = hd.dollar;
    h->rev_dollar = hd.rev_dollar;
    h->has_rev = hd.has_rev != 0;
    h->both_strands = hd.both_strands != 0;
    h->sa_rate = hd.sa_rate;
    h->n_sa_sample = hd.n_sa;
    int rc = alloc_common(h);
    uint64_t sum = fnv1a(kFnvSeed, &hd, sizeof(hd));
    const size_t chunk = (size_t)256 << 20;
    std::vector<uint8_t> buf;
    auto fill = [&](uint8_t **dptr, size_t bytes) {
        if (rc) return;
        cudaError_t e = cudaMalloc((void **)dptr, bytes ? bytes : 16);
        if (e != cudaSuccess) {
            rc = cuda_status(h, e, "cudaMalloc(index)");
            return;
        }
        for (size_t o = 0; o < bytes; o += chunk) {
            size_t b = bytes - o < chunk ? bytes - o : chunk;
            buf.resize(b);
            if (fread(buf.data(), 1, b, f) != b) {
                rc = set_error(h, FM_EIO, "truncated index file");
                return;
            }
            sum = fnv1a(sum, buf.data(), b);
            e = cudaMemcpy(*dptr + o, buf.data(), b, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                rc = cuda_status(h, e, "cudaMemcpy(index)");
                return;
            }
        }
    };
    fill(&h->d_fwd, h->n_blocks * h->bbytes);
    if (h->has_rev) fill(&h->d_rev, h->n_blocks * h->bbytes);
    fill((uint8_t **)&h->d_sa_sample, h->n_sa_sample * 4);
    if (!rc) {
        uint64_t stored = 0;
        if (fread(&stored, 8, 1, f) != 1 || stored != sum)
            rc = set_error(h, FM_EIO, "index file checksum mismatch");
    }
    fclose(f);
    if (rc) {
        set_global_error(rc, h->err);
        release(h);
        return rc;
    }
    *out = h;
    return FM_OK;
}

int fm_occ8(fm_index *h, const uint32_t *k, const uint32_t *l, uint32_t *out8, uint64_t N,
            void *stream) {
    if (int rc = check_handle(h)) return rc;
    if (N && (!k || !l || !out8)) return set_error(h, FM_EINVAL, "null buffer");
    DeviceGuard g(h->device);
    apply_l2(h);
    cudaStream_t st = (cudaStream_t)stream;
    FM_CUDA_TRY(h, cudaMemsetAsync(h->d_err + kErrOcc, 0, 4, st));
    if (int rc = launch_occ8(h, k, l, out8, N, st)) return rc;
    uint32_t errw = 0;
    if (int rc = take_err(h, kErrOcc, st, &errw)) return rc;
    if (errw & kErrDomain) return set_error(h, FM_EINVAL, "a query is outside 0<=k<=n+1, 0<=l<=n");
    return FM_OK;
}

int fm_exact(fm_index *h, const uint8_t *reads, const uint32_t *offs, uint32_t n_reads,
             uint32_t *k_out, uint32_t *l_out, void *stream) {
    if (int rc = check_handle(h)) return rc;
    if (n_reads && (!reads || !offs || !k_out || !l_out)) return set_error(h, FM_EINVAL, "null buffer");
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    FM_CUDA_TRY(h, cudaMemsetAsync(h->d_err + kErrExact, 0, 4, st));
    if (int rc = launch_exact(h, reads, offs, n_reads, k_out, l_out, st)) return rc;
    uint32_t errw = 0;
    if (int rc = take_err(h, kErrExact, st, &errw)) return rc;
    if (errw) return set_error(h, FM_EINVAL, "a read holds a code above 3");
    return FM_OK;
}

int fm_locate(fm_index *h, const uint32_t *rows, uint64_t N, uint32_t *pos_out, uint64_t *steps,
              void *stream) {
    if (int rc = check_handle(h)) return rc;
    if (N && (!rows || !pos_out)) return set_error(h, FM_EINVAL, "null buffer");
    if (!h->d_sa_sample) return set_error(h, FM_EINVAL, "index holds no SA samples");
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    FM_CUDA_TRY(h, cudaMemsetAsync(h->d_err + kErrExact, 0, 4, st));
    if (int rc = launch_locate(h, rows, N, pos_out, (unsigned long long *)steps, st)) return rc;
    uint32_t errw = 0;
    if (int rc = take_err(h, kErrExact, st, &errw)) return rc;
    if (errw) return set_error(h, FM_EINVAL, "a row is above n");
    return FM_OK;
}

int fm_dcalc(fm_index *h, const uint8_t *reads, const uint32_t *offs, uint32_t n_reads,
             uint32_t strands, uint8_t *D_out, void *stream) {
    if (int rc = check_handle(h)) return rc;
    if (!h->has_rev) return set_error(h, FM_EINVAL, "index built without reverse(R)");
    if (strands != 1 && strands != 2) return set_error(h, FM_EINVAL, "strands must be 1 or 2");
    if (n_reads && (!reads || !offs || !D_out)) return set_error(h, FM_EINVAL, "null buffer");
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    FM_CUDA_TRY(h, cudaMemsetAsync(h->d_err + kErrDcalc, 0, 4, st));
    if (int rc = launch_dcalc(h, reads, offs, n_reads, strands, nullptr, D_out, st)) return rc;
    uint32_t errw = 0;
    if (int rc = take_err(h, kErrDcalc, st, &errw)) return rc;
    if (errw & kErrReadLen) return set_error(h, FM_EINVAL, "a read is longer than 255 symbols");
    if (errw) return set_error(h, FM_EINVAL, "a read holds a code above 3");
    return FM_OK;
}

int fm_inexact(fm_index *h, const uint8_t *reads, const uint32_t *offs, uint32_t n_reads,
               const fm_search_params *sp, uint32_t *counts, uint64_t *offsets, uint32_t *pairs,
               uint64_t pair_capacity, uint64_t *pairs_needed, void *stream) {
    if (int rc = check_handle(h)) return rc;
    if (!sp) return set_error(h, FM_EINVAL, "search params are NULL");
    if (!h->has_rev) return set_error(h, FM_EINVAL, "index built without reverse(R)");
    if (sp->z > (uint32_t)kMaxZ) return set_error(h, FM_EINVAL, "z must be at most 7");
    if (sp->max_gaps > (uint32_t)kMaxGaps) return set_error(h, FM_EINVAL, "max_gaps must be at most 7");
    if (sp->strands != 1 && sp->strands != 2) return set_error(h, FM_EINVAL, "strands must be 1 or 2");
    if (sp->kernel > FM_KERNEL_PERSISTENT) return set_error(h, FM_EINVAL, "unknown kernel");
    if (sp->best > 1) return set_error(h, FM_EINVAL, "best must be 0 or 1");
    if (sp->indel_end_skip > 255) return set_error(h, FM_EINVAL, "indel_end_skip must be at most 255");
    if (!offsets || (n_reads && (!reads || !offs || !counts))) return set_error(h, FM_EINVAL, "null buffer");
    if (pair_capacity && !pairs) return set_error(h, FM_EINVAL, "pairs is NULL");
    DeviceGuard g(h->device);
    apply_l2(h);
    cudaStream_t st = (cudaStream_t)stream;
    FM_CUDA_TRY(h, cudaMemsetAsync(h->d_err + kErrDcalc, 0, 8, st));   // dcalc and search words
    return run_inexact(h, reads, offs, n_reads, sp, counts, offsets, pairs, pair_capacity,
                       pairs_needed, st);
}

int fm_inexact_fetch(fm_index *h, uint32_t *pairs, uint64_t pair_capacity, void *stream) {
    if (int rc = check_handle(h)) return rc;
    DeviceGuard g(h->device);
    return fetch_inexact(h, pairs, pair_capacity, (cudaStream_t)stream);
}

int fm_set_tuning(fm_index *h, const fm_tuning *t) {
    if (int rc = check_handle(h)) return rc;
    if (!t) return set_error(h, FM_EINVAL, "tuning is NULL");
    // every value is checked before any is applied: a rejected call changes nothing
    if (t->warps_per_block > 8 || t->chunk > 32 || (t->plain_block && (t->plain_block % 32 || t->plain_block > 256)))
        return set_error(h, FM_EINVAL, "tuning value out of range");
    if (t->graphs > 2) return set_error(h, FM_EINVAL, "graphs must be 0, 1 or 2");
    if (t->occ_per_thread && t->occ_per_thread != 1 && t->occ_per_thread != 2 && t->occ_per_thread != 4)
        return set_error(h, FM_EINVAL, "occ_per_thread must be 1, 2 or 4");
    if (t->l2_fetch_bytes && t->l2_fetch_bytes != 32 && t->l2_fetch_bytes != 64 && t->l2_fetch_bytes != 128)
        return set_error(h, FM_EINVAL, "l2_fetch_bytes must be 32, 64 or 128");
    if (t->canonical > 2) return set_error(h, FM_EINVAL, "canonical must be 0, 1 or 2");
    if (t->pair_steps > 2) return set_error(h, FM_EINVAL, "pair_steps must be 0, 1 or 2");
    if (t->kmer_depth > fm::kMaxKmerDepth && t->kmer_depth != FM_KMER_AUTO && t->kmer_depth != FM_KMER_OFF)
        return set_error(h, FM_EINVAL, "kmer_depth must be 0, 1..15, FM_KMER_AUTO or FM_KMER_OFF");
    if (t->refill > 288) return set_error(h, FM_EINVAL, "refill must be 0..288");
    if (t->chain2_min > 32) return set_error(h, FM_EINVAL, "chain2_min must be 0..32");
    if (t->stage > 2) return set_error(h, FM_EINVAL, "stage must be 0, 1 or 2");
    if (t->warps_per_block) h->tune.warps_per_block = t->warps_per_block;
    if (t->blocks_per_sm) h->tune.blocks_per_sm = t->blocks_per_sm;
    if (t->chunk) h->tune.chunk = t->chunk;
    if (t->plain_block) h->tune.plain_block = t->plain_block;
    if (t->occ_per_thread) h->tune.occ_q = t->occ_per_thread;
    if (t->l2_fetch_bytes) h->tune.l2_fetch = t->l2_fetch_bytes;
    if (t->canonical) h->tune.canon = t->canonical == 1 ? 1u : 0u;
    if (t->kmer_depth) h->tune.kmer = t->kmer_depth;
    if (t->pair_steps) h->tune.pairs = t->pair_steps == 1 ? 1u : 0u;
    if (t->graphs) h->use_graphs = t->graphs == 1;
    if (t->refill) h->tune.refill = t->refill;
    if (t->chain2_min) h->tune.chain2_min = t->chain2_min;
    if (t->stage) h->tune.stage = t->stage == 1 ? 1u : 0u;
    return FM_OK;
}

int fm_get_tuning(const fm_index *h, fm_tuning *t) {
    if (int rc = check_handle(h)) return rc;
    if (!t) return FM_EINVAL;
    t->warps_per_block = h->tune.warps_per_block;
    t->blocks_per_sm = h->tune.blocks_per_sm;
    t->chunk = h->tune.chunk;
    t->plain_block = h->tune.plain_block;
    t->graphs = h->use_graphs ? 1u : 2u;
    t->occ_per_thread = h->tune.occ_q;
    t->l2_fetch_bytes = h->tune.l2_fetch;
    t->canonical = h->tune.canon ? 1u : 2u;
    const uint32_t kd = fm::kmer_depth_for(h);
    t->kmer_depth = kd ? kd : FM_KMER_OFF;
    t->pair_steps = h->tune.pairs ? 1u : 2u;
    t->refill = h->tune.refill;
    t->chain2_min = h->tune.chain2_min;
    t->stage = h->tune.stage ? 1u : 2u;
    return FM_OK;
}

}  // extern "C"
