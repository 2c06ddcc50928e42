// The C ABI of librb3 (declared in include/rb3.h): argument checks, host/device
// pointer handling, index lifetime, export / save / load, profiling and errors.
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>

#include <algorithm>

#include "common.cuh"
#include "wait.cuh"

namespace rb3 {

std::atomic<int64_t> g_launches{0};

static thread_local std::string g_err;

void set_error(const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

std::string rb3_last_error_str() { return g_err; }

int cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    cudaGetLastError();  // clear a sticky-free error so later calls start clean
    set_error("CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
    return e == cudaErrorMemoryAllocation ? RB3_E_NOMEM : RB3_E_CUDA;
}

static void ensure_pool() {
    static const bool done = [] {  // thread-safe one-time initialisation
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return false;
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            // keep up to 64 GiB of freed scratch in the pool between calls
            uint64_t thr = 64ull << 30;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
            // never make a stream wait for another stream's frees to reuse memory:
            // builds and merges run on separate streams and must not be serialised
            int no = 0;
            cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
        }
        return true;
    }();
    (void)done;
}

int dev_alloc(void **p, size_t bytes, cudaStream_t st) {
    ensure_pool();
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? RB3_E_NOMEM : RB3_E_CUDA;
    }
    return RB3_OK;
}

void dev_free(void *p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

int wait_stream_blocking(cudaStream_t st) {
    thread_local cudaEvent_t ev = nullptr;  // released with the context
    if (!ev) RB3_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventBlockingSync | cudaEventDisableTiming));
    RB3_CUDA_TRY(cudaEventRecord(ev, st));
    RB3_CUDA_TRY(cudaEventSynchronize(ev));
    return RB3_OK;
}

int DevBuf::alloc(size_t nbytes, cudaStream_t s) {
    release();
    st = s;
    int r = dev_alloc(&p, nbytes, s);
    if (r == RB3_OK) bytes = nbytes;
    return r;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---- profiling ---------------------------------------------------------------
static std::atomic<bool> g_prof{false};
static std::mutex g_prof_mu;
struct Pending {
    const char *name;
    cudaEvent_t a, b;
    double bytes;
};
struct Acc {
    double ms = 0.0, bytes = 0.0;
    int64_t calls = 0;
};
static std::vector<Pending> g_pending;
static std::map<std::string, Acc> g_acc;
static std::vector<std::string> g_names;  // stable storage for names handed out
// Timeline: every drained phase with its start relative to the origin event
// recorded by rb3_profile_reset (events of any stream of the device compare).
struct Span {
    const char *name;
    float start, dur;
};
static std::vector<Span> g_spans;
static cudaEvent_t g_origin = nullptr;

bool profile_on() { return g_prof.load(std::memory_order_relaxed); }

void profile_push(const char *name, cudaEvent_t a, cudaEvent_t b, double bytes) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_pending.push_back({name, a, b, bytes});
}

static void profile_drain() {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &p : g_pending) {
        float ms = 0.f, t0 = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            Acc &e = g_acc[p.name];
            e.ms += ms;
            e.bytes += p.bytes;
            e.calls += 1;
            if (g_origin && cudaEventElapsedTime(&t0, g_origin, p.a) == cudaSuccess) g_spans.push_back({p.name, t0, ms});
        }
        cudaGetLastError();
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    g_pending.clear();
}

// ---- index utilities ----------------------------------------------------------
__global__ void k_counts_at_n(OccView V, int64_t *__restrict__ out) {
    int64_t r[SIGMA];
    rank_all_any(V, V.n, r);
    for (int a = 0; a < SIGMA; ++a) out[a] = r[a];
}

int finalize_counts(rb3_index *x, cudaStream_t st) {
    DevBuf b;
    RB3_TRY(b.alloc(sizeof(int64_t) * SIGMA, st));
    RB3_LAUNCH(k_counts_at_n, 1, 1, 0, st, occ_view(x), b.as<int64_t>());
    int64_t h[SIGMA];
    RB3_CUDA_TRY(cudaMemcpyAsync(h, b.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    x->C[0] = 0;
    for (int a = 0; a < SIGMA; ++a) x->C[a + 1] = x->C[a] + h[a];
    if (x->C[SIGMA] != x->n || h[0] != x->m) {
        set_error("index counts inconsistent: sum %lld n %lld, sentinels %lld m %lld", (long long)x->C[SIGMA],
                  (long long)x->n, (long long)h[0], (long long)x->m);
        return RB3_E_CUDA;
    }
    return RB3_OK;
}

// one thread per 8 symbols
__global__ void k_unpack(OccView V, uint8_t *__restrict__ codes) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t q0 = t * 8;
    if (q0 >= V.n) return;
    const uint8_t *blk = V.blocks + (q0 >> V.log2D) * (int64_t)V.bb;
    int o = (int)(q0 & ((1 << V.log2D) - 1));
    uint32_t p0 = blk[plane_byte(o, 0, V.log2D)], p1 = blk[plane_byte(o, 1, V.log2D)],
             p2 = blk[plane_byte(o, 2, V.log2D)];
    for (int j = 0; j < 8 && q0 + j < V.n; ++j)
        codes[q0 + j] = (uint8_t)(((p0 >> j) & 1u) | (((p1 >> j) & 1u) << 1) | (((p2 >> j) & 1u) << 2));
}

__global__ void k_occ_export(OccView V, int64_t nblocks, int64_t *__restrict__ occ) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    const uint8_t *h = V.blocks + b * (int64_t)V.bb;
    if (V.log2D == 5) {  // D = 32: the rank at the block start (offset 0)
        int64_t r[SIGMA];
        rank_all<0>(V, b * 32, r);
        for (int a = 0; a < SIGMA; ++a) occ[b * SIGMA + a] = r[a];
        return;
    }
    for (int a = 0; a < SIGMA; ++a)
        occ[b * SIGMA + a] = (int64_t)(*reinterpret_cast<const uint32_t *>(h + 4 * a)) | ((int64_t)h[24 + a] << 32);
}

int export_impl(const rb3_index *x, uint8_t *codes, int64_t *occ, cudaStream_t st) {
    if (x->rle) return rle_export_impl(x, codes, occ, st);
    OccView V = occ_view(x);
    if (codes && x->n > 0) {
        int64_t th = (x->n + 7) / 8;
        RB3_LAUNCH(k_unpack, (unsigned)((th + 255) / 256), 256, 0, st, V, codes);
    }
    if (occ) RB3_LAUNCH(k_occ_export, (unsigned)((x->nblocks + 255) / 256), 256, 0, st, V, x->nblocks, occ);
    return RB3_OK;
}

static int make_empty(const rb3_opts *o, cudaStream_t st, rb3_index **out) {
    int D = (o && o->occ_interval) ? o->occ_interval : kDefaultOccInterval;
    RB3_CHECK_ARG(valid_occ_interval(D), "occ_interval must be 32, 64, 128 or 256");
    rb3_index *x = new rb3_index();
    x->D = D;
    x->log2D = ilog2(D);
    x->block_bytes = block_bytes_for(D);
    x->single_strand = (o && o->single_strand) ? 1 : 0;
    x->nblocks = 1;
    cudaGetDevice(&x->device);
    int r = dev_alloc((void **)&x->blocks, x->block_bytes, st);
    if (r != RB3_OK) {
        delete x;
        return r;
    }
    cudaError_t e = cudaMemsetAsync(x->blocks, 0, x->block_bytes, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        dev_free(x->blocks, st);
        delete x;
        return cuda_fail(e, "make_empty", __FILE__, __LINE__);
    }
    *out = x;
    return RB3_OK;
}

static void free_index(rb3_index *x) {
    if (!x) return;
    cudaStream_t st = 0;
    dev_free(x->blocks, st);
    dev_free(x->gbase, st);
    dev_free(x->payload, st);
    dev_free(x->text, st);
    dev_free(x->isa, st);
    free_samples(x);
    cudaStreamSynchronize(st);
    free_hot(x);
    delete x;
}

// Copies a caller array to the device when it is host memory.
struct InArg {
    const void *dev = nullptr;
    DevBuf buf;
    int set(const void *p, size_t bytes, cudaStream_t st) {
        if (is_device_ptr(p) || bytes == 0) {
            dev = p;
            return RB3_OK;
        }
        RB3_TRY(buf.alloc(bytes, st));
        RB3_CUDA_TRY(cudaMemcpyAsync(buf.p, p, bytes, cudaMemcpyHostToDevice, st));
        dev = buf.p;
        return RB3_OK;
    }
};

static int read_i64(const int64_t *p, int64_t n, std::vector<int64_t> &v, cudaStream_t st) {
    v.resize(n);
    if (n == 0) return RB3_OK;
    if (is_device_ptr(p)) {
        RB3_CUDA_TRY(cudaMemcpyAsync(v.data(), p, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, st));
        RB3_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
        memcpy(v.data(), p, sizeof(int64_t) * n);
    }
    return RB3_OK;
}

static int check_qoff(const std::vector<int64_t> &qo) {
    if (qo.empty()) return RB3_OK;
    RB3_CHECK_ARG(qo[0] >= 0, "qoff[0] < 0");
    for (size_t i = 1; i < qo.size(); ++i) RB3_CHECK_ARG(qo[i] >= qo[i - 1], "qoff must be non-decreasing");
    return RB3_OK;
}

}  // namespace rb3

using namespace rb3;

// ---------------------------------------------------------------------------
RB3_EXPORT int rb3_walk_stats(int64_t *out, int32_t reset) {
    g_err.clear();
    RB3_CHECK_ARG(out != nullptr, "NULL argument");
    return walk_stats(out, reset != 0);
}

RB3_EXPORT int rb3_search_stats(int64_t *out, int32_t reset) {
    g_err.clear();
    RB3_CHECK_ARG(out != nullptr, "NULL argument");
    return search_stats(out, reset != 0);
}

RB3_EXPORT int rb3_selftest_wait(int32_t limit, void *stream) {
    g_err.clear();
    RB3_CHECK_ARG(limit >= 1 && limit <= (1 << 20), "limit must be in [1, 2^20]");
    return wait_selftest(limit, (cudaStream_t)stream);
}

RB3_EXPORT int rb3_device_peak(int64_t *used_high, int32_t reset) {
    g_err.clear();
    RB3_CHECK_ARG(used_high != nullptr, "NULL argument");
    ensure_pool();
    int dev = 0;
    RB3_CUDA_TRY(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    RB3_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t v = 0;
    if (reset) {
        uint64_t zero = 0;  // resets the mark to the memory in use now, which is returned
        RB3_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
        RB3_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v));
    } else {
        RB3_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &v));
    }
    *used_high = (int64_t)v;
    return RB3_OK;
}

RB3_EXPORT void rb3_opts_default(rb3_opts *o) {
    if (o) memset(o, 0, sizeof(*o));
}

RB3_EXPORT const char *rb3_last_error(void) { return g_err.c_str(); }

RB3_EXPORT int rb3_build_batch(const uint8_t *seq, const int64_t *len, int64_t n_seq, const rb3_opts *o, void *stream,
                               rb3_index **out) {
    g_err.clear();
    RB3_CHECK_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    RB3_CHECK_ARG(n_seq >= 0, "n_seq < 0");
    RB3_CHECK_ARG(n_seq == 0 || len != nullptr, "len is NULL");
    rb3_opts opts;
    rb3_opts_default(&opts);
    if (o) opts = *o;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int64_t> lens;
    RB3_TRY(read_i64(len, n_seq, lens, st));
    int64_t total = 0;
    for (int64_t i = 0; i < n_seq; ++i) {
        RB3_CHECK_ARG(lens[i] >= 0, "negative string length");
        total += lens[i];
    }
    RB3_CHECK_ARG(total == 0 || seq != nullptr, "seq is NULL");
    InArg s;
    RB3_TRY(s.set(seq, (size_t)total, st));
    rb3_index *x = new rb3_index();
    cudaGetDevice(&x->device);
    int r = build_batch_impl(static_cast<const uint8_t *>(s.dev), lens.data(), n_seq, opts, st, x);
    if (r == RB3_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) r = cuda_fail(e, "rb3_build_batch", __FILE__, __LINE__);
    }
    if (r != RB3_OK) {
        free_index(x);
        return r;
    }
    *out = x;
    return RB3_OK;
}

RB3_EXPORT int rb3_index_empty(const rb3_opts *o, rb3_index **out) {
    g_err.clear();
    RB3_CHECK_ARG(out != nullptr, "out is NULL");
    return make_empty(o, 0, out);
}

RB3_EXPORT int rb3_merge_opts(rb3_index *dst, const rb3_index *src, const rb3_opts *o, void *stream) {
    g_err.clear();
    RB3_CHECK_ARG(dst && src, "NULL index");
    rb3_opts opts;
    rb3_opts_default(&opts);
    if (o) opts = *o;
    cudaStream_t st = (cudaStream_t)stream;
    RB3_TRY(merge_any(dst, src, opts, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    return RB3_OK;
}

RB3_EXPORT int rb3_merge(rb3_index *dst, const rb3_index *src, void *stream) {
    return rb3_merge_opts(dst, src, nullptr, stream);
}

// Longest string first, each to the part with the fewest symbols so far
// (ties: the lower part); host only.
RB3_EXPORT int rb3_merge_partition(const int64_t *len, int64_t n_seq, int32_t parts, int32_t *owner) {
    g_err.clear();
    RB3_CHECK_ARG(n_seq >= 0 && parts >= 1, "n_seq < 0 or parts < 1");
    if (n_seq == 0) return RB3_OK;
    RB3_CHECK_ARG(len && owner, "NULL argument");
    for (int64_t i = 0; i < n_seq; ++i) RB3_CHECK_ARG(len[i] >= 0, "negative length");
    std::vector<int64_t> ord(n_seq);
    for (int64_t i = 0; i < n_seq; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return len[a] > len[b]; });
    std::vector<int64_t> load(parts, 0);
    for (int64_t i : ord) {
        int32_t best = 0;
        for (int32_t p = 1; p < parts; ++p)
            if (load[p] < load[best]) best = p;
        owner[i] = best;
        load[best] += len[i] + 1;
    }
    return RB3_OK;
}

RB3_EXPORT int rb3_merge_positions(const rb3_index *dst, const rb3_index *src, const rb3_opts *o,
                                   const int32_t *owner, int32_t part, int64_t *pos, void *stream) {
    g_err.clear();
    RB3_CHECK_ARG(dst && src, "NULL index");
    RB3_CHECK_ARG(dst != src, "dst and src must differ");
    RB3_CHECK_ARG(!src->rle, "the batch merged in must be a plain index");
    RB3_CHECK_ARG(dst->single_strand == src->single_strand || dst->n == 0,
                  "cannot merge a single-strand index with a double-strand one");
    if (src->n == 0) return RB3_OK;
    RB3_CHECK_ARG(pos != nullptr && is_device_ptr(pos), "pos must be a device pointer");
    rb3_opts opts;
    rb3_opts_default(&opts);
    if (o) opts = *o;
    cudaStream_t st = (cudaStream_t)stream;
    RB3_TRY(merge_positions(dst, src, opts, st, pos, nullptr, owner, part));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    return RB3_OK;
}

RB3_EXPORT int rb3_merge_apply(rb3_index *dst, const rb3_index *src, const int64_t *pos, void *stream) {
    g_err.clear();
    RB3_CHECK_ARG(dst && src, "NULL index");
    if (src->n == 0) return merge_apply(dst, src, nullptr, nullptr, (cudaStream_t)stream);
    RB3_CHECK_ARG(pos != nullptr, "NULL pos");
    cudaStream_t st = (cudaStream_t)stream;
    InArg dp;
    RB3_TRY(dp.set(pos, sizeof(int64_t) * src->n, st));
    RB3_TRY(merge_apply(dst, src, static_cast<const int64_t *>(dp.dev), nullptr, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    return RB3_OK;
}

RB3_EXPORT int rb3_backward_search(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, int64_t nq,
                                   int64_t *lo_hi, void *stream) {
    g_err.clear();
    RB3_CHECK_ARG(idx != nullptr, "NULL index");
    RB3_CHECK_ARG(nq >= 0, "nq < 0");
    if (nq == 0) return RB3_OK;
    RB3_CHECK_ARG(qoff && lo_hi, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int64_t> qo;
    RB3_TRY(read_i64(qoff, nq + 1, qo, st));
    RB3_TRY(check_qoff(qo));
    RB3_CHECK_ARG(qo[nq] == 0 || q != nullptr, "q is NULL");
    InArg dq, doff;
    RB3_TRY(dq.set(q, (size_t)qo[nq], st));
    RB3_TRY(doff.set(qoff, sizeof(int64_t) * (nq + 1), st));
    bool dev_out = is_device_ptr(lo_hi);
    DevBuf ob;
    int64_t *o = lo_hi;
    if (!dev_out) {
        RB3_TRY(ob.alloc(sizeof(int64_t) * 2 * nq, st));
        o = ob.as<int64_t>();
    }
    RB3_TRY(backward_search_impl(idx, static_cast<const uint8_t *>(dq.dev), static_cast<const int64_t *>(doff.dev), nq,
                                 qo[nq], o, st));
    if (!dev_out) RB3_CUDA_TRY(cudaMemcpyAsync(lo_hi, o, sizeof(int64_t) * 2 * nq, cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    return RB3_OK;
}

RB3_EXPORT int rb3_bwasw(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, int64_t nq, int32_t a,
                         int32_t b, int32_t gap_open, int32_t gap_ext, int32_t W, int64_t *out, int64_t cap,
                         int64_t *n_out, void *stream) {
    g_err.clear();
    RB3_CHECK_ARG(idx != nullptr && n_out != nullptr, "NULL argument");
    *n_out = 0;
    RB3_CHECK_ARG(nq >= 0 && cap >= 0, "negative size");
    RB3_CHECK_ARG(!idx->single_strand, "BWA-SW needs a double-strand index");
    RB3_CHECK_ARG(a >= 1 && b >= 0 && gap_open >= 0 && gap_ext >= 1, "scores: a >= 1, b >= 0, q >= 0, e >= 1");
    RB3_CHECK_ARG(a <= 65536 && b <= 65536 && gap_open <= 65536 && gap_ext <= 65536, "a score above 65536");
    RB3_CHECK_ARG(W >= 1 && W <= 32, "W must be in 1..32");
    if (nq == 0) return RB3_OK;
    RB3_CHECK_ARG(qoff != nullptr && (cap == 0 || out != nullptr), "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int64_t> qo;
    RB3_TRY(read_i64(qoff, nq + 1, qo, st));
    RB3_TRY(check_qoff(qo));
    RB3_CHECK_ARG(qo[nq] == qo[0] || q != nullptr, "q is NULL");
    for (int64_t i = 0; i < nq; ++i) RB3_CHECK_ARG(qo[i + 1] - qo[i] <= 2047, "BWA-SW queries are at most 2047 bases");
    InArg dq, doff;
    RB3_TRY(dq.set(q, (size_t)qo[nq], st));
    RB3_TRY(doff.set(qoff, sizeof(int64_t) * (nq + 1), st));
    const bool dev_out = cap == 0 || is_device_ptr(out);
    DevBuf ob;
    int64_t *o = out;
    if (!dev_out) {
        RB3_TRY(ob.alloc(sizeof(int64_t) * 7 * (size_t)cap, st));
        o = ob.as<int64_t>();
    }
    const int32_t prm[5] = {a, b, gap_open, gap_ext, W};
    const int r = bwasw_impl(idx, static_cast<const uint8_t *>(dq.dev), static_cast<const int64_t *>(doff.dev), qo, nq,
                             prm, o, cap, n_out, st);
    if (r != RB3_OK) return r;
    if (!dev_out && *n_out > 0)
        RB3_CUDA_TRY(cudaMemcpyAsync(out, o, sizeof(int64_t) * 7 * (size_t)*n_out, cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    return RB3_OK;
}

RB3_EXPORT int rb3_haplotype_diversity(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, int64_t nq,
                                       int32_t a, int32_t b, int32_t gap_open, int32_t gap_ext, int32_t W,
                                       int32_t redundancy, int64_t *out, int64_t *n_out, void *stream) {
    g_err.clear();
    RB3_CHECK_ARG(idx != nullptr, "NULL index");
    RB3_CHECK_ARG(nq >= 0, "nq < 0");
    RB3_CHECK_ARG(!idx->single_strand, "haplotype diversity needs a double-strand index");
    RB3_CHECK_ARG(a >= 1 && b >= 0 && gap_open >= 0 && gap_ext >= 1, "scores: a >= 1, b >= 0, q >= 0, e >= 1");
    RB3_CHECK_ARG(a <= 65536 && b <= 65536 && gap_open <= 65536 && gap_ext <= 65536, "a score above 65536");
    RB3_CHECK_ARG(W >= 1 && W <= 32, "W must be in 1..32");
    RB3_CHECK_ARG(redundancy == 0 || redundancy == 1, "redundancy must be 0 or 1");
    if (nq == 0) return RB3_OK;
    RB3_CHECK_ARG(qoff && out && n_out, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int64_t> qo;
    RB3_TRY(read_i64(qoff, nq + 1, qo, st));
    RB3_TRY(check_qoff(qo));
    RB3_CHECK_ARG(qo[nq] == 0 || q != nullptr, "q is NULL");
    for (int64_t i = 0; i < nq; ++i) RB3_CHECK_ARG((qo[i + 1] - qo[i]) * (int64_t)a < ((int64_t)1 << 29), "query too long for its match score");
    InArg dq, doff;
    RB3_TRY(dq.set(q, (size_t)qo[nq], st));
    RB3_TRY(doff.set(qoff, sizeof(int64_t) * (nq + 1), st));
    const size_t out_bytes = sizeof(int64_t) * 4 * (size_t)W * nq, n_bytes = sizeof(int64_t) * nq;
    const bool dev_out = is_device_ptr(out), dev_n = is_device_ptr(n_out);
    DevBuf ob, nb;
    int64_t *o = out, *no = n_out;
    if (!dev_out) {
        RB3_TRY(ob.alloc(out_bytes, st));
        o = ob.as<int64_t>();
    }
    if (!dev_n) {
        RB3_TRY(nb.alloc(n_bytes, st));
        no = nb.as<int64_t>();
    }
    const int32_t prm[6] = {a, b, gap_open, gap_ext, W, redundancy};
    RB3_TRY(diversity_impl(idx, static_cast<const uint8_t *>(dq.dev), static_cast<const int64_t *>(doff.dev), nq,
                           qo[nq], prm, o, no, st));
    if (!dev_out) RB3_CUDA_TRY(cudaMemcpyAsync(out, o, out_bytes, cudaMemcpyDeviceToHost, st));
    std::vector<int64_t> counts(nq);
    RB3_CUDA_TRY(cudaMemcpyAsync(counts.data(), no, n_bytes, cudaMemcpyDeviceToHost, st));
    if (!dev_n) RB3_CUDA_TRY(cudaMemcpyAsync(n_out, no, n_bytes, cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < nq; ++i)
        if (counts[i] < 0) {
            set_error("query %lld: a step left more than 65534 candidate cells", (long long)i);
            return RB3_E_CAPACITY;
        }
    return RB3_OK;
}

RB3_EXPORT int rb3_diversity_stats(int64_t *out, int32_t reset) {
    g_err.clear();
    RB3_CHECK_ARG(out != nullptr, "out is NULL");
    RB3_CUDA_TRY(cudaDeviceSynchronize());
    return diversity_stats(out, reset != 0);
}

RB3_EXPORT int rb3_mem_search_opts(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, int64_t nq,
                                   int32_t min_len, int64_t min_occ, const rb3_opts *o, rb3_smem *out, int64_t cap,
                                   int64_t *n_out, void *stream) {
    g_err.clear();
    RB3_CHECK_ARG(idx != nullptr && n_out != nullptr, "NULL argument");
    *n_out = 0;
    RB3_CHECK_ARG(nq >= 0 && cap >= 0, "negative size");
    RB3_CHECK_ARG(min_len >= 1, "min_len must be >= 1");
    RB3_CHECK_ARG(min_occ >= 1, "min_occ must be >= 1");
    RB3_CHECK_ARG(!idx->single_strand, "SMEM search needs a double-strand index");
    if (nq == 0) return RB3_OK;
    RB3_CHECK_ARG(qoff != nullptr, "qoff is NULL");
    RB3_CHECK_ARG(cap == 0 || out != nullptr, "out is NULL");
    rb3_opts opts;
    rb3_opts_default(&opts);
    if (o) opts = *o;
    RB3_CHECK_ARG(opts.hot_depth >= -1 && opts.hot_depth <= HOT_MAX, "hot_depth must be -1..12");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int64_t> qo;
    RB3_TRY(read_i64(qoff, nq + 1, qo, st));
    RB3_TRY(check_qoff(qo));
    for (int64_t i = 0; i < nq; ++i)
        RB3_CHECK_ARG(qo[i + 1] - qo[i] < (int64_t(1) << 31), "query longer than 2^31 - 1");
    RB3_CHECK_ARG(qo[nq] == 0 || q != nullptr, "q is NULL");
    InArg dq, doff;
    RB3_TRY(dq.set(q, (size_t)qo[nq], st));
    RB3_TRY(doff.set(qoff, sizeof(int64_t) * (nq + 1), st));
    bool dev_out = cap == 0 || is_device_ptr(out);
    DevBuf ob;
    rb3_smem *od = out;
    if (!dev_out) {
        RB3_TRY(ob.alloc(sizeof(rb3_smem) * cap, st));
        od = ob.as<rb3_smem>();
    }
    int64_t cnt = 0;
    int r = mem_search_impl(idx, static_cast<const uint8_t *>(dq.dev), static_cast<const int64_t *>(doff.dev),
                            qo.data(), nq, qo[nq], min_len, min_occ, opts, od, cap, &cnt, st);
    *n_out = cnt;
    if (r != RB3_OK) return r;
    if (!dev_out && cnt > 0)
        RB3_CUDA_TRY(cudaMemcpyAsync(out, od, sizeof(rb3_smem) * cnt, cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    return RB3_OK;
}

RB3_EXPORT int rb3_mem_search(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, int64_t nq, int32_t min_len,
                              int64_t min_occ, rb3_smem *out, int64_t cap, int64_t *n_out, void *stream) {
    return rb3_mem_search_opts(idx, q, qoff, nq, min_len, min_occ, nullptr, out, cap, n_out, stream);
}

RB3_EXPORT int rb3_export(const rb3_index *idx, uint8_t *codes, int64_t *occ, void *stream) {
    g_err.clear();
    RB3_CHECK_ARG(idx != nullptr, "NULL index");
    cudaStream_t st = (cudaStream_t)stream;
    bool dc = !codes || is_device_ptr(codes), doc = !occ || is_device_ptr(occ);
    DevBuf cb, obuf;
    uint8_t *c = codes;
    int64_t *oc = occ;
    if (!dc) {
        RB3_TRY(cb.alloc((size_t)idx->n, st));
        c = cb.as<uint8_t>();
    }
    if (!doc) {
        RB3_TRY(obuf.alloc(sizeof(int64_t) * SIGMA * idx->nblocks, st));
        oc = obuf.as<int64_t>();
    }
    RB3_TRY(export_impl(idx, c, oc, st));
    if (!dc && idx->n) RB3_CUDA_TRY(cudaMemcpyAsync(codes, c, (size_t)idx->n, cudaMemcpyDeviceToHost, st));
    if (!doc)
        RB3_CUDA_TRY(cudaMemcpyAsync(occ, oc, sizeof(int64_t) * SIGMA * idx->nblocks, cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    return RB3_OK;
}

RB3_EXPORT int rb3_index_info(const rb3_index *idx, int64_t *n, int64_t *m, int64_t *C, int32_t *occ_interval,
                              int32_t *flags) {
    g_err.clear();
    RB3_CHECK_ARG(idx != nullptr, "NULL index");
    if (n) *n = idx->n;
    if (m) *m = idx->m;
    if (C)
        for (int a = 0; a <= SIGMA; ++a) C[a] = idx->C[a];
    if (occ_interval) *occ_interval = idx->D;
    if (flags)
        *flags = (idx->single_strand ? 1 : 0) | ((idx->text && idx->isa) ? 2 : 0) | (idx->rle ? 4 : 0) |
                 (idx->sa_s << 8);
    return RB3_OK;
}

RB3_EXPORT int rb3_drop_build_data(rb3_index *idx) {
    g_err.clear();
    RB3_CHECK_ARG(idx != nullptr, "NULL index");
    dev_free(idx->text, 0);
    dev_free(idx->isa, 0);
    idx->text = nullptr;
    idx->isa = nullptr;
    idx->str_end.clear();
    RB3_CUDA_TRY(cudaStreamSynchronize(0));
    return RB3_OK;
}

static const char k_magic[8] = {'R', 'B', '3', 'I', 'D', 'X', 0, 1};

RB3_EXPORT int rb3_index_save(const rb3_index *idx, const char *path) {
    g_err.clear();
    RB3_CHECK_ARG(idx && path, "NULL argument");
    size_t bytes = (size_t)idx->nblocks * idx->block_bytes;
    std::vector<uint8_t> host(bytes);
    RB3_CUDA_TRY(cudaMemcpy(host.data(), idx->blocks, bytes, cudaMemcpyDeviceToHost));
    FILE *f = fopen(path, "wb");
    if (!f) {
        set_error("cannot open %s for writing", path);
        return RB3_E_IO;
    }
    int64_t hdr[12] = {1, idx->n, idx->m, idx->C[0], idx->C[1], idx->C[2], idx->C[3], idx->C[4], idx->C[5],
                       idx->C[6], idx->nblocks,
                       ((int64_t)idx->sa_s << 32) | ((int64_t)idx->D << 8) | (idx->rle ? 2 : 0) |
                           (idx->single_strand ? 1 : 0)};
    bool ok = fwrite(k_magic, 1, 8, f) == 8 && fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
              fwrite(host.data(), 1, bytes, f) == bytes;
    if (ok && idx->gbase) {  // D = 32 or run-length past 2^32 symbols: the span bases follow the blocks
        std::vector<int64_t> gb(5 * gbase_rows(idx->n));
        if (cudaMemcpy(gb.data(), idx->gbase, sizeof(int64_t) * gb.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
            fclose(f);
            return cuda_fail(cudaGetLastError(), "rb3_index_save", __FILE__, __LINE__);
        }
        ok = fwrite(gb.data(), sizeof(int64_t), gb.size(), f) == gb.size();
    }
    if (ok && idx->rle) {  // run-length layout: payload size, run count, the runs
        std::vector<uint8_t> pl((size_t)idx->payload_bytes);
        if (!pl.empty() &&
            cudaMemcpy(pl.data(), idx->payload, pl.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
            fclose(f);
            return cuda_fail(cudaGetLastError(), "rb3_index_save", __FILE__, __LINE__);
        }
        const int64_t pr[2] = {idx->payload_bytes, idx->runs};
        ok = fwrite(pr, sizeof(pr), 1, f) == 1 && fwrite(pl.data(), 1, pl.size(), f) == pl.size();
    }
    if (ok && idx->sa_s) {  // sampled suffix array: its count, the row directory, the values
        std::vector<uint64_t> sd(2 * (idx->n / 64 + 1)), sv(idx->n_samples);
        if (cudaMemcpy(sd.data(), idx->sdir, sizeof(uint64_t) * sd.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
            (idx->n_samples && cudaMemcpy(sv.data(), idx->svals, sizeof(uint64_t) * sv.size(),
                                          cudaMemcpyDeviceToHost) != cudaSuccess)) {
            fclose(f);
            return cuda_fail(cudaGetLastError(), "rb3_index_save", __FILE__, __LINE__);
        }
        const int64_t ns = idx->n_samples;
        ok = fwrite(&ns, sizeof(ns), 1, f) == 1 && fwrite(sd.data(), sizeof(uint64_t), sd.size(), f) == sd.size() &&
             fwrite(sv.data(), sizeof(uint64_t), sv.size(), f) == sv.size();
    }
    ok = (fclose(f) == 0) && ok;
    if (!ok) {
        set_error("write to %s failed", path);
        return RB3_E_IO;
    }
    return RB3_OK;
}

RB3_EXPORT int rb3_index_load(const char *path, void *stream, rb3_index **out) {
    g_err.clear();
    RB3_CHECK_ARG(path && out, "NULL argument");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) {
        set_error("cannot open %s", path);
        return RB3_E_IO;
    }
    char mg[8];
    int64_t hdr[12];
    if (fread(mg, 1, 8, f) != 8 || memcmp(mg, k_magic, 8) != 0 || fread(hdr, sizeof(hdr), 1, f) != 1 || hdr[0] != 1) {
        fclose(f);
        set_error("%s: not an rb3 index image", path);
        return RB3_E_IO;
    }
    int D = (int)((hdr[11] >> 8) & 0xFFFFFF);
    const int sa_s = (int)(hdr[11] >> 32);
    const bool rle = (hdr[11] & 2) != 0;
    int64_t n = hdr[1], nblocks = hdr[10];
    if (!(rle ? valid_rle_span(D) : valid_occ_interval(D)) || n < 0 || nblocks != n / D + 1 || hdr[9] != n) {
        fclose(f);
        set_error("%s: inconsistent header", path);
        return RB3_E_IO;
    }
    rb3_index *x = new rb3_index();
    x->n = n;
    x->m = hdr[2];
    for (int a = 0; a < 7; ++a) x->C[a] = hdr[3 + a];
    x->D = D;
    x->log2D = ilog2(D);
    x->rle = rle ? 1 : 0;
    x->block_bytes = rle ? RLE_HDR_BYTES : block_bytes_for(D);
    x->single_strand = (int)(hdr[11] & 1);
    x->nblocks = nblocks;
    cudaGetDevice(&x->device);
    size_t bytes = (size_t)nblocks * x->block_bytes;
    std::vector<uint8_t> host(bytes);
    bool ok = fread(host.data(), 1, bytes, f) == bytes;
    std::vector<int64_t> gb;
    if (ok && (D == 32 || rle) && (n >> GSPAN_LOG2)) {
        gb.resize(5 * gbase_rows(n));
        ok = fread(gb.data(), sizeof(int64_t), gb.size(), f) == gb.size();
    }
    std::vector<uint8_t> pl;
    if (ok && rle) {
        int64_t pr[2];
        // a run takes at least one byte and at most three per symbol it covers
        ok = fread(pr, sizeof(pr), 1, f) == 1 && pr[0] >= 0 && pr[0] <= 3 * n && pr[1] >= 0 && pr[1] <= n;
        if (ok) {
            x->payload_bytes = pr[0];
            x->runs = pr[1];
            pl.resize((size_t)pr[0]);
            ok = fread(pl.data(), 1, pl.size(), f) == pl.size();
        }
    }
    std::vector<uint64_t> sd, sv;
    if (ok && sa_s) {
        int64_t ns = 0;
        ok = fread(&ns, sizeof(ns), 1, f) == 1 && ns >= 0 && ns <= n + 1;
        if (ok) {
            sd.resize(2 * (n / 64 + 1));
            sv.resize(ns);
            ok = fread(sd.data(), sizeof(uint64_t), sd.size(), f) == sd.size() &&
                 fread(sv.data(), sizeof(uint64_t), sv.size(), f) == sv.size();
        }
    }
    fclose(f);
    if (!ok) {
        delete x;
        set_error("%s: truncated", path);
        return RB3_E_IO;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int r = dev_alloc((void **)&x->blocks, bytes, st);
    if (r == RB3_OK) {
        cudaError_t e = cudaMemcpyAsync(x->blocks, host.data(), bytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) r = cuda_fail(e, "rb3_index_load", __FILE__, __LINE__);
    }
    if (r == RB3_OK && sa_s) {
        x->sa_s = sa_s;
        x->n_samples = (int64_t)sv.size();
        r = dev_alloc((void **)&x->sdir, sizeof(uint64_t) * sd.size(), st);
        if (r == RB3_OK) r = dev_alloc((void **)&x->svals, sizeof(uint64_t) * (sv.empty() ? 1 : sv.size()), st);
        if (r == RB3_OK) {
            cudaError_t e = cudaMemcpyAsync(x->sdir, sd.data(), sizeof(uint64_t) * sd.size(), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess && !sv.empty())
                e = cudaMemcpyAsync(x->svals, sv.data(), sizeof(uint64_t) * sv.size(), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) r = cuda_fail(e, "rb3_index_load", __FILE__, __LINE__);
        }
    }
    if (r == RB3_OK && !gb.empty()) {
        r = dev_alloc((void **)&x->gbase, sizeof(int64_t) * gb.size(), st);
        if (r == RB3_OK) {
            cudaError_t e = cudaMemcpyAsync(x->gbase, gb.data(), sizeof(int64_t) * gb.size(), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) r = cuda_fail(e, "rb3_index_load", __FILE__, __LINE__);
        }
    }
    if (r == RB3_OK && rle) {  // the runs, checked before any rank decodes them
        r = dev_alloc((void **)&x->payload, pl.size() + 16, st);
        if (r == RB3_OK) {
            cudaError_t e = cudaMemsetAsync(x->payload + pl.size(), 0, 16, st);
            if (e == cudaSuccess && !pl.empty())
                e = cudaMemcpyAsync(x->payload, pl.data(), pl.size(), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) r = cuda_fail(e, "rb3_index_load", __FILE__, __LINE__);
        }
        if (r == RB3_OK) r = rle_check_impl(x, st);
        if (r != RB3_OK && r != RB3_E_CUDA) set_error("%s: run-length data inconsistent", path);
    }
    if (r == RB3_OK) {
        int64_t C0[7];
        memcpy(C0, x->C, sizeof(C0));
        r = finalize_counts(x, st);
        if (r == RB3_OK && memcmp(C0, x->C, sizeof(C0)) != 0) {
            set_error("%s: counts do not match the blocks", path);
            r = RB3_E_IO;
        }
    }
    if (r != RB3_OK) {
        free_index(x);
        return r;
    }
    *out = x;
    return RB3_OK;
}

RB3_EXPORT void rb3_index_free(rb3_index *idx) { free_index(idx); }

RB3_EXPORT int rb3_encode_ascii(const char *ascii, int64_t n, uint8_t *codes) {
    g_err.clear();
    RB3_CHECK_ARG(n >= 0 && (n == 0 || (ascii && codes)), "bad argument");
    for (int64_t i = 0; i < n; ++i) {
        switch (ascii[i]) {
            case 'A': case 'a': codes[i] = 1; break;
            case 'C': case 'c': codes[i] = 2; break;
            case 'G': case 'g': codes[i] = 3; break;
            case 'T': case 't': codes[i] = 4; break;
            default: codes[i] = 5;
        }
    }
    return RB3_OK;
}

RB3_EXPORT int rb3_profile_enable(int on) {
    g_prof.store(on != 0);
    return RB3_OK;
}

RB3_EXPORT int rb3_profile_reset(void) {
    profile_drain();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_acc.clear();
    g_spans.clear();
    if (!g_origin) RB3_CUDA_TRY(cudaEventCreate(&g_origin));
    RB3_CUDA_TRY(cudaEventRecord(g_origin, 0));
    return RB3_OK;
}

RB3_EXPORT int rb3_profile_timeline(const char **names, double *start_ms, double *dur_ms, int64_t cap, int64_t *n) {
    profile_drain();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    const int64_t m = (int64_t)g_spans.size();
    for (int64_t i = 0; i < m && i < cap; ++i) {
        if (names) names[i] = g_spans[i].name;
        if (start_ms) start_ms[i] = g_spans[i].start;
        if (dur_ms) dur_ms[i] = g_spans[i].dur;
    }
    if (n) *n = m;
    return RB3_OK;
}

RB3_EXPORT int rb3_profile_read(const char **names, double *ms, int64_t *calls, double *bytes, int32_t cap,
                                int32_t *n) {
    profile_drain();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int32_t i = 0;
    g_names.clear();
    g_names.reserve(g_acc.size());
    for (auto &kv : g_acc) g_names.push_back(kv.first);
    for (auto &kv : g_acc) {
        if (i < cap) {
            if (names) names[i] = g_names[i].c_str();
            if (ms) ms[i] = kv.second.ms;
            if (calls) calls[i] = kv.second.calls;
            if (bytes) bytes[i] = kv.second.bytes;
        }
        ++i;
    }
    if (n) *n = i;
    return RB3_OK;
}

RB3_EXPORT int64_t rb3_launch_count(void) { return g_launches.load(); }
