// SMEM search without any device allocation.
//
// Some callers cannot allocate device memory on the search path: their device
// memory is handed out by their own allocator or fixed memory plan, or their
// request loop must not call cudaMalloc / cudaFree, which can block and
// synchronize the device.  rb3_mem_search_noalloc serves them.  Its scratch
// (per-query chunk offsets, per-chunk record counts and offsets, scan partials,
// a flag) is the file-scope array below, of fixed size, which every GPU that
// loads the library holds until the process exits.  The caller passes device
// inputs and a device output buffer.
//
// The search is the same Algorithm 4 loop as rb3_mem_search's chunked form.
// To order the records by (query, start) without a sort (a sort needs scratch
// proportional to the output), it runs twice: the first pass counts the SMEMs
// of every chunk, a scan turns the counts into output offsets, and the second
// pass writes each chunk's SMEMs, which it finds in increasing start order, at
// its offset.
#include <mutex>

#include "smem.cuh"

namespace rb3 {

constexpr int64_t NA_MAX_QUERIES = 131072;  // queries per call
constexpr int64_t NA_MAX_CHUNKS = 524288;   // query chunks of NA_CHUNK bases per call
constexpr int64_t NA_CHUNK = 256;
constexpr int64_t NA_PARTS = 2048;           // scan partials
constexpr int64_t NA_QITEMS = 0;                                // [NA_MAX_QUERIES + 1] chunks per query -> offsets
constexpr int64_t NA_RCNT = NA_QITEMS + NA_MAX_QUERIES + 1;     // [NA_MAX_CHUNKS + 1] SMEMs per chunk
constexpr int64_t NA_ROFF = NA_RCNT + NA_MAX_CHUNKS + 1;        // [NA_MAX_CHUNKS + 1] output offsets
constexpr int64_t NA_PART = NA_ROFF + NA_MAX_CHUNKS + 1;        // [NA_PARTS]
constexpr int64_t NA_MISC = NA_PART + NA_PARTS;                 // [16]: word 0 = bad-symbol flag, 1 = bad-qoff flag
constexpr int64_t NA_WORDS = NA_MISC + 16;                      // 4,726,868 bytes in all

static __device__ __align__(256) uint32_t g_noalloc_scratch[NA_WORDS];

// Device address of the scratch array on the current device, looked up once
// per device (the host-side name g_noalloc_scratch is not a device address).
static uint32_t *g_na_addr[256];
static std::mutex g_na_mu;

static int noalloc_scratch(uint32_t **out) {
    int dev = 0;
    RB3_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) {
        set_error("device ordinal %d out of range", dev);
        return RB3_E_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        RB3_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_na_addr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_na_addr[dev];
    return RB3_OK;
}

__global__ void k_na_check(const uint8_t *__restrict__ q, int64_t b, int64_t e, uint32_t *__restrict__ bad) {
    for (int64_t i = b + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < e; i += (int64_t)gridDim.x * blockDim.x) {
        uint8_t c = q[i];
        if (c < 1 || c > 5) atomicOr(bad, 1u);
    }
}

// chunks of query i (at least one); entry nq is 0 so that the scan's last
// value is the total.  A query whose offsets run backwards, or whose length
// does not fit the records' 32-bit start / end, sets *bad_qoff (the host
// refuses the call before any search kernel runs); with non-decreasing
// offsets every query lies inside [qoff[0], qoff[nq]), the range the symbol
// check covers.
__global__ void k_na_qitems(const int64_t *__restrict__ qoff, int64_t nq, uint32_t *__restrict__ qitems,
                            uint32_t *__restrict__ bad_qoff) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > nq) return;
    if (i == nq) {
        qitems[i] = 0;
        return;
    }
    int64_t len = qoff[i + 1] - qoff[i];
    if (len < 0 || len >= ((int64_t)1 << 31)) {
        atomicOr(bad_qoff, 1u);
        len = 0;
    }
    qitems[i] = (uint32_t)(len <= NA_CHUNK ? 1 : (len + NA_CHUNK - 1) / NA_CHUNK);
}

struct EmitCount {
    uint32_t n;
    __device__ __forceinline__ void operator()(int64_t, int64_t, int64_t, const BiInt &) { ++n; }
};

struct EmitAt {
    rb3_smem *out;
    int64_t at;
    __device__ __forceinline__ void operator()(int64_t qid, int64_t st, int64_t en, const BiInt &x) {
        rb3_smem r;
        r.qid = qid;
        r.start = (int32_t)st;
        r.end = (int32_t)en;
        r.k = x.k;
        r.kp = x.kp;
        r.s = x.s;
        out[at++] = r;
    }
};

template <int NS, bool WRITE>
__global__ void __launch_bounds__(256) k_na_smem(OccView V, const uint8_t *__restrict__ q,
                                                 const int64_t *__restrict__ qoff, int64_t nq,
                                                 const uint32_t *__restrict__ item_off, int64_t nitems, int ell,
                                                 int64_t smin, uint32_t *__restrict__ rcnt,
                                                 const uint32_t *__restrict__ roff, rb3_smem *__restrict__ out) {
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < nitems;
         it += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = nq;  // largest query index i with item_off[i] <= it
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) >> 1;
            if ((int64_t)item_off[mid] <= it) lo = mid;
            else hi = mid;
        }
        const int64_t qi = lo;
        const int64_t len = qoff[qi + 1] - qoff[qi];
        const int64_t x0 = (it - (int64_t)item_off[qi]) * NA_CHUNK;
        const int64_t x1 = x0 + NA_CHUNK < len ? x0 + NA_CHUNK : len;
        if (WRITE) {
            EmitAt em{out, (int64_t)roff[it]};
            smem_range<NS>(V, q + qoff[qi], len, qi, x0, x1, ell, smin, em);
        } else {
            EmitCount em{0};
            smem_range<NS>(V, q + qoff[qi], len, qi, x0, x1, ell, smin, em);
            rcnt[it] = em.n;
        }
    }
}

static inline unsigned nb_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

static int mem_search_noalloc(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, int64_t nq,
                              int32_t min_len, int64_t min_occ, rb3_smem *out, int64_t cap, int64_t *n_out,
                              cudaStream_t st) {
    RB3_CHECK_ARG(idx != nullptr && n_out != nullptr, "NULL argument");
    *n_out = 0;
    RB3_CHECK_ARG(nq >= 0 && cap >= 0, "negative size");
    if (nq > NA_MAX_QUERIES) {
        set_error("rb3_mem_search_noalloc: %lld queries, at most %lld per call", (long long)nq,
                  (long long)NA_MAX_QUERIES);
        return RB3_E_INVAL;
    }
    RB3_CHECK_ARG(min_len >= 1, "min_len must be >= 1");
    RB3_CHECK_ARG(min_occ >= 1, "min_occ must be >= 1");
    RB3_CHECK_ARG(!idx->single_strand, "SMEM search needs a double-strand index");
    if (nq == 0) return RB3_OK;
    RB3_CHECK_ARG(is_device_ptr(qoff) && (q == nullptr || is_device_ptr(q)),
                  "rb3_mem_search_noalloc takes device pointers for q and qoff");
    RB3_CHECK_ARG(cap == 0 || (out != nullptr && is_device_ptr(out)), "out must be a device pointer");
    uint32_t *ws = nullptr;
    RB3_TRY(noalloc_scratch(&ws));
    uint32_t *qitems = ws + NA_QITEMS, *rcnt = ws + NA_RCNT, *roff = ws + NA_ROFF, *part = ws + NA_PART;
    uint32_t *bad = ws + NA_MISC, *bad_qoff = ws + NA_MISC + 1;
    int64_t ends[2] = {0, 0};
    RB3_CUDA_TRY(cudaMemcpyAsync(&ends[0], qoff, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaMemcpyAsync(&ends[1], qoff + nq, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaMemsetAsync(bad, 0, 2 * sizeof(uint32_t), st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    RB3_CHECK_ARG(ends[0] >= 0 && ends[1] >= ends[0], "bad qoff");
    RB3_CHECK_ARG(ends[1] == ends[0] || q != nullptr, "q is NULL");
    // every chunk holds at most NA_CHUNK bases, so more bases than this are more
    // chunks than the limit (checked here, before the per-query counts are added
    // up in 32 bits)
    if (ends[1] - ends[0] > NA_MAX_CHUNKS * NA_CHUNK) {
        set_error("rb3_mem_search_noalloc: %lld query bases, more than the limit of %lld chunks of %lld bases",
                  (long long)(ends[1] - ends[0]), (long long)NA_MAX_CHUNKS, (long long)NA_CHUNK);
        return RB3_E_INVAL;
    }
    if (ends[1] > ends[0]) {
        unsigned grid = nb_for(ends[1] - ends[0], 256);
        if (grid > (unsigned)num_sms() * 8) grid = (unsigned)num_sms() * 8;
        RB3_LAUNCH(k_na_check, grid, 256, 0, st, q, ends[0], ends[1], bad);
    }
    RB3_LAUNCH(k_na_qitems, nb_for(nq + 1, 256), 256, 0, st, qoff, nq, qitems, bad_qoff);
    RB3_TRY(scan_u32_ws(qitems, qitems, nq + 1, false, part, NA_PARTS, st));
    uint32_t hv[3] = {0, 0, 0};
    RB3_CUDA_TRY(cudaMemcpyAsync(&hv[0], qitems + nq, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaMemcpyAsync(&hv[1], bad, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    if (hv[2]) {
        set_error("rb3_mem_search_noalloc: qoff decreases, or a query is 2^31 bases or longer");
        return RB3_E_INVAL;
    }
    if (hv[1]) {
        set_error("query symbol outside 1..5 (A,C,G,T,N codes)");
        return RB3_E_INVAL;
    }
    const int64_t nitems = hv[0];
    if (nitems > NA_MAX_CHUNKS) {
        set_error("rb3_mem_search_noalloc: %lld query chunks of %lld bases, at most %lld per call", (long long)nitems,
                  (long long)NA_CHUNK, (long long)NA_MAX_CHUNKS);
        return RB3_E_INVAL;
    }
    const OccView V = occ_view(idx);
    const unsigned grid = nb_for(nitems, 256) < (unsigned)num_sms() * 8 ? nb_for(nitems, 256) : (unsigned)num_sms() * 8;
    RB3_CUDA_TRY(cudaMemsetAsync(rcnt + nitems, 0, sizeof(uint32_t), st));
    RB3_WITH_NS(idx->D, RB3_LAUNCH((k_na_smem<NS, false>), grid, 256, 0, st, V, q, qoff, nq, qitems, nitems,
                                   (int)min_len, min_occ, rcnt, (const uint32_t *)nullptr, (rb3_smem *)nullptr));
    RB3_TRY(scan_u32_ws(rcnt, roff, nitems + 1, false, part, NA_PARTS, st));
    uint32_t total = 0;
    RB3_CUDA_TRY(cudaMemcpyAsync(&total, roff + nitems, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    *n_out = total;
    if ((int64_t)total > cap) {
        set_error("mem_search: %lld SMEMs found, output capacity %lld", (long long)total, (long long)cap);
        return RB3_E_CAPACITY;
    }
    if (total > 0)
        RB3_WITH_NS(idx->D, RB3_LAUNCH((k_na_smem<NS, true>), grid, 256, 0, st, V, q, qoff, nq, qitems, nitems,
                                       (int)min_len, min_occ, (uint32_t *)nullptr, (const uint32_t *)roff, out));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    return RB3_OK;
}

}  // namespace rb3

RB3_EXPORT int rb3_mem_search_noalloc(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, int64_t nq,
                                      int32_t min_len, int64_t min_occ, rb3_smem *out, int64_t cap, int64_t *n_out,
                                      void *stream) {
    rb3::set_error("%s", "");
    return rb3::mem_search_noalloc(idx, q, qoff, nq, min_len, min_occ, out, cap, n_out, (cudaStream_t)stream);
}
