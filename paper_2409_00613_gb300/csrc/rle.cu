// Run-length index (Section "BWT construction", Fig. 2b: the static form of the
// BWT, run-length encoded and interleaved with marginal counts per block, with
// an index into it for fast access).
//
// Here the BWT is cut into spans of S symbols.  Each span has a 64-byte header
// (the marginal counts at its start, where its runs begin, and two decode
// marks inside it) in a directory indexed by l >> log2 S, so a rank is one
// header read plus a decode of the span's runs from the last mark before l.
// Runs are bytes (a 3-bit symbol and a 5-bit length,
// with one or two extra length bytes for long runs; format in common.cuh),
// not the paper's Elias-delta bit code: a byte code decodes with plain shifts
// and needs no bit-level cursor on the GPU.  The index is built from a finished
// plain index, and grows by merges: the walk ranks its spans, and the merged
// spans are written from its old runs and the new batch's symbols at their
// merged rows (the BWT's dynamic form, kept static between merges).  Every
// query (backward search, SMEM search, locate, export) runs on it through the
// same kernels, with the rank primitives of the run-length layout.
#include "common.cuh"

namespace rb3 {

static inline unsigned nb_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Mark j of a span of slen symbols: the run holding offset (j + 1) * slen / 3.
__host__ __device__ __forceinline__ int64_t rle_mark_target(int j, int64_t slen) { return (j + 1) * slen / 3; }

// Encoder of one span's runs, fed (symbol, count) pieces in row order: a piece
// of the pending run's symbol extends it, so the runs are maximal.  WRITE = false
// counts bytes and runs only; WRITE = true also writes the run bytes from p and
// the decode marks into the header words w[8..15].
template <bool WRITE> struct SpanEnc {
    uint8_t *p0 = nullptr, *p = nullptr;
    uint32_t *w = nullptr;
    int64_t slen = 0, at = 0;  // the span's symbols; offset of the pending run
    int j = 0;                 // next mark
    uint32_t cnt[SIGMA] = {0, 0, 0, 0, 0, 0};
    uint64_t bytes = 0, runs = 0;
    int cur = -1;
    int64_t len = 0;
    __device__ __forceinline__ void put(int a, int64_t t) {
        if (t <= 0) return;
        if (a == cur) {
            len += t;
            return;
        }
        flush();
        cur = a;
        len = t;
    }
    __device__ __forceinline__ void flush() {
        if (len == 0) return;
        const int64_t e = at + len;
        if constexpr (WRITE) {
            while (j < RLE_MARKS && rle_mark_target(j, slen) < e) {  // this run holds mark j's offset
                w[8 + 4 * j] = (uint32_t)at | (cnt[1] << 16);
                w[9 + 4 * j] = cnt[2] | (cnt[3] << 16);
                w[10 + 4 * j] = cnt[4] | (cnt[5] << 16);
                w[11 + 4 * j] = (uint32_t)(p - p0);
                ++j;
            }
            if (len < RLE_BASE1) {
                *p++ = (uint8_t)((cur << 5) | (len - 1));
            } else if (len < RLE_BASE2) {
                *p++ = (uint8_t)((cur << 5) | RLE_F1);
                *p++ = (uint8_t)(len - RLE_BASE1);
            } else {
                const int64_t x = len - RLE_BASE2;
                *p++ = (uint8_t)((cur << 5) | RLE_F2);
                *p++ = (uint8_t)(x & 0xFF);
                *p++ = (uint8_t)(x >> 8);
            }
        }
        bytes += (uint64_t)rle_run_bytes(len);
        ++runs;
        cnt[cur] += (uint32_t)len;
        at = e;
        len = 0;
    }
};

// One thread per span: runs of codes[s0, s1) and the bytes they take.
__global__ void k_rle_size(const uint8_t *__restrict__ codes, int64_t n, int log2S, int64_t nspans,
                           uint64_t *__restrict__ bytes, uint64_t *__restrict__ runs) {
    const int64_t sp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (sp >= nspans) return;
    const int64_t s0 = sp << log2S, s1 = s0 + ((int64_t)1 << log2S) < n ? s0 + ((int64_t)1 << log2S) : n;
    SpanEnc<false> enc;
    int64_t i = s0;
    while (i < s1) {
        const uint8_t a = codes[i];
        int64_t j = i + 1;
        while (j < s1 && codes[j] == a) ++j;
        enc.put(a, j - i);
        i = j;
    }
    enc.flush();
    bytes[sp] = enc.bytes;
    runs[sp] = enc.runs;
}

// One thread per span: header (ranks at the span start from the plain index,
// minus the gbase of their 2^32 range; where the runs begin; the marks) and runs.
__global__ void k_rle_write(const uint8_t *__restrict__ codes, OccView src, int log2S, int64_t nspans,
                            const uint64_t *__restrict__ off, const uint64_t *__restrict__ runs,
                            const int64_t *__restrict__ gbase, uint8_t *__restrict__ hdr,
                            uint8_t *__restrict__ payload) {
    const int64_t sp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (sp >= nspans) return;
    const int64_t n = src.n, s0 = sp << log2S;
    const int64_t s1 = s0 + ((int64_t)1 << log2S) < n ? s0 + ((int64_t)1 << log2S) : n;
    int64_t r[SIGMA];
    rank_all_any(src, s0, r);
    uint32_t w[16];
    const int64_t *g = gbase ? gbase + 5 * (s0 >> GSPAN_LOG2) : nullptr;
    for (int a = 1; a < SIGMA; ++a) w[a - 1] = (uint32_t)(r[a] - (g ? g[a - 1] : 0));
    w[5] = (uint32_t)off[sp];
    w[6] = (uint32_t)(off[sp] >> 32);
    w[7] = (uint32_t)runs[sp];
    for (int k = 8; k < 16; ++k) w[k] = 0;
    SpanEnc<true> enc;
    enc.p0 = enc.p = payload + off[sp];
    enc.w = w;
    enc.slen = s1 - s0;
    int64_t i = s0;
    while (i < s1) {
        const uint8_t a = codes[i];
        int64_t e = i + 1;
        while (e < s1 && codes[e] == a) ++e;
        enc.put(a, e - i);
        i = e;
    }
    enc.flush();
    uint4 *h = reinterpret_cast<uint4 *>(hdr + sp * RLE_HDR_BYTES);
    for (int k = 0; k < 4; ++k) h[k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
}

// gbase[5 g + a - 1] = rank(a, g * 2^32) of the plain index.
__global__ void k_rle_gbase(OccView src, int64_t rows, int64_t *__restrict__ gbase) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= rows) return;
    int64_t r[SIGMA];
    rank_all_any(src, g << GSPAN_LOG2, r);
    for (int a = 1; a < SIGMA; ++a) gbase[5 * g + a - 1] = r[a];
}

// One thread per span: its runs written out as codes.
__global__ void k_rle_unpack(OccView V, int64_t nspans, uint8_t *__restrict__ codes) {
    const int64_t sp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (sp >= nspans) return;
    const int64_t s0 = sp << V.log2D;
    int64_t slen = V.n - s0;
    if (slen > ((int64_t)1 << V.log2D)) slen = (int64_t)1 << V.log2D;
    if (slen <= 0) return;
    int64_t base[SIGMA], pos;
    uint64_t acc[2];
    RunRd rd;
    rd.init(rle_start(V, sp, 0, base, &pos, acc));  // offset 0: the span's first run
    while (pos < slen) {
        int a;
        int64_t len;
        rd.run(&a, &len);
        for (int64_t t = 0; t < len && pos + t < slen; ++t) codes[s0 + pos + t] = (uint8_t)a;
        pos += len;
    }
}

// occ[sp * 6 + a] = rank(a, sp * S): the span headers.
__global__ void k_rle_occ(OccView V, int64_t nspans, int64_t *__restrict__ occ) {
    const int64_t sp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (sp >= nspans) return;
    int64_t r[SIGMA], pos;
    uint64_t acc[2];
    rle_start(V, sp, 0, r, &pos, acc);
    r[0] = (sp << V.log2D) - (r[1] + r[2] + r[3] + r[4] + r[5]);
    for (int a = 0; a < SIGMA; ++a) occ[sp * SIGMA + a] = r[a];
}

// ---- merge into a run-length index -------------------------------------------
// The merged BWT of a run-length B1 and a plain B2 at the rows pos (increasing)
// is written span by span, without a plain copy: output span sp holds merged
// rows [r0, r1), of which pos[a0, a1) are B2's, a0 = |{pos < r0}|, and the rest
// are B1's rows from o0 = r0 - a0 on, in order.  One thread per output span
// reads B1's runs from o0 and puts B2's symbols between them.

__device__ __forceinline__ int64_t lower_bound_i64(const int64_t *__restrict__ a, int64_t n, int64_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Sequential reader of a run-length B's runs from a row on, across spans.
struct RunCursor {
    int64_t sp, s0, slen, pos;  // span, its first row, its symbols, offset after the current run
    RunRd rd;
    int sym = 0;
    int64_t left = 0;  // rows of the current run not yet taken
    __device__ __forceinline__ void open_span(const OccView &v, int64_t s, int64_t o) {
        sp = s;
        s0 = s << v.log2D;
        slen = v.n - s0 < ((int64_t)1 << v.log2D) ? v.n - s0 : ((int64_t)1 << v.log2D);
        int64_t base[SIGMA];
        uint64_t acc[2];
        rd.init(rle_start(v, s, o, base, &pos, acc));
    }
    // the run holding row l < n, with the rows of it from l on
    __device__ __forceinline__ void open(const OccView &v, int64_t l) {
        open_span(v, l >> v.log2D, l - ((l >> v.log2D) << v.log2D));
        left = 0;
        while (left == 0 && pos < slen) {
            int64_t len;
            rd.run(&sym, &len);
            pos += len;
            if (s0 + pos > l) left = s0 + pos - l;
        }
    }
    // the next run (the caller takes rows only below n)
    __device__ __forceinline__ void next(const OccView &v) {
        if (pos >= slen) open_span(v, sp + 1, 0);
        int64_t len;
        rd.run(&sym, &len);
        pos += len;
        left = len;
    }
};

template <bool WRITE>
__global__ void k_rle_merge(OccView V1, OccView V2, const uint8_t *__restrict__ codes2,
                            const int64_t *__restrict__ pos, int64_t n2, int64_t nM, int64_t nspans,
                            const uint64_t *__restrict__ off, uint64_t *__restrict__ bytes,
                            uint64_t *__restrict__ runs, const int64_t *__restrict__ gbase,
                            uint8_t *__restrict__ hdr, uint8_t *__restrict__ payload) {
    const int64_t sp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (sp >= nspans) return;
    const int log2S = V1.log2D;
    const int64_t r0 = sp << log2S;
    const int64_t r1 = r0 + ((int64_t)1 << log2S) < nM ? r0 + ((int64_t)1 << log2S) : nM;
    const int64_t a0 = lower_bound_i64(pos, n2, r0);
    SpanEnc<WRITE> enc;
    enc.slen = r1 > r0 ? r1 - r0 : 0;
    uint32_t w[16];
    if constexpr (WRITE) {
        // ranks at the span start: B1's below o0 plus B2's below a0
        int64_t q1[SIGMA], q2[SIGMA];
        rank_all_any(V1, r0 - a0, q1);
        rank_all_any(V2, a0, q2);
        const int64_t *g = gbase ? gbase + 5 * (r0 >> GSPAN_LOG2) : nullptr;
        for (int a = 1; a < SIGMA; ++a) w[a - 1] = (uint32_t)(q1[a] + q2[a] - (g ? g[a - 1] : 0));
        w[5] = (uint32_t)off[sp];
        w[6] = (uint32_t)(off[sp] >> 32);
        w[7] = (uint32_t)runs[sp];
        for (int k = 8; k < 16; ++k) w[k] = 0;
        enc.p0 = enc.p = payload + off[sp];
        enc.w = w;
    }
    RunCursor old;
    bool opened = false;
    int64_t a = a0, r = r0;
    while (r < r1) {
        const int64_t nx = a < n2 && pos[a] < r1 ? pos[a] : r1;  // the next B2 row (or the span end)
        while (r < nx) {  // B1's rows up to it: old row r - a
            if (!opened) {
                old.open(V1, r - a);
                opened = true;
            } else if (old.left == 0) {
                old.next(V1);
            }
            const int64_t t = old.left < nx - r ? old.left : nx - r;
            enc.put(old.sym, t);
            old.left -= t;
            r += t;
        }
        if (nx < r1) {
            enc.put(codes2[a], 1);
            ++a;
            ++r;
        }
    }
    enc.flush();
    if constexpr (WRITE) {
        uint4 *h = reinterpret_cast<uint4 *>(hdr + sp * RLE_HDR_BYTES);
        for (int k = 0; k < 4; ++k) h[k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
    } else {
        bytes[sp] = enc.bytes;
        runs[sp] = enc.runs;
    }
}

// gbase[5 g + a - 1] = rank(a, g * 2^32) of the merged BWT.
__global__ void k_rle_merge_gbase(OccView V1, OccView V2, const int64_t *__restrict__ pos, int64_t n2, int64_t rows,
                                  int64_t *__restrict__ gbase) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= rows) return;
    const int64_t R = g << GSPAN_LOG2, a = lower_bound_i64(pos, n2, R);
    int64_t q1[SIGMA], q2[SIGMA];
    rank_all_any(V1, R - a, q1);
    rank_all_any(V2, a, q2);
    for (int c = 1; c < SIGMA; ++c) gbase[5 * g + c - 1] = q1[c] + q2[c];
}

// Consistency of a run-length image read from a file, every read bounds-checked:
// each span's runs start at its header's offset, end where the next span's
// begin, cover exactly its symbols, match the header's run count, and advance
// the counts to the next header's.  bad != 0 on the first failure.
__global__ void k_rle_check(OccView V, int64_t pbytes, int64_t nspans, unsigned int *__restrict__ bad) {
    const int64_t sp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (sp >= nspans) return;
    const uint8_t *hdr = V.blocks, *payload = V.payload;
    const int64_t n = V.n, *gbase = V.gbase;
    const int log2S = V.log2D;
    const uint32_t *h = reinterpret_cast<const uint32_t *>(hdr + sp * RLE_HDR_BYTES);
    const int64_t s0 = sp << log2S;
    int64_t slen = n - s0;
    if (slen > ((int64_t)1 << log2S)) slen = (int64_t)1 << log2S;
    if (slen < 0) slen = 0;
    const uint64_t b0 = (uint64_t)h[5] | ((uint64_t)h[6] << 32);
    uint64_t b1 = (uint64_t)pbytes;
    if (sp + 1 < nspans) {
        const uint32_t *hn = reinterpret_cast<const uint32_t *>(hdr + (sp + 1) * RLE_HDR_BYTES);
        b1 = (uint64_t)hn[5] | ((uint64_t)hn[6] << 32);
    }
    if (b0 > b1 || b1 > (uint64_t)pbytes) {
        atomicOr(bad, 1u);
        return;
    }
    int64_t cnt[SIGMA] = {0, 0, 0, 0, 0, 0};
    int64_t pos = 0, nr = 0;
    uint64_t q = b0;
    uint32_t mk[4 * RLE_MARKS];  // the marks as the encoder places them
    for (int k = 0; k < 4 * RLE_MARKS; ++k) mk[k] = 0;
    int j = 0;
    while (pos < slen) {
        if (q >= b1) {
            atomicOr(bad, 2u);
            return;
        }
        const uint32_t b = payload[q++], f = b & 31u;
        const int a = (int)(b >> 5);
        int64_t len;
        if (f < (uint32_t)RLE_F1) {
            len = (int64_t)f + 1;
        } else if (f == (uint32_t)RLE_F1) {
            if (q >= b1) {
                atomicOr(bad, 2u);
                return;
            }
            len = RLE_BASE1 + (int64_t)payload[q++];
        } else {
            if (q + 1 >= b1) {
                atomicOr(bad, 2u);
                return;
            }
            len = RLE_BASE2 + (int64_t)(payload[q] | (payload[q + 1] << 8));
            q += 2;
        }
        if (a >= SIGMA || pos + len > slen) {
            atomicOr(bad, 4u);
            return;
        }
        while (j < RLE_MARKS && rle_mark_target(j, slen) < pos + len) {
            mk[4 * j] = (uint32_t)pos | ((uint32_t)cnt[1] << 16);
            mk[4 * j + 1] = (uint32_t)cnt[2] | ((uint32_t)cnt[3] << 16);
            mk[4 * j + 2] = (uint32_t)cnt[4] | ((uint32_t)cnt[5] << 16);
            mk[4 * j + 3] = (uint32_t)(q - b0 - rle_run_bytes(len));
            ++j;
        }
        cnt[a] += len;
        pos += len;
        ++nr;
    }
    if (q != b1 || nr != (int64_t)h[7]) {
        atomicOr(bad, 8u);
        return;
    }
    for (int k = 0; k < 4 * RLE_MARKS; ++k)
        if (h[8 + k] != mk[k]) {
            atomicOr(bad, 32u);
            return;
        }
    // the counts start at 0, advance by the span's runs to the next header's
    // (both relative to their 2^32 range) and end at the symbol totals
    const int64_t *g0 = gbase ? gbase + 5 * (s0 >> GSPAN_LOG2) : nullptr;
    const uint32_t *hn = sp + 1 < nspans ? reinterpret_cast<const uint32_t *>(hdr + (sp + 1) * RLE_HDR_BYTES) : nullptr;
    const int64_t *g1 = gbase ? gbase + 5 * ((s0 + ((int64_t)1 << log2S)) >> GSPAN_LOG2) : nullptr;
    for (int a = 1; a < SIGMA; ++a) {
        const int64_t c0 = (int64_t)h[a - 1] + (g0 ? g0[a - 1] : 0);
        const int64_t c1 = hn ? (int64_t)hn[a - 1] + (g1 ? g1[a - 1] : 0) : V.C[a + 1] - V.C[a];
        if ((sp == 0 && c0 != 0) || c0 + cnt[a] != c1) {
            atomicOr(bad, 16u);
            return;
        }
    }
}

int rle_export_impl(const rb3_index *x, uint8_t *codes, int64_t *occ, cudaStream_t st) {
    OccView V = occ_view(x);
    if (codes && x->n > 0) RB3_LAUNCH(k_rle_unpack, nb_for(x->nblocks, 128), 128, 0, st, V, x->nblocks, codes);
    if (occ) RB3_LAUNCH(k_rle_occ, nb_for(x->nblocks, 256), 256, 0, st, V, x->nblocks, occ);
    return RB3_OK;
}

int rle_check_impl(const rb3_index *x, cudaStream_t st) {
    DevBuf bad;
    RB3_TRY(bad.alloc(sizeof(unsigned int), st));
    RB3_CUDA_TRY(cudaMemsetAsync(bad.p, 0, sizeof(unsigned int), st));
    RB3_LAUNCH(k_rle_check, nb_for(x->nblocks, 128), 128, 0, st, occ_view(x), x->payload_bytes, x->nblocks,
               bad.as<unsigned int>());
    unsigned int h = 0;
    RB3_CUDA_TRY(cudaMemcpyAsync(&h, bad.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    if (h) {
        set_error("run-length image is inconsistent (check bits %u)", h);
        return RB3_E_IO;
    }
    return RB3_OK;
}

static int copy_samples(const rb3_index *src, rb3_index *x, cudaStream_t st) {
    if (!(src->sa_s && src->sdir)) return RB3_OK;
    const int64_t nw = src->n / 64 + 1;
    x->sa_s = src->sa_s;
    x->n_samples = src->n_samples;
    RB3_TRY(dev_alloc((void **)&x->sdir, sizeof(uint64_t) * 2 * nw, st));
    RB3_TRY(dev_alloc((void **)&x->svals, sizeof(uint64_t) * (x->n_samples > 0 ? x->n_samples : 1), st));
    RB3_CUDA_TRY(cudaMemcpyAsync(x->sdir, src->sdir, sizeof(uint64_t) * 2 * nw, cudaMemcpyDeviceToDevice, st));
    if (x->n_samples)
        RB3_CUDA_TRY(
            cudaMemcpyAsync(x->svals, src->svals, sizeof(uint64_t) * x->n_samples, cudaMemcpyDeviceToDevice, st));
    return RB3_OK;
}

static int compress_impl(const rb3_index *src, int S, cudaStream_t st, rb3_index *x) {
    const int64_t n = src->n;
    x->n = n;
    x->m = src->m;
    for (int a = 0; a < 7; ++a) x->C[a] = src->C[a];
    x->rle = 1;
    x->D = S;
    x->log2D = ilog2(S);
    x->block_bytes = RLE_HDR_BYTES;
    x->single_strand = src->single_strand;
    x->nblocks = n / S + 1;
    x->str_end = src->str_end;
    x->device = src->device;
    const int64_t ns = x->nblocks;
    OccView V = occ_view(src);
    if (n >> GSPAN_LOG2) {
        const int64_t rows = gbase_rows(n);
        RB3_TRY(dev_alloc((void **)&x->gbase, sizeof(int64_t) * 5 * rows, st));
        RB3_LAUNCH(k_rle_gbase, nb_for(rows, 64), 64, 0, st, V, rows, x->gbase);
    }
    DevBuf codes, bytes, runs, off;
    RB3_TRY(codes.alloc((size_t)(n > 0 ? n : 1), st));
    RB3_TRY(bytes.alloc(sizeof(uint64_t) * ns, st));
    RB3_TRY(runs.alloc(sizeof(uint64_t) * ns, st));
    RB3_TRY(off.alloc(sizeof(uint64_t) * ns, st));
    RB3_TRY(export_impl(src, codes.as<uint8_t>(), nullptr, st));
    RB3_LAUNCH(k_rle_size, nb_for(ns, 128), 128, 0, st, codes.as<uint8_t>(), n, x->log2D, ns, bytes.as<uint64_t>(),
               runs.as<uint64_t>());
    RB3_TRY(scan_u64(bytes.as<uint64_t>(), off.as<uint64_t>(), ns, false, st));
    uint64_t tail[4];
    RB3_CUDA_TRY(cudaMemcpyAsync(&tail[0], off.as<uint64_t>() + ns - 1, 8, cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaMemcpyAsync(&tail[1], bytes.as<uint64_t>() + ns - 1, 8, cudaMemcpyDeviceToHost, st));
    // total runs: the same exclusive scan over the run counts, reusing `bytes` as its output
    RB3_TRY(scan_u64(runs.as<uint64_t>(), bytes.as<uint64_t>(), ns, false, st));
    RB3_CUDA_TRY(cudaMemcpyAsync(&tail[2], bytes.as<uint64_t>() + ns - 1, 8, cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaMemcpyAsync(&tail[3], runs.as<uint64_t>() + ns - 1, 8, cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    x->payload_bytes = (int64_t)(tail[0] + tail[1]);
    x->runs = (int64_t)(tail[2] + tail[3]);
    RB3_TRY(dev_alloc((void **)&x->blocks, (size_t)ns * RLE_HDR_BYTES, st));
    RB3_TRY(dev_alloc((void **)&x->payload, (size_t)x->payload_bytes + 16, st));
    RB3_CUDA_TRY(cudaMemsetAsync(x->payload + x->payload_bytes, 0, 16, st));
    RB3_LAUNCH(k_rle_write, nb_for(ns, 128), 128, 0, st, codes.as<uint8_t>(), V, x->log2D, ns, off.as<uint64_t>(),
               runs.as<uint64_t>(), x->gbase, x->blocks, x->payload);
    RB3_TRY(copy_samples(src, x, st));  // the sampled suffix array is per row: rows do not change
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    return RB3_OK;
}

// One thread per D = 32 block of a plain copy: the ranks at its start from the
// run-length index (minus the same span bases), the planes from the codes.
__global__ void k_rle_to_plain32(OccView V, const uint8_t *__restrict__ codes, int64_t nb32,
                                 uint8_t *__restrict__ blocks) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb32) return;
    const int64_t l0 = b * 32;
    int64_t r[SIGMA];
    rle_rank<false>(V, l0, r, nullptr);
    const int64_t *g = V.gbase ? V.gbase + 5 * (l0 >> GSPAN_LOG2) : nullptr;
    uint32_t w[8];
    for (int a = 1; a < SIGMA; ++a) w[a - 1] = (uint32_t)(r[a] - (g ? g[a - 1] : 0));
    uint32_t p0 = 0, p1 = 0, p2 = 0;
    for (int j = 0; j < 32 && l0 + j < V.n; ++j) {
        const uint32_t c = codes[l0 + j];
        p0 |= (c & 1u) << j;
        p1 |= ((c >> 1) & 1u) << j;
        p2 |= ((c >> 2) & 1u) << j;
    }
    w[5] = p0;
    w[6] = p1;
    w[7] = p2;
    uint4 *h = reinterpret_cast<uint4 *>(blocks + b * 32);
    h[0] = make_uint4(w[0], w[1], w[2], w[3]);
    h[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// Plain D = 32 copy of a run-length index (same rows, same sampled suffix array).
static int decompress_impl(const rb3_index *x, cudaStream_t st, rb3_index *P) {
    const int64_t n = x->n;
    P->n = n;
    P->m = x->m;
    for (int a = 0; a < 7; ++a) P->C[a] = x->C[a];
    P->D = 32;
    P->log2D = 5;
    P->block_bytes = 32;
    P->single_strand = x->single_strand;
    P->nblocks = n / 32 + 1;
    P->str_end = x->str_end;
    P->device = x->device;
    DevBuf codes;
    RB3_TRY(codes.alloc((size_t)(n > 0 ? n : 1), st));
    RB3_TRY(rle_export_impl(x, codes.as<uint8_t>(), nullptr, st));
    RB3_TRY(dev_alloc((void **)&P->blocks, (size_t)P->nblocks * 32, st));
    RB3_LAUNCH(k_rle_to_plain32, nb_for(P->nblocks, 128), 128, 0, st, occ_view(x), codes.as<uint8_t>(), P->nblocks,
               P->blocks);
    if (x->gbase) {  // the same span bases: rank(a, g * 2^32)
        const size_t gb = sizeof(int64_t) * 5 * gbase_rows(n);
        RB3_TRY(dev_alloc((void **)&P->gbase, gb, st));
        RB3_CUDA_TRY(cudaMemcpyAsync(P->gbase, x->gbase, gb, cudaMemcpyDeviceToDevice, st));
    }
    RB3_TRY(copy_samples(x, P, st));
    int64_t Cw[7];
    for (int a = 0; a < 7; ++a) Cw[a] = P->C[a];
    RB3_TRY(finalize_counts(P, st));
    for (int a = 0; a < 7; ++a)
        if (P->C[a] != Cw[a]) {
            set_error("run-length decode: counts differ from the index's");
            return RB3_E_CUDA;
        }
    return RB3_OK;
}

// The run-length arrays of dst merged with src at rows pos (src plain; the
// span, strand mode and everything but the sampled suffix array): out's n, m,
// C, layout fields, gbase, blocks (headers) and payload.
int rle_merge_arrays(const rb3_index *dst, const rb3_index *src, const int64_t *pos, cudaStream_t st,
                     rb3_index *out) {
    const int64_t n2 = src->n, nM = dst->n + n2;
    out->n = nM;
    out->m = dst->m + src->m;
    for (int a = 0; a < 7; ++a) out->C[a] = dst->C[a] + src->C[a];
    out->rle = 1;
    out->D = dst->D;
    out->log2D = dst->log2D;
    out->block_bytes = RLE_HDR_BYTES;
    out->single_strand = src->single_strand;
    out->nblocks = nM / dst->D + 1;
    out->device = dst->device;
    const int64_t ns = out->nblocks;
    const OccView V1 = occ_view(dst), V2 = occ_view(src);
    DevBuf codes2, bytes, runs, off;
    RB3_TRY(codes2.alloc((size_t)(n2 > 0 ? n2 : 1), st));
    RB3_TRY(bytes.alloc(sizeof(uint64_t) * ns, st));
    RB3_TRY(runs.alloc(sizeof(uint64_t) * ns, st));
    RB3_TRY(off.alloc(sizeof(uint64_t) * ns, st));
    RB3_TRY(export_impl(src, codes2.as<uint8_t>(), nullptr, st));
    if (nM >> GSPAN_LOG2) {
        const int64_t rows = gbase_rows(nM);
        RB3_TRY(dev_alloc((void **)&out->gbase, sizeof(int64_t) * 5 * rows, st));
        RB3_LAUNCH(k_rle_merge_gbase, nb_for(rows, 64), 64, 0, st, V1, V2, pos, n2, rows, out->gbase);
    }
    {
        Phase ph("merge.rle_size", st);
        RB3_LAUNCH(k_rle_merge<false>, nb_for(ns, 128), 128, 0, st, V1, V2, codes2.as<uint8_t>(), pos, n2, nM, ns,
                   (const uint64_t *)nullptr, bytes.as<uint64_t>(), runs.as<uint64_t>(), (const int64_t *)nullptr,
                   (uint8_t *)nullptr, (uint8_t *)nullptr);
    }
    RB3_TRY(scan_u64(bytes.as<uint64_t>(), off.as<uint64_t>(), ns, false, st));
    uint64_t tail[4];
    RB3_CUDA_TRY(cudaMemcpyAsync(&tail[0], off.as<uint64_t>() + ns - 1, 8, cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaMemcpyAsync(&tail[1], bytes.as<uint64_t>() + ns - 1, 8, cudaMemcpyDeviceToHost, st));
    RB3_TRY(scan_u64(runs.as<uint64_t>(), bytes.as<uint64_t>(), ns, false, st));  // total runs
    RB3_CUDA_TRY(cudaMemcpyAsync(&tail[2], bytes.as<uint64_t>() + ns - 1, 8, cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaMemcpyAsync(&tail[3], runs.as<uint64_t>() + ns - 1, 8, cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    out->payload_bytes = (int64_t)(tail[0] + tail[1]);
    out->runs = (int64_t)(tail[2] + tail[3]);
    RB3_TRY(dev_alloc((void **)&out->blocks, (size_t)ns * RLE_HDR_BYTES, st));
    RB3_TRY(dev_alloc((void **)&out->payload, (size_t)out->payload_bytes + 16, st));
    RB3_CUDA_TRY(cudaMemsetAsync(out->payload + out->payload_bytes, 0, 16, st));
    {
        Phase ph("merge.rle_write", st);
        RB3_LAUNCH(k_rle_merge<true>, nb_for(ns, 128), 128, 0, st, V1, V2, codes2.as<uint8_t>(), pos, n2, nM, ns,
                   off.as<uint64_t>(), (uint64_t *)nullptr, runs.as<uint64_t>(), out->gbase, out->blocks,
                   out->payload);
    }
    // the merged image passes the same checks as one read from a file
    return rle_check_impl(out, st);
}

// Owns a temporary index.
struct TmpIndex {
    rb3_index *p = nullptr;
    ~TmpIndex() {
        if (p) rb3_index_free(p);
    }
};

int merge_any(rb3_index *dst, const rb3_index *src, const rb3_opts &o, cudaStream_t st) {
    if (!src->rle) return merge_impl(dst, src, o, st);  // a run-length dst is merged into as it is
    RB3_CHECK_ARG(dst != src, "dst and src must differ");
    // the walk reads B2's LF (a run-length index has no build data): a plain copy of it
    TmpIndex Q;
    Q.p = new rb3_index();
    RB3_TRY(decompress_impl(src, st, Q.p));
    return merge_impl(dst, Q.p, o, st);
}

}  // namespace rb3

using namespace rb3;

RB3_EXPORT int rb3_index_compress(const rb3_index *src, int32_t span, void *stream, rb3_index **out) {
    set_error("%s", "");
    RB3_CHECK_ARG(src && out, "NULL argument");
    *out = nullptr;
    const int S = span ? span : kDefaultRleSpan;
    RB3_CHECK_ARG(valid_rle_span(S), "span must be a power of two from 512 to 16384");
    RB3_CHECK_ARG(!src->rle, "the index is already run-length encoded");
    cudaStream_t st = (cudaStream_t)stream;
    rb3_index *x = new rb3_index();
    const int r = compress_impl(src, S, st, x);
    if (r != RB3_OK) {
        cudaStreamSynchronize(st);
        rb3_index_free(x);
        return r;
    }
    *out = x;
    return RB3_OK;
}

RB3_EXPORT int rb3_index_bytes(const rb3_index *idx, int64_t *device_bytes, int64_t *runs) {
    set_error("%s", "");
    RB3_CHECK_ARG(idx != nullptr, "NULL index");
    int64_t b = idx->nblocks * (int64_t)idx->block_bytes;
    if (idx->rle) b += idx->payload_bytes + 16;
    if (idx->gbase) b += (int64_t)sizeof(int64_t) * 5 * gbase_rows(idx->n);
    if (idx->sa_s && idx->sdir) b += (int64_t)sizeof(uint64_t) * (2 * (idx->n / 64 + 1) + idx->n_samples);
    if (device_bytes) *device_bytes = b;
    if (runs) *runs = idx->rle ? idx->runs : -1;
    return RB3_OK;
}
