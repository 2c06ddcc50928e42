// Locating suffixes (Section "Locating with FM-index", Algorithm 2).
//
// The paper stores S(i) for rows i that are multiples of s and reaches one of
// them by LF steps.  Here the sample is taken by text position instead: a row is
// sampled when its suffix starts at an offset of its string that is a multiple
// of s.  That set does not move when a batch is merged in (rows move, texts do
// not), so a merge only interleaves the two inputs' samples the way it
// interleaves their rows (sample_merge, merge.cu); and since offset 0 of every
// string is sampled, a walk back from any row meets a sampled row within s - 1
// LF steps without crossing into the previous string, so the sentinel-rank
// array R of Algorithm 2 is not needed.  A located row is reported, as in the
// paper, as (string index, offset on the string): string t of the index is
// the t-th sentinel-terminated string of its concatenation (P0, rc(P0), P1,
// ... for a double-strand index).
#include "common.cuh"

namespace rb3 {

static inline unsigned nb_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// String of text position p (str_end ascending: the sentinel position ending
// each string) and the offset of p on it.
__device__ __forceinline__ void string_of(const int64_t *__restrict__ str_end, int64_t ns, int64_t p, int64_t *t,
                                          int64_t *off) {
    int64_t lo = -1, hi = ns - 1;  // smallest s with str_end[s] >= p
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (str_end[mid] >= p) hi = mid;
        else lo = mid;
    }
    *t = hi;
    *off = p - (hi == 0 ? 0 : str_end[hi - 1] + 1);
}

// One thread per 64 rows: the bit set of sampled rows and its count.
__global__ void k_sample_words(const int32_t *__restrict__ SA, int64_t n, const int64_t *__restrict__ str_end,
                               int64_t ns, int64_t s, int64_t nwords, uint64_t *__restrict__ sdir,
                               uint64_t *__restrict__ cnt) {
    const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w >= nwords) return;
    uint64_t bits = 0;
    const int64_t r0 = w * 64, r1 = r0 + 64 < n ? r0 + 64 : n;
    for (int64_t r = r0; r < r1; ++r) {
        int64_t t, off;
        string_of(str_end, ns, SA[r], &t, &off);
        if ((off & (s - 1)) == 0) bits |= 1ull << (r - r0);
    }
    sdir[2 * w] = bits;
    cnt[w] = __popcll(bits);
}

__global__ void k_sample_fill(const int32_t *__restrict__ SA, const int64_t *__restrict__ str_end, int64_t ns,
                              const uint64_t *__restrict__ excl, int64_t nwords, uint64_t *__restrict__ sdir,
                              uint64_t *__restrict__ svals) {
    const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w >= nwords) return;
    const uint64_t base = excl[w];
    sdir[2 * w + 1] = base;
    uint64_t bits = sdir[2 * w];
    uint64_t o = base;
    while (bits) {
        const int b = __ffsll((long long)bits) - 1;
        bits &= bits - 1;
        int64_t t, off;
        string_of(str_end, ns, SA[w * 64 + b], &t, &off);
        svals[o++] = ((uint64_t)t << SVAL_OFF_BITS) | (uint64_t)off;
    }
}

void free_samples(rb3_index *x) {
    dev_free(x->sdir, 0);
    dev_free(x->svals, 0);
    x->sdir = nullptr;
    x->svals = nullptr;
    x->n_samples = 0;
}

int sample_batch(rb3_index *x, const int32_t *SA, cudaStream_t st) {
    const int64_t n = x->n, ns = (int64_t)x->str_end.size(), s = x->sa_s;
    const int64_t nwords = n / 64 + 1;
    RB3_TRY(dev_alloc((void **)&x->sdir, sizeof(uint64_t) * 2 * nwords, st));
    RB3_CUDA_TRY(cudaMemsetAsync(x->sdir, 0, sizeof(uint64_t) * 2 * nwords, st));
    DevBuf ends, cnt, excl;
    RB3_TRY(ends.alloc(sizeof(int64_t) * (ns > 0 ? ns : 1), st));
    RB3_TRY(cnt.alloc(sizeof(uint64_t) * nwords, st));
    RB3_TRY(excl.alloc(sizeof(uint64_t) * nwords, st));
    if (ns > 0)
        RB3_CUDA_TRY(cudaMemcpyAsync(ends.p, x->str_end.data(), sizeof(int64_t) * ns, cudaMemcpyHostToDevice, st));
    RB3_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(uint64_t) * nwords, st));
    if (n > 0)
        RB3_LAUNCH(k_sample_words, nb_for(nwords, 256), 256, 0, st, SA, n, ends.as<int64_t>(), ns, s, nwords, x->sdir,
                   cnt.as<uint64_t>());
    RB3_TRY(scan_u64(cnt.as<uint64_t>(), excl.as<uint64_t>(), nwords, false, st));
    int64_t tail[2];
    RB3_CUDA_TRY(cudaMemcpyAsync(&tail[0], excl.as<uint64_t>() + nwords - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaMemcpyAsync(&tail[1], cnt.as<uint64_t>() + nwords - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    x->n_samples = tail[0] + tail[1];
    RB3_TRY(dev_alloc((void **)&x->svals, sizeof(uint64_t) * (x->n_samples > 0 ? x->n_samples : 1), st));
    RB3_LAUNCH(k_sample_fill, nb_for(nwords, 256), 256, 0, st, SA, ends.as<int64_t>(), ns, excl.as<uint64_t>(),
               nwords, x->sdir, x->svals);
    return RB3_OK;
}

// One thread per row: LF steps back until a sampled row (at most s - 1).
template <int NS>
__global__ void k_locate(OccView V, const uint64_t *__restrict__ sdir, const uint64_t *__restrict__ svals, int64_t s,
                         const int64_t *__restrict__ rows, int64_t nr, int64_t *__restrict__ out,
                         unsigned int *__restrict__ err) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nr) return;
    int64_t j = rows[i];
    if (j < 0 || j >= V.n) {
        atomicOr(err, 1u);
        out[2 * i] = out[2 * i + 1] = -1;
        return;
    }
    for (int64_t k = 0; k < s; ++k) {
        int64_t vi;
        if (sample_at(sdir, j, &vi)) {
            const uint64_t v = svals[vi];
            out[2 * i] = (int64_t)(v >> SVAL_OFF_BITS);
            out[2 * i + 1] = (int64_t)(v & ((1ull << SVAL_OFF_BITS) - 1)) + k;
            return;
        }
        int a;
        int64_t r;
        if constexpr (NS == 0) {  // symbol and rank from the one sector of the block
            const BlockLd<0> b = block_load<0>(V, j);
            a = (int)(((b.h.w[5] >> b.o) & 1u) | (((b.h.w[6] >> b.o) & 1u) << 1) | (((b.h.w[7] >> b.o) & 1u) << 2));
            r = block_rank<0>(b, a);
        } else if constexpr (NS == NS_RLE) {  // symbol and rank from one decode of the span
            const BlockLd<NS_RLE> b = block_load<NS_RLE>(V, j);
            a = b.sym;
            r = block_rank<NS_RLE>(b, a);
        } else {
            a = sym_at(V, j);
            r = rank1<NS>(V, a, j);
        }
        j = C_of(V, a) + r;  // pi(j): the row of the suffix one position earlier
    }
    atomicOr(err, 2u);  // no sampled row within s steps: the sample is inconsistent
    out[2 * i] = out[2 * i + 1] = -1;
}

int locate_impl(const rb3_index *idx, const int64_t *rows, int64_t nr, int64_t *out, cudaStream_t st) {
    if (nr == 0) return RB3_OK;
    DevBuf err;
    RB3_TRY(err.alloc(sizeof(unsigned int), st));
    RB3_CUDA_TRY(cudaMemsetAsync(err.p, 0, sizeof(unsigned int), st));
    {
        Phase ph("k.locate", st);
        RB3_WITH_NS(idx->D, RB3_LAUNCH(k_locate<NS>, nb_for(nr, 128), 128, 0, st, occ_view(idx), idx->sdir,
                                       idx->svals, (int64_t)idx->sa_s, rows, nr, out, err.as<unsigned int>()));
    }
    unsigned int h = 0;
    RB3_CUDA_TRY(cudaMemcpyAsync(&h, err.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    if (h & 1u) {
        set_error("locate: a row outside [0, n)");
        return RB3_E_INVAL;
    }
    if (h) {
        set_error("locate: no sampled row within the sample rate (corrupt sample)");
        return RB3_E_CUDA;
    }
    return RB3_OK;
}

}  // namespace rb3

using namespace rb3;

RB3_EXPORT int rb3_locate(const rb3_index *idx, const int64_t *rows, int64_t n_rows, int64_t *out, void *stream) {
    set_error("%s", "");
    RB3_CHECK_ARG(idx && n_rows >= 0 && (n_rows == 0 || (rows && out)), "bad argument");
    RB3_CHECK_ARG(idx->sa_s > 0 && idx->sdir, "the index keeps no sampled suffix array (build with sa_sample)");
    cudaStream_t st = (cudaStream_t)stream;
    if (n_rows == 0) return RB3_OK;
    const bool rdev = is_device_ptr(rows), odev = is_device_ptr(out);
    DevBuf drows, dout;
    const int64_t *r = rows;
    int64_t *o = out;
    if (!rdev) {
        RB3_TRY(drows.alloc(sizeof(int64_t) * n_rows, st));
        RB3_CUDA_TRY(cudaMemcpyAsync(drows.p, rows, sizeof(int64_t) * n_rows, cudaMemcpyHostToDevice, st));
        r = drows.as<int64_t>();
    }
    if (!odev) {
        RB3_TRY(dout.alloc(sizeof(int64_t) * 2 * n_rows, st));
        o = dout.as<int64_t>();
    }
    RB3_TRY(locate_impl(idx, r, n_rows, o, st));
    if (!odev) {
        RB3_CUDA_TRY(cudaMemcpyAsync(out, o, sizeof(int64_t) * 2 * n_rows, cudaMemcpyDeviceToHost, st));
        RB3_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return RB3_OK;
}
