// Autotuner.  The merge's segment length trades seed work against walk
// parallelism, its seed cap trades seed work against candidate walks and
// second walks of unconverged segments, the SMEM search's chunk length trades
// load balance against the chunks' extra first steps, and its hot-level depth
// trades table bytes (32 B x 4^K / 0.75) against the extensions a table read
// replaces; the best values depend on the inputs' shape.
// rb3_tune_merge / rb3_tune_search time candidates on the caller's own inputs
// (the merge's walk phase runs into scratch, so the index is not modified) and
// remember the winner per input shape: device, Occ interval, strand mode and
// the log2 size classes of the inputs.  rb3_merge and rb3_mem_search use a
// remembered value whenever the caller leaves the knob at 0.  With the
// environment variable RB3_TUNE_FILE set, choices are also appended to that
// file and read back by later processes.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"

namespace rb3 {

namespace {
using Key = std::tuple<int, int, int, int, int, int, int>;  // kind, dev, D, single, c1, c2, c3
std::mutex g_mu;
std::map<Key, int64_t> g_cache;
bool g_loaded = false;

int size_class(int64_t x) { return x <= 1 ? 0 : ilog2(x); }

void load_file_locked() {
    if (g_loaded) return;
    g_loaded = true;
    const char *path = getenv("RB3_TUNE_FILE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    int k, d, D, s, c1, c2, c3;
    long long v;
    while (fscanf(f, "%d %d %d %d %d %d %d %lld", &k, &d, &D, &s, &c1, &c2, &c3, &v) == 8)
        g_cache[Key(k, d, D, s, c1, c2, c3)] = v;
    fclose(f);
}

void store(const Key &key, int64_t v) {
    std::lock_guard<std::mutex> lk(g_mu);
    load_file_locked();
    g_cache[key] = v;
    if (const char *path = getenv("RB3_TUNE_FILE")) {
        if (FILE *f = fopen(path, "a")) {
            fprintf(f, "%d %d %d %d %d %d %d %lld\n", std::get<0>(key), std::get<1>(key), std::get<2>(key),
                    std::get<3>(key), std::get<4>(key), std::get<5>(key), std::get<6>(key), (long long)v);
            fclose(f);
        }
    }
}

int64_t lookup(const Key &key) {
    std::lock_guard<std::mutex> lk(g_mu);
    load_file_locked();
    auto it = g_cache.find(key);
    return it == g_cache.end() ? 0 : it->second;
}

Key merge_key(const rb3_index *dst, const rb3_index *src) {
    int dev = 0;
    cudaGetDevice(&dev);
    return Key(0, dev, dst->D, dst->single_strand, size_class(dst->n), size_class(src->n), size_class(src->m));
}

Key search_key(const rb3_index *idx, int64_t nq, int64_t total_q) {
    int dev = 0;
    cudaGetDevice(&dev);
    return Key(1, dev, idx->D, 0, size_class(idx->n), size_class(nq ? total_q / nq : 0), size_class(nq));
}
}  // namespace

int64_t tuned_seg_len(const rb3_index *dst, const rb3_index *src) { return lookup(merge_key(dst, src)); }

int64_t tuned_seed_cap(const rb3_index *dst, const rb3_index *src) {
    Key k = merge_key(dst, src);
    std::get<0>(k) = 2;
    return lookup(k);
}

int64_t tuned_chunk_len(const rb3_index *idx, int64_t nq, int64_t total_q) {
    return lookup(search_key(idx, nq, total_q));
}

int64_t tuned_hot_depth(const rb3_index *idx, int64_t nq, int64_t total_q) {
    Key k = search_key(idx, nq, total_q);
    std::get<0>(k) = 3;
    return lookup(k);
}

static int time_ms(cudaStream_t st, float *ms, const std::function<int()> &fn) {
    cudaEvent_t a, b;
    RB3_CUDA_TRY(cudaEventCreate(&a));
    RB3_CUDA_TRY(cudaEventCreate(&b));
    RB3_CUDA_TRY(cudaEventRecord(a, st));
    int r = fn();
    RB3_CUDA_TRY(cudaEventRecord(b, st));
    RB3_CUDA_TRY(cudaEventSynchronize(b));
    RB3_CUDA_TRY(cudaEventElapsedTime(ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return r;
}

int tune_merge(const rb3_index *dst, const rb3_index *src, const rb3_opts &base, rb3_opts *best, double *best_ms,
               cudaStream_t st) {
    *best = base;
    if (dst->n == 0 || src->n == 0 || !src->text || !src->isa) return RB3_OK;  // nothing to tune
    DevBuf pos;
    RB3_TRY(pos.alloc(sizeof(int64_t) * src->n, st));
    int64_t L0 = src->n / ((int64_t)num_sms() * 512);
    if (L0 < 512) L0 = 512;
    // segment lengths around the default, each with seed caps of 1, 2 and 4
    // segment lengths (the bounded-seed forms; the chain form takes no cap)
    std::vector<std::pair<int64_t, int64_t>> cand;
    rb3_opts o = base;
    if (o.merge_form != 2 && o.merge_form != 3) o.merge_form = 0;  // a segmented form
    for (int64_t L : {L0 / 2, L0, 2 * L0, 4 * L0}) {
        if (L < 256 || L > 65536) continue;
        if (base.seed_cap > 0 || o.merge_form == 3)
            cand.push_back({L, base.seed_cap});
        else
            for (int64_t c : {L, 2 * L, 4 * L}) cand.push_back({L, c});
    }
    o.seg_len = L0;
    o.seed_cap = base.seed_cap;
    RB3_TRY(merge_positions(dst, src, o, st, pos.as<int64_t>()));  // warm-up
    float bestt = 1e30f;
    int64_t bestL = L0, bestC = base.seed_cap;
    for (const auto &lc : cand) {
        o.seg_len = lc.first;
        o.seed_cap = lc.second;
        float t = 0.f;
        RB3_TRY(time_ms(st, &t, [&] { return merge_positions(dst, src, o, st, pos.as<int64_t>()); }));
        if (t < bestt) {
            bestt = t;
            bestL = lc.first;
            bestC = lc.second;
        }
    }
    Key k = merge_key(dst, src);
    store(k, bestL);
    if (bestC > 0 && o.merge_form != 3) {
        std::get<0>(k) = 2;
        store(k, bestC);
    }
    best->seg_len = bestL;
    best->seed_cap = bestC;
    if (best_ms) *best_ms = bestt;
    return RB3_OK;
}

int tune_search(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, const int64_t *qoff_host, int64_t nq,
                int64_t total_q, int32_t min_len, int64_t min_occ, const rb3_opts &base, rb3_opts *best,
                double *best_ms, cudaStream_t st) {
    *best = base;
    if (nq == 0) return RB3_OK;
    int64_t cap = total_q / 8 + 4096;
    DevBuf out;
    RB3_TRY(out.alloc(sizeof(rb3_smem) * cap, st));
    rb3_opts o = base;
    int64_t n = 0;
    o.search_form = 0;
    o.chunk_len = 256;
    int r = mem_search_impl(idx, q, qoff, qoff_host, nq, total_q, min_len, min_occ, o, out.as<rb3_smem>(), cap, &n,
                            st);  // warm-up; also sizes the output
    if (r == RB3_E_CAPACITY) {
        cap = n + 4096;
        RB3_TRY(out.alloc(sizeof(rb3_smem) * cap, st));
        r = mem_search_impl(idx, q, qoff, qoff_host, nq, total_q, min_len, min_occ, o, out.as<rb3_smem>(), cap, &n, st);
    }
    RB3_TRY(r);
    float bestt = 1e30f;
    int64_t bestC = 256;
    for (int64_t C : {64, 128, 256, 512, 1024, 4096}) {
        o.chunk_len = C;
        float t = 0.f;
        RB3_TRY(time_ms(st, &t, [&] {
            return mem_search_impl(idx, q, qoff, qoff_host, nq, total_q, min_len, min_occ, o, out.as<rb3_smem>(), cap,
                                   &n, st);
        }));
        if (t < bestt) {
            bestt = t;
            bestC = C;
        }
    }
    store(search_key(idx, nq, total_q), bestC);
    best->search_form = 0;
    best->chunk_len = bestC;
    // then the hot-level table's depth at that chunk length (each table is
    // built by an untimed call first; -1 = none)
    if (base.hot_depth == 0) {
        o.chunk_len = bestC;
        int bestK = -1;
        float bestkt = 1e30f;
        for (int K : {-1, 6, 8, 10}) {
            o.hot_depth = K;
            RB3_TRY(mem_search_impl(idx, q, qoff, qoff_host, nq, total_q, min_len, min_occ, o, out.as<rb3_smem>(),
                                    cap, &n, st));
            for (int rep = 0; rep < 2; ++rep) {  // the better of two timings (the gaps are a few %)
                float t = 0.f;
                RB3_TRY(time_ms(st, &t, [&] {
                    return mem_search_impl(idx, q, qoff, qoff_host, nq, total_q, min_len, min_occ, o,
                                           out.as<rb3_smem>(), cap, &n, st);
                }));
                if (t < bestkt) {
                    bestkt = t;
                    bestK = K;
                }
            }
        }
        Key k = search_key(idx, nq, total_q);
        std::get<0>(k) = 3;
        store(k, bestK);
        best->hot_depth = bestK;
        bestt = bestkt;
    }
    if (best_ms) *best_ms = bestt;
    return RB3_OK;
}

// Layout tuner for a whole incremental build (rb3_tune_build): batch 1 built
// and merged into batch 0 at each Occ interval D, each with the merge tuner's
// segment length and seed cap; the fastest D whose projected index fits the
// budget wins.  Bytes per symbol of a plain index: block bytes / D (32 B per 32
// symbols at D = 32, 64 B per 64, 96 B per 128).
static const int kTuneD[3] = {32, 64, 128};

int tune_build(const uint8_t *seq_dev, const std::vector<int64_t> &lens, const std::vector<int64_t> &ends,
               const rb3_opts &base, int64_t index_mb, rb3_opts *best, double cand_ms[3], double cand_mb[3],
               cudaStream_t st) {
    *best = base;
    if (ends.size() < 2 || ends[0] == 0 || ends[1] == ends[0]) return RB3_OK;  // needs two non-empty batches
    int64_t off1 = 0, total_sym = 0;
    for (int64_t i = 0; i < ends[0]; ++i) off1 += lens[i];
    for (size_t i = 0; i < lens.size(); ++i) total_sym += (lens[i] + 1) * (base.single_strand ? 1 : 2);
    float bestt = 1e30f, smallest = 1e30f;
    int bestD = kDefaultOccInterval, smallD = kDefaultOccInterval;
    rb3_opts bo = base;
    for (int c = 0; c < 3; ++c) {
        const int D = kTuneD[c];
        rb3_opts o = base;
        o.occ_interval = D;
        o.seg_len = 0;
        o.seed_cap = 0;
        rb3_index *A = new rb3_index(), *B = new rb3_index();
        auto done = [&](int r) {
            rb3_index_free(A);
            rb3_index_free(B);
            return r;
        };
        cudaGetDevice(&A->device);
        B->device = A->device;
        int r = build_batch_impl(seq_dev, lens.data(), ends[0], o, st, A);
        float tb = 0.f;
        if (r == RB3_OK)
            r = time_ms(st, &tb, [&] {
                return build_batch_impl(seq_dev + off1, lens.data() + ends[0], ends[1] - ends[0], o, st, B);
            });
        rb3_opts tuned = o;
        double walk_ms = 0;
        if (r == RB3_OK) r = tune_merge(A, B, o, &tuned, &walk_ms, st);
        float tm = 0.f;
        if (r == RB3_OK) r = time_ms(st, &tm, [&] { return merge_impl(A, B, tuned, st); });
        if (r != RB3_OK) return done(r);
        const double mb = (double)total_sym * block_bytes_for(D) / D / 1048576.0;
        cand_ms[c] = (double)(tb + tm);
        cand_mb[c] = mb;
        if ((index_mb <= 0 || mb <= (double)index_mb) && tb + tm < bestt) {
            bestt = tb + tm;
            bestD = D;
            bo = tuned;
        }
        if (mb < smallest) {
            smallest = (float)mb;
            smallD = D;
            if (bestt >= 1e30f) bo = tuned;
        }
        done(RB3_OK);
    }
    if (bestt >= 1e30f) bestD = smallD;  // nothing fits: the smallest layout
    *best = bo;
    best->occ_interval = bestD;
    return RB3_OK;
}

}  // namespace rb3

using namespace rb3;

RB3_EXPORT int rb3_tune_build(const uint8_t *seq, const int64_t *len, int64_t n_seq, const int64_t *batch_end,
                              int64_t n_batches, const rb3_opts *base, int64_t index_mb, rb3_opts *best,
                              double *cand_ms, double *cand_mb, void *stream) {
    set_error("%s", "");
    RB3_CHECK_ARG(best && len && batch_end && n_seq >= 0 && n_batches >= 2, "bad argument (two batches needed)");
    rb3_opts o;
    rb3_opts_default(&o);
    if (base) o = *base;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int64_t> lens(n_seq), ends(n_batches);
    if (is_device_ptr(len)) RB3_CUDA_TRY(cudaMemcpy(lens.data(), len, sizeof(int64_t) * n_seq, cudaMemcpyDeviceToHost));
    else memcpy(lens.data(), len, sizeof(int64_t) * n_seq);
    if (is_device_ptr(batch_end))
        RB3_CUDA_TRY(cudaMemcpy(ends.data(), batch_end, sizeof(int64_t) * n_batches, cudaMemcpyDeviceToHost));
    else memcpy(ends.data(), batch_end, sizeof(int64_t) * n_batches);
    int64_t prev = 0;
    for (int64_t b = 0; b < n_batches; ++b) {
        RB3_CHECK_ARG(ends[b] >= prev && ends[b] <= n_seq, "batch_end must be non-decreasing and <= n_seq");
        prev = ends[b];
    }
    int64_t two = 0;
    for (int64_t i = 0; i < ends[1]; ++i) {
        RB3_CHECK_ARG(lens[i] >= 0, "negative string length");
        two += lens[i];
    }
    RB3_CHECK_ARG(two == 0 || seq != nullptr, "seq is NULL");
    // the first two batches on the device
    const uint8_t *sd = seq;
    DevBuf copy;
    if (two > 0 && !is_device_ptr(seq)) {
        RB3_TRY(copy.alloc((size_t)two, st));
        RB3_CUDA_TRY(cudaMemcpyAsync(copy.p, seq, (size_t)two, cudaMemcpyHostToDevice, st));
        sd = copy.as<uint8_t>();
    }
    double ms[3] = {0, 0, 0}, mb[3] = {0, 0, 0};
    RB3_TRY(tune_build(sd, lens, ends, o, index_mb, best, ms, mb, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    for (int c = 0; c < 3; ++c) {
        if (cand_ms) cand_ms[c] = ms[c];
        if (cand_mb) cand_mb[c] = mb[c];
    }
    return RB3_OK;
}

RB3_EXPORT int rb3_tune_merge(const rb3_index *dst, const rb3_index *src, const rb3_opts *base, rb3_opts *best,
                              double *best_ms, void *stream) {
    set_error("%s", "");
    RB3_CHECK_ARG(dst && src && best, "NULL argument");
    RB3_CHECK_ARG(!src->rle, "the batch merged in must be a plain index");
    rb3_opts o;
    rb3_opts_default(&o);
    if (base) o = *base;
    cudaStream_t st = (cudaStream_t)stream;
    RB3_TRY(tune_merge(dst, src, o, best, best_ms, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    return RB3_OK;
}

RB3_EXPORT int rb3_tune_search(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, int64_t nq, int32_t min_len,
                               int64_t min_occ, const rb3_opts *base, rb3_opts *best, double *best_ms, void *stream) {
    set_error("%s", "");
    RB3_CHECK_ARG(idx && best && qoff && nq >= 0, "bad argument");
    RB3_CHECK_ARG(min_len >= 1 && min_occ >= 1, "min_len and min_occ must be >= 1");
    RB3_CHECK_ARG(!idx->single_strand, "SMEM search needs a double-strand index");
    RB3_CHECK_ARG(is_device_ptr(qoff) && (nq == 0 || is_device_ptr(q)), "q and qoff must be device pointers");
    rb3_opts o;
    rb3_opts_default(&o);
    if (base) o = *base;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int64_t> qo(nq + 1);
    RB3_CUDA_TRY(cudaMemcpy(qo.data(), qoff, sizeof(int64_t) * (nq + 1), cudaMemcpyDeviceToHost));
    RB3_TRY(tune_search(idx, q, qoff, qo.data(), nq, qo[nq], min_len, min_occ, o, best, best_ms, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    return RB3_OK;
}
