// Autotuner.  The merge's segment length trades seed work against walk
// parallelism, its seed cap trades seed work against candidate walks and
// second walks of unconverged segments, and the SMEM search's chunk length
// trades load balance against the chunks' extra first steps; the best values
// depend on the inputs' shape.
// rb3_tune_merge / rb3_tune_search time candidates on the caller's own inputs
// (the merge's walk phase runs into scratch, so the index is not modified) and
// remember the winner per input shape: device, Occ interval, strand mode and
// the log2 size classes of the inputs.  rb3_merge and rb3_mem_search use a
// remembered value whenever the caller leaves the knob at 0.  With the
// environment variable RB3_TUNE_FILE set, choices are also appended to that
// file and read back by later processes.
#include <cmath>
#include <cstdlib>
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
    if (best_ms) *best_ms = bestt;
    return RB3_OK;
}

}  // namespace rb3

using namespace rb3;

RB3_EXPORT int rb3_tune_merge(const rb3_index *dst, const rb3_index *src, const rb3_opts *base, rb3_opts *best,
                              double *best_ms, void *stream) {
    set_error("%s", "");
    RB3_CHECK_ARG(dst && src && best, "NULL argument");
    RB3_CHECK_ARG(!dst->rle && !src->rle, "merge tuning needs plain-layout indexes");
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
