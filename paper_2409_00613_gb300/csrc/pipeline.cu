// Incremental construction driver: build the BWT of each batch and merge it
// into the index, one batch after another (the driver loop of Section
// "Methods"), with the build of batch b+1 on the device while batch b is being
// merged -- the paper runs BWT merge and partial BWT construction together
// (Table 2, note 7) to keep its threads busy when few, long strings leave the
// merge with little parallelism.  On one GPU the two run on separate streams
// from two host threads.  At most one built batch waits for its merge while
// the next is being built, which bounds the extra memory to two batches'
// indexes and build data.
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>

#include "common.cuh"

namespace rb3 {

namespace {

struct Built {
    rb3_index *idx = nullptr;
    int code = RB3_OK;
    std::string err;
};

struct Channel {
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Built> q;
    bool stop = false;  // consumer gave up
};

void free_built(rb3_index *x) {
    if (!x) return;
    dev_free(x->blocks, 0);
    dev_free(x->gbase, 0);
    free_samples(x);
    dev_free(x->text, 0);
    dev_free(x->isa, 0);
    cudaStreamSynchronize(0);
    delete x;
}

}  // namespace

int append_batches(rb3_index *dst, const uint8_t *seq, const int64_t *lens, int64_t n_seq, const int64_t *batch_end,
                   int64_t n_batches, const rb3_opts &o, cudaStream_t caller) {
    int dev = 0;
    RB3_CUDA_TRY(cudaGetDevice(&dev));
    std::vector<int64_t> off(n_seq + 1, 0);
    for (int64_t i = 0; i < n_seq; ++i) off[i + 1] = off[i] + lens[i];
    const bool seq_dev = off[n_seq] == 0 || is_device_ptr(seq);
    cudaStream_t sb = nullptr, sm = nullptr;
    cudaEvent_t start = nullptr;
    // builds first: the merge walk's long chains fill what the next batch's
    // build leaves free (measured 2-3 % faster than the merge first)
    int prio_low = 0, prio_high = 0;
    RB3_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
    RB3_CUDA_TRY(cudaStreamCreateWithPriority(&sb, cudaStreamNonBlocking, prio_high));
    RB3_CUDA_TRY(cudaStreamCreateWithPriority(&sm, cudaStreamNonBlocking, prio_low));
    RB3_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    // host strings: the next batch's copy runs on its own stream while the
    // current batch builds (two staging buffers, an event per copy)
    cudaStream_t sc = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr};
    if (!seq_dev) {
        RB3_CUDA_TRY(cudaStreamCreateWithPriority(&sc, cudaStreamNonBlocking, prio_high));
        RB3_CUDA_TRY(cudaEventCreateWithFlags(&copied[0], cudaEventDisableTiming));
        RB3_CUDA_TRY(cudaEventCreateWithFlags(&copied[1], cudaEventDisableTiming));
    }
    // the internal streams start after the work already on the caller's stream
    RB3_CUDA_TRY(cudaEventRecord(start, caller));
    RB3_CUDA_TRY(cudaStreamWaitEvent(sb, start, 0));
    RB3_CUDA_TRY(cudaStreamWaitEvent(sm, start, 0));
    if (sc) RB3_CUDA_TRY(cudaStreamWaitEvent(sc, start, 0));

    Channel ch;
    std::thread builder([&] {
        cudaSetDevice(dev);
        DevBuf stage[2];
        // copy of batch b's strings into stage[b & 1] on sc, marked by copied[b & 1]
        auto issue_copy = [&](int64_t b) -> int {
            const int64_t s0 = b == 0 ? 0 : batch_end[b - 1], s1 = batch_end[b];
            const size_t bytes = (size_t)(off[s1] - off[s0]);
            if (bytes == 0) return RB3_OK;
            RB3_TRY(stage[b & 1].alloc(bytes, sc));  // its last reader, batch b - 2's build, is done
            RB3_CUDA_TRY(cudaMemcpyAsync(stage[b & 1].p, seq + off[s0], bytes, cudaMemcpyHostToDevice, sc));
            RB3_CUDA_TRY(cudaEventRecord(copied[b & 1], sc));
            return RB3_OK;
        };
        int rc = (!seq_dev && n_batches > 0) ? issue_copy(0) : RB3_OK;
        for (int64_t b = 0; b < n_batches; ++b) {
            const int64_t s0 = b == 0 ? 0 : batch_end[b - 1], s1 = batch_end[b];
            Built out;
            rb3_index *x = new rb3_index();
            x->device = dev;
            int r = rc;
            const uint8_t *src = seq + off[s0];
            const size_t bytes = (size_t)(off[s1] - off[s0]);
            if (r == RB3_OK && !seq_dev && bytes) {
                if (cudaStreamWaitEvent(sb, copied[b & 1], 0) != cudaSuccess)
                    r = cuda_fail(cudaGetLastError(), "append: wait for copy", __FILE__, __LINE__);
                src = stage[b & 1].as<uint8_t>();
            }
            if (r == RB3_OK && !seq_dev && b + 1 < n_batches) r = issue_copy(b + 1);  // overlaps this build
            if (r == RB3_OK) r = build_batch_impl(src, lens + s0, s1 - s0, o, sb, x);
            if (r == RB3_OK && cudaStreamSynchronize(sb) != cudaSuccess)
                r = cuda_fail(cudaGetLastError(), "append: build", __FILE__, __LINE__);
            if (r != RB3_OK) {
                out.code = r;
                out.err = rb3_last_error_str();
                free_built(x);
            } else {
                out.idx = x;
            }
            std::unique_lock<std::mutex> lk(ch.mu);
            // hand over; wait while one built batch is already waiting for its merge
            ch.cv.wait(lk, [&] { return ch.stop || ch.q.size() < 1; });
            if (ch.stop) {
                free_built(out.idx);
                return;
            }
            ch.q.push_back(std::move(out));
            ch.cv.notify_all();
            if (r != RB3_OK) return;
        }
    });

    int result = RB3_OK;
    std::string err;
    for (int64_t b = 0; b < n_batches; ++b) {
        Built got;
        {
            std::unique_lock<std::mutex> lk(ch.mu);
            ch.cv.wait(lk, [&] { return !ch.q.empty(); });
            got = std::move(ch.q.front());
            ch.q.pop_front();
            ch.cv.notify_all();
        }
        if (got.code != RB3_OK) {
            result = got.code;
            err = got.err;
            break;
        }
        {
            Phase ph("append.merge", sm);
            result = merge_impl(dst, got.idx, o, sm);
        }
        if (result == RB3_OK && cudaStreamSynchronize(sm) != cudaSuccess)
            result = cuda_fail(cudaGetLastError(), "append: merge", __FILE__, __LINE__);
        free_built(got.idx);
        if (result != RB3_OK) {
            err = rb3_last_error_str();
            break;
        }
    }
    {
        std::lock_guard<std::mutex> lk(ch.mu);
        ch.stop = true;
        for (auto &g : ch.q) free_built(g.idx);
        ch.q.clear();
        ch.cv.notify_all();
    }
    builder.join();
    cudaStreamSynchronize(sb);
    cudaStreamSynchronize(sm);
    cudaStreamDestroy(sb);
    cudaStreamDestroy(sm);
    if (sc) {
        cudaStreamSynchronize(sc);
        cudaStreamDestroy(sc);
        cudaEventDestroy(copied[0]);
        cudaEventDestroy(copied[1]);
    }
    cudaEventDestroy(start);
    if (result != RB3_OK) set_error("%s", err.c_str());
    return result;
}

}  // namespace rb3

using namespace rb3;

RB3_EXPORT int rb3_append_batches(rb3_index *dst, const uint8_t *seq, const int64_t *len, int64_t n_seq,
                                  const int64_t *batch_end, int64_t n_batches, const rb3_opts *o, void *stream) {
    set_error("%s", "");
    RB3_CHECK_ARG(dst != nullptr, "NULL index");
    RB3_CHECK_ARG(n_seq >= 0 && n_batches >= 0, "negative size");
    if (n_batches == 0) return RB3_OK;
    RB3_CHECK_ARG(batch_end != nullptr && (n_seq == 0 || len != nullptr), "NULL argument");
    rb3_opts opts;
    rb3_opts_default(&opts);
    if (o) opts = *o;
    RB3_CHECK_ARG(dst->n == 0 || dst->single_strand == opts.single_strand,
                  "strand mode of the batches differs from the index's");
    std::vector<int64_t> lens(n_seq), ends(n_batches);
    cudaStream_t st = (cudaStream_t)stream;
    if (n_seq) {
        if (is_device_ptr(len)) RB3_CUDA_TRY(cudaMemcpy(lens.data(), len, sizeof(int64_t) * n_seq, cudaMemcpyDeviceToHost));
        else memcpy(lens.data(), len, sizeof(int64_t) * n_seq);
    }
    if (is_device_ptr(batch_end))
        RB3_CUDA_TRY(cudaMemcpy(ends.data(), batch_end, sizeof(int64_t) * n_batches, cudaMemcpyDeviceToHost));
    else
        memcpy(ends.data(), batch_end, sizeof(int64_t) * n_batches);
    int64_t prev = 0, total = 0;
    for (int64_t b = 0; b < n_batches; ++b) {
        RB3_CHECK_ARG(ends[b] >= prev && ends[b] <= n_seq, "batch_end must be non-decreasing and <= n_seq");
        prev = ends[b];
    }
    RB3_CHECK_ARG(ends[n_batches - 1] == n_seq, "batch_end[n_batches-1] must be n_seq");
    for (int64_t i = 0; i < n_seq; ++i) {
        RB3_CHECK_ARG(lens[i] >= 0, "negative string length");
        total += lens[i];
    }
    RB3_CHECK_ARG(total == 0 || seq != nullptr, "seq is NULL");
    RB3_CHECK_ARG(opts.batch_mb >= 0, "batch_mb < 0");
    if (opts.batch_mb > 0) {  // cut each batch into runs of whole strings that fit the budget
        const int64_t budget = (int64_t)opts.batch_mb << 20, mult = opts.single_strand ? 1 : 2;
        std::vector<int64_t> cut;
        int64_t s0 = 0;
        for (int64_t b = 0; b < n_batches; ++b) {
            int64_t acc = 0;
            for (int64_t i = s0; i < ends[b]; ++i) {
                const int64_t sym = mult * (lens[i] + 1);
                if (acc > 0 && (acc + sym) * RB3_BUILD_BYTES_PER_SYMBOL > budget) {
                    cut.push_back(i);
                    acc = 0;
                }
                acc += sym;
            }
            if (cut.empty() || cut.back() != ends[b]) cut.push_back(ends[b]);
            s0 = ends[b];
        }
        ends.swap(cut);
        n_batches = (int64_t)ends.size();
    }
    // a run-length dst takes each batch as it is (its spans rewritten per merge)
    RB3_TRY(append_batches(dst, seq, lens.data(), n_seq, ends.data(), n_batches, opts, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    return RB3_OK;
}
