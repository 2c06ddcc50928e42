// Served SMEM search: continuous batching over a device-resident index.
//
// Requests (one query each) are queued on submit.  `slots` worker threads,
// each with its own CUDA stream and its own pinned / device buffers of a fixed
// size, loop: take every waiting request that fits the slot's budget of query
// bases (at least one; a request longer than the budget is taken alone), run
// them as one micro-batch of the chunked SMEM search, hand each request its
// records and its timestamps, and go back to the queue.  A request that
// arrives while micro-batches are on the GPU is admitted by the next slot to
// free up, so several micro-batches overlap on the device; memory is bounded by
// slots x budget.  Results do not depend on the batching: a query's SMEMs are
// a function of the query and the index only.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "common.cuh"
#include "wait.cuh"

struct rb3_server {
    const rb3_index *idx = nullptr;
    rb3_server_opts o{};
    int dev = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    struct Req {
        int64_t id, tag, t_submit;
        std::vector<uint8_t> q;
    };
    std::deque<Req> pending;
    std::deque<rb3_completion> completions;
    std::map<int64_t, std::vector<rb3_smem>> results;
    int64_t next_id = 1;
    bool stop = false;
    std::vector<std::thread> workers;
    int first_error = RB3_OK;
    std::string error_msg;
    std::atomic<int64_t> batches{0};
    // worker time (rb3_server_stats): requests and bases taken, ns gathering
    // queries into the slot's pinned buffer, ns in the micro-batch's search
    // (copies in, search, records back, synchronized), ns splitting records and
    // publishing completions
    std::atomic<int64_t> st_requests{0}, st_bases{0}, st_gather_ns{0}, st_search_ns{0}, st_publish_ns{0};
    // slots whose stream and buffers are set up (rb3_server_create waits for
    // all of them), and the first setup failure
    int ready = 0;
    int setup_error = RB3_OK;
};

namespace rb3 {

static int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

static void server_worker(rb3_server *S) {
    cudaSetDevice(S->dev);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    const int64_t budget = S->o.max_batch_bases;
    uint8_t *h_q = nullptr;
    int64_t *h_off = nullptr;
    cudaMallocHost(&h_q, (size_t)budget);
    cudaMallocHost(&h_off, sizeof(int64_t) * (size_t)(S->o.max_batch_requests + 1));
    uint8_t *d_q = nullptr;
    int64_t *d_off = nullptr;
    rb3_smem *d_out = nullptr;
    int64_t out_cap = 0;
    int64_t qcap = budget;
    int setup = st ? RB3_OK : RB3_E_CUDA;
    if (setup == RB3_OK) setup = h_q && h_off ? RB3_OK : RB3_E_NOMEM;
    if (setup == RB3_OK) setup = dev_alloc((void **)&d_q, (size_t)qcap, st);
    if (setup == RB3_OK)
        setup = dev_alloc((void **)&d_off, sizeof(int64_t) * (size_t)(S->o.max_batch_requests + 1), st);
    if (setup == RB3_OK && cudaStreamSynchronize(st) != cudaSuccess) setup = RB3_E_CUDA;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        ++S->ready;
        if (setup != RB3_OK && S->setup_error == RB3_OK) S->setup_error = setup;
        if (setup != RB3_OK) S->stop = true;  // the server is not started; the other slots leave too
    }
    S->cv_done.notify_all();
    std::vector<rb3_smem> h_out;
    rb3_opts so;
    rb3_opts_default(&so);
    so.search_form = (int32_t)S->o.search_form;
    so.hot_depth = (int32_t)S->o.hot_depth;
    for (;;) {
        std::vector<rb3_server::Req> batch;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty(); });
            if (S->stop) break;
            int64_t bases = 0;
            while (!S->pending.empty() && (int64_t)batch.size() < S->o.max_batch_requests) {
                const int64_t L = (int64_t)S->pending.front().q.size();
                if (!batch.empty() && bases + L > budget) break;
                bases += L;
                batch.push_back(std::move(S->pending.front()));
                S->pending.pop_front();
            }
        }
        const int64_t t_take = now_ns();
        // concatenate (a request longer than the budget gets its own buffer)
        int64_t total = 0;
        for (auto &r : batch) total += (int64_t)r.q.size();
        const int64_t nq = (int64_t)batch.size();
        uint8_t *hq = h_q;
        std::vector<uint8_t> big;
        if (total > budget) {
            big.resize((size_t)total);
            hq = big.data();
        }
        h_off[0] = 0;
        for (int64_t i = 0; i < nq; ++i) {
            memcpy(hq + h_off[i], batch[i].q.data(), batch[i].q.size());
            h_off[i + 1] = h_off[i] + (int64_t)batch[i].q.size();
        }
        const int64_t t_gathered = now_ns();
        int r = RB3_OK;
        if (total > qcap) {
            dev_free(d_q, st);
            qcap = total;
            r = dev_alloc((void **)&d_q, (size_t)qcap, st);
        }
        if (r == RB3_OK && total > 0 && cudaMemcpyAsync(d_q, hq, (size_t)total, cudaMemcpyHostToDevice, st) != cudaSuccess)
            r = cuda_fail(cudaGetLastError(), "server: copy queries", __FILE__, __LINE__);
        if (r == RB3_OK &&
            cudaMemcpyAsync(d_off, h_off, sizeof(int64_t) * (nq + 1), cudaMemcpyHostToDevice, st) != cudaSuccess)
            r = cuda_fail(cudaGetLastError(), "server: copy offsets", __FILE__, __LINE__);
        int64_t n = 0;
        if (r == RB3_OK && !d_out) {
            out_cap = total / 16 + 4096;
            r = dev_alloc((void **)&d_out, sizeof(rb3_smem) * (size_t)out_cap, st);
        }
        if (r == RB3_OK) {
            // the symbols were checked by rb3_server_submit
            r = mem_search_impl(S->idx, d_q, d_off, h_off, nq, total, S->o.min_len, S->o.min_occ, so, d_out, out_cap,
                                &n, st, true);
            if (r == RB3_E_CAPACITY) {  // grow once to the size reported and rerun
                dev_free(d_out, st);
                out_cap = n + 4096;
                r = dev_alloc((void **)&d_out, sizeof(rb3_smem) * (size_t)out_cap, st);
                if (r == RB3_OK)
                    r = mem_search_impl(S->idx, d_q, d_off, h_off, nq, total, S->o.min_len, S->o.min_occ, so, d_out,
                                        out_cap, &n, st, true);
            }
        }
        if (r == RB3_OK) {
            h_out.resize((size_t)n);
            if (n && cudaMemcpyAsync(h_out.data(), d_out, sizeof(rb3_smem) * n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
                r = cuda_fail(cudaGetLastError(), "server: copy results", __FILE__, __LINE__);
            if (r == RB3_OK) r = wait_stream_blocking(st);  // slots sleep while their batch runs
        }
        const int64_t t_done = now_ns();
        S->batches.fetch_add(1);
        // split records by query (sorted by (qid, start)), publish
        std::vector<std::vector<rb3_smem>> per(nq);
        if (r == RB3_OK)
            for (int64_t i = 0; i < n;) {  // each request's records are contiguous
                const int64_t qi = h_out[i].qid;
                int64_t j = i + 1;
                while (j < n && h_out[j].qid == qi) ++j;
                per[qi].assign(h_out.begin() + i, h_out.begin() + j);
                for (auto &x : per[qi]) x.qid = 0;
                i = j;
            }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (r != RB3_OK && S->first_error == RB3_OK) {
                S->first_error = r;
                S->error_msg = rb3_last_error_str();
            }
            for (int64_t i = 0; i < nq; ++i) {
                rb3_completion c;
                c.req_id = batch[i].id;
                c.tag = batch[i].tag;
                c.n_smem = (int64_t)per[i].size();
                c.status = r;
                c.batch_requests = (int32_t)nq;
                c.t_submit_ns = batch[i].t_submit;
                c.t_done_ns = t_done;
                S->completions.push_back(c);
                S->results[c.req_id] = std::move(per[i]);
            }
        }
        S->cv_done.notify_all();
        S->st_requests.fetch_add(nq);
        S->st_bases.fetch_add(total);
        S->st_gather_ns.fetch_add(t_gathered - t_take);
        S->st_search_ns.fetch_add(t_done - t_gathered);
        S->st_publish_ns.fetch_add(now_ns() - t_done);
    }
    dev_free(d_q, st);
    dev_free(d_off, st);
    dev_free(d_out, st);
    cudaStreamSynchronize(st);
    cudaFreeHost(h_q);
    cudaFreeHost(h_off);
    if (st) cudaStreamDestroy(st);
}

}  // namespace rb3

using namespace rb3;

RB3_EXPORT void rb3_server_opts_default(rb3_server_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->min_len = 31;
    o->min_occ = 1;
    o->slots = 4;
    o->max_batch_bases = 32 << 20;
    o->max_batch_requests = 4096;
}

RB3_EXPORT int rb3_server_create(const rb3_index *idx, const rb3_server_opts *o, rb3_server **out) {
    set_error("%s", "");
    RB3_CHECK_ARG(idx && out, "NULL argument");
    RB3_CHECK_ARG(!idx->single_strand, "SMEM search needs a double-strand index");
    rb3_server_opts opt;
    rb3_server_opts_default(&opt);
    if (o) opt = *o;
    RB3_CHECK_ARG(opt.min_len >= 1 && opt.min_occ >= 1, "min_len and min_occ must be >= 1");
    RB3_CHECK_ARG(opt.slots >= 1 && opt.slots <= 64, "slots must be in [1, 64]");
    RB3_CHECK_ARG(opt.max_batch_bases >= 1 && opt.max_batch_requests >= 1, "batch limits must be >= 1");
    RB3_CHECK_ARG(opt.search_form >= 0 && opt.search_form <= 2, "search_form must be 0, 1 or 2");
    RB3_CHECK_ARG(opt.hot_depth >= -1 && opt.hot_depth <= HOT_MAX, "hot_depth must be -1..12");
    if (opt.search_form == 0) {  // the hot-level table now, not in the first micro-batch
        rb3_opts so;
        rb3_opts_default(&so);
        so.hot_depth = (int32_t)opt.hot_depth;
        const int K = hot_depth_for(idx, so, 0, 0);
        const HotEnt *tab = nullptr;
        if (K > 0) RB3_TRY(hot_table(idx, K, 0, &tab));
    }
    rb3_server *S = new rb3_server();
    S->idx = idx;
    S->o = opt;
    cudaGetDevice(&S->dev);
    for (int i = 0; i < opt.slots; ++i) S->workers.emplace_back(server_worker, S);
    {  // every slot's stream and buffers exist before the first request arrives
        std::unique_lock<std::mutex> lk(S->mu);
        S->cv_done.wait(lk, [&] { return S->ready == opt.slots; });
    }
    if (S->setup_error != RB3_OK) {
        const int e = S->setup_error;
        rb3_server_destroy(S);
        set_error("server: a slot's stream or buffers could not be set up");
        return e;
    }
    *out = S;
    return RB3_OK;
}

// A request of the query q[0, len), its symbols checked (A,C,G,T,N codes).
static int make_req(const uint8_t *q, int64_t len, int64_t tag, rb3_server::Req *r) {
    RB3_CHECK_ARG((len == 0 || q) && len >= 0, "bad argument");
    RB3_CHECK_ARG(len < (int64_t(1) << 31), "query longer than 2^31 - 1");
    unsigned bad = 0;  // branch-free, so the compiler vectorizes the check
    for (int64_t i = 0; i < len; ++i) bad |= (unsigned)((uint8_t)(q[i] - 1u) > 4u);
    if (bad) {
        set_error("query symbol outside 1..5 (A,C,G,T,N codes)");
        return RB3_E_INVAL;
    }
    r->tag = tag;
    r->q.assign(q, q + len);
    r->t_submit = now_ns();
    return RB3_OK;
}

RB3_EXPORT int rb3_server_submit(rb3_server *S, const uint8_t *q, int64_t len, int64_t tag, int64_t *req_id) {
    RB3_CHECK_ARG(S != nullptr, "bad argument");
    rb3_server::Req r;
    RB3_TRY(make_req(q, len, tag, &r));
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r.id = S->next_id++;
        if (req_id) *req_id = r.id;
        S->pending.push_back(std::move(r));
    }
    S->cv_work.notify_one();
    return RB3_OK;
}

RB3_EXPORT int rb3_server_poll(rb3_server *S, rb3_completion *out, int64_t cap, int64_t *n, int32_t wait_us) {
    RB3_CHECK_ARG(S && n && (cap == 0 || out), "bad argument");
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->completions.empty() && wait_us > 0)
        S->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), [&] { return !S->completions.empty(); });
    int64_t k = 0;
    while (k < cap && !S->completions.empty()) {
        out[k++] = S->completions.front();
        S->completions.pop_front();
    }
    *n = k;
    if (S->first_error != RB3_OK) {
        set_error("%s", S->error_msg.c_str());
        return S->first_error;
    }
    return RB3_OK;
}

RB3_EXPORT int rb3_server_take(rb3_server *S, int64_t req_id, rb3_smem *out, int64_t cap, int64_t *n) {
    RB3_CHECK_ARG(S && n, "bad argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->results.find(req_id);
    if (it == S->results.end()) {
        set_error("request %lld has no results (not completed or already taken)", (long long)req_id);
        return RB3_E_INVAL;
    }
    *n = (int64_t)it->second.size();
    if (*n > cap) {
        set_error("request %lld has %lld SMEMs, capacity %lld", (long long)req_id, (long long)*n, (long long)cap);
        return RB3_E_CAPACITY;
    }
    if (*n) memcpy(out, it->second.data(), sizeof(rb3_smem) * (size_t)*n);
    S->results.erase(it);
    return RB3_OK;
}

RB3_EXPORT int64_t rb3_server_batches(rb3_server *S) { return S ? S->batches.load() : 0; }

RB3_EXPORT int rb3_server_stats(rb3_server *S, int64_t out[6]) {
    RB3_CHECK_ARG(S && out, "NULL argument");
    out[0] = S->batches.load();
    out[1] = S->st_requests.load();
    out[2] = S->st_bases.load();
    out[3] = S->st_gather_ns.load();
    out[4] = S->st_search_ns.load();
    out[5] = S->st_publish_ns.load();
    return RB3_OK;
}

// Open-loop replay of an arrival trace from native threads: four submitting
// threads queue request i at t0 + arrival_ns[i] (sleeping until shortly
// before, then spinning), while the calling thread collects the completions and
// drops their records; done_ns[i] = completion time - t0 (CLOCK_MONOTONIC),
// batch[i] = size of its micro-batch.
RB3_EXPORT int rb3_server_replay(rb3_server *S, const uint8_t *q, const int64_t *qoff, int64_t n,
                                 const int64_t *arrival_ns, int64_t *done_ns, int32_t *batch) {
    set_error("%s", "");
    RB3_CHECK_ARG(S && qoff && arrival_ns && done_ns && n >= 0, "bad argument");
    for (int64_t i = 0; i < n; ++i) {
        RB3_CHECK_ARG(qoff[i + 1] >= qoff[i] && (i == 0 || arrival_ns[i] >= arrival_ns[i - 1]),
                      "qoff and arrival_ns must not decrease");
        done_ns[i] = -1;
    }
    RB3_CHECK_ARG(n == 0 || qoff[n] == qoff[0] || q, "q is NULL");
    const int64_t t0 = now_ns() + 2000000;
    std::atomic<int> sub_err{RB3_OK};
    // several submitting threads (as several clients would be), thread t taking
    // requests t, t + T, t + 2T, ...: each copies and checks every one of its
    // requests due by now outside the lock, then queues them under one lock
    // with one wake-up
    constexpr int T = 4;
    auto submit_part = [&](int t) {
        std::vector<rb3_server::Req> due;
        for (int64_t i = t; i < n && sub_err.load() == RB3_OK;) {
            const int64_t target = t0 + arrival_ns[i];
            for (int64_t now = now_ns(); now < target; now = now_ns())
                if (target - now > 60000) std::this_thread::sleep_for(std::chrono::nanoseconds(target - now - 40000));
            const int64_t now = now_ns();
            due.clear();
            int64_t j = i;
            for (; j < n && t0 + arrival_ns[j] <= now && (int64_t)due.size() < 4096; j += T) {
                due.emplace_back();
                const int r = make_req(q + qoff[j], qoff[j + 1] - qoff[j], j, &due.back());
                if (r != RB3_OK) {
                    sub_err.store(r);
                    due.pop_back();
                    break;
                }
            }
            {
                std::lock_guard<std::mutex> lk(S->mu);
                for (auto &r : due) {
                    r.id = S->next_id++;
                    S->pending.push_back(std::move(r));
                }
            }
            S->cv_work.notify_all();
            i = j;
        }
    };
    std::vector<std::thread> submitters;
    for (int t = 0; t < T; ++t) submitters.emplace_back(submit_part, t);
    int64_t got = 0;
    int status = RB3_OK;
    std::vector<rb3_completion> c(4096);
    while (got < n && sub_err.load() == RB3_OK) {
        int64_t k = 0;
        status = rb3_server_poll(S, c.data(), (int64_t)c.size(), &k, 20000);
        if (status != RB3_OK) break;
        std::lock_guard<std::mutex> lk(S->mu);
        for (int64_t j = 0; j < k; ++j) {
            const int64_t i = c[j].tag;
            if (i >= 0 && i < n) {
                done_ns[i] = c[j].t_done_ns - t0;
                if (batch) batch[i] = c[j].batch_requests;
            }
            S->results.erase(c[j].req_id);
            ++got;
        }
    }
    for (auto &th : submitters) th.join();
    if (status == RB3_OK && sub_err.load() != RB3_OK) status = sub_err.load();
    return status;
}

RB3_EXPORT void rb3_server_destroy(rb3_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto &t : S->workers) t.join();
    delete S;
}
