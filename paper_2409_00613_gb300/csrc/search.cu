// Searches on a resident index: backward search (S5) and SMEM finding (S6).
//
// Backward search, Section "Suffix array interval and backward search":
// [lo, hi) starts at [0, n) and becomes [pi(a,lo), pi(a,hi)) for the query's
// symbols from last to first.
//
// SMEMs, Section "Finding supermaximal exact matches", Algorithm 4 over the
// bi-interval extensions of Algorithm 3, with these readings: after the
// forward loop e = |P| if it ran out and e = j if it broke at j, and the
// SMEM's bi-interval is the one before the failing ForwardExt; when e = |P|
// FindSMEM1 returns |P|; when the last backward loop runs out it returns i+1.
//
// Chunked form: a long query is cut at multiples of chunk_len; chunk c runs
// the same loop from x0 = c*chunk_len and keeps SMEMs that start in
// [x0, x0 + chunk_len).  Every start FindSMEM1 returns (other than the one it
// was started from) is an SMEM candidate whatever the loop started from, and
// no SMEM start is ever skipped, so the chunks together give exactly the
// unchunked set; the one start that may be spurious is x0 itself, kept only
// if P[x0-1, e) occurs fewer than s_min times (then f(x0) > f(x0-1)).
#include <cooperative_groups.h>

#include <mutex>

#include "common.cuh"
#include "wait.cuh"
#include "smem.cuh"

namespace cg = cooperative_groups;

namespace rb3 {

__global__ void k_check_codes(const uint8_t *__restrict__ q, int64_t n, int *__restrict__ bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint8_t c = q[i];
        if (c < 1 || c > 5) atomicOr(bad, 1);
    }
}

template <int NS>
__global__ void k_bsearch(OccView V, const uint8_t *__restrict__ q, const int64_t *__restrict__ qoff, int64_t nq,
                          int64_t *__restrict__ lohi) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nq) return;
    int64_t lo = 0, hi = V.n;
    for (int64_t j = qoff[i + 1] - 1; j >= qoff[i]; --j) {
        int a = q[j];
        if (lo == hi) {  // empty interval: lo and hi move together
            lo = hi = C_of(V, a) + rank1<NS>(V, a, lo);
        } else {
            BlockLd<NS> bl = block_load<NS>(V, lo), bh = block_load<NS>(V, hi);
            lo = C_of(V, a) + block_rank<NS>(bl, a);
            hi = C_of(V, a) + block_rank<NS>(bh, a);
        }
    }
    lohi[2 * i] = lo;
    lohi[2 * i + 1] = hi;
}

// Plain form: one thread per query, the whole query.
template <int NS>
__global__ void k_smem_plain(OccView V, const uint8_t *__restrict__ q, const int64_t *__restrict__ qoff, int64_t nq,
                             int ell, int64_t smin, rb3_smem *__restrict__ out, int64_t cap,
                             unsigned long long *__restrict__ count) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nq) return;
    int64_t len = qoff[i + 1] - qoff[i];
    EmitAppend em{out, cap, count};
    smem_range<NS>(V, q + qoff[i], len, i, 0, len, ell, smin, em);
}

// Chunked form: items are (query, chunk); item_off[i] = first item of query i.
// Persistent threads take items with a warp-aggregated atomic counter.
template <int NS>
__global__ void __launch_bounds__(256) k_smem_chunked(OccView V, const uint8_t *__restrict__ q,
                                                      const int64_t *__restrict__ qoff, int64_t nq,
                                                      const int64_t *__restrict__ item_off, int64_t nitems,
                                                      int64_t chunk, int ell, int64_t smin,
                                                      unsigned long long *__restrict__ next,
                                                      rb3_smem *__restrict__ out, int64_t cap,
                                                      unsigned long long *__restrict__ count) {
    for (;;) {
        cg::coalesced_group grp = cg::coalesced_threads();
        unsigned long long base = 0;
        if (grp.thread_rank() == 0) base = atomicAdd(next, (unsigned long long)grp.size());
        base = grp.shfl(base, 0);
        int64_t it = (int64_t)base + grp.thread_rank();
        if (it >= nitems) break;
        // query of item it: largest i with item_off[i] <= it
        int64_t lo = 0, hi = nq;
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) >> 1;
            if (item_off[mid] <= it) lo = mid;
            else hi = mid;
        }
        int64_t qi = lo;
        int64_t len = qoff[qi + 1] - qoff[qi];
        int64_t x0 = (it - item_off[qi]) * chunk;
        int64_t x1 = x0 + chunk < len ? x0 + chunk : len;
        EmitAppend em{out, cap, count};
        smem_range<NS>(V, q + qoff[qi], len, qi, x0, x1, ell, smin, em);
    }
}

// Step-machine form of the chunked search.  The loops of FindSMEM1 (the
// backward check of a start's first min_len symbols, the forward extension,
// the chunk-start check and the backward scan for the next start) have
// data-dependent lengths, so lanes that run them as loops spend most of their
// time waiting for one another.  Here every lane keeps its place in those
// loops as a small state, and each turn of the kernel's loop performs exactly
// one extension for every lane -- a ForwardExt is a BackwardExt of the
// swapped bi-interval by the complement symbol (Algorithm 3), so all lanes run
// the same code -- then moves each lane's state on.  Same starts, same
// extensions, same records as smem_range.
enum : int { SM_ITEM = 0, SM_B1, SM_F, SM_CHK, SM_B2, SM_DONE };

// Counts of the step-machine search since the last reset (rb3_search_stats):
// [0] extensions (BackwardExt or ForwardExt), [1] Occ block reads (one per
// extension whose two interval ends share a block, else two).
__device__ unsigned long long g_search_stats[2];

template <int NS> __device__ __forceinline__ BiInt ext_dir(const OccView &V, BiInt x, int a, bool fwd) {
    const BiInt xi = fwd ? BiInt{x.kp, x.k, x.s} : x;
    const BiInt y = backward_ext<NS>(V, xi, fwd ? comp_sym(a) : a);
    return fwd ? BiInt{y.kp, y.k, y.s} : y;
}

template <int NS>
__global__ void __launch_bounds__(256) k_smem_steps(OccView V, const uint8_t *__restrict__ q,
                                                    const int64_t *__restrict__ qoff, int64_t nq,
                                                    const int64_t *__restrict__ item_off, int64_t nitems,
                                                    int64_t chunk, int ell, int64_t smin,
                                                    unsigned long long *__restrict__ next,
                                                    rb3_smem *__restrict__ out, int64_t cap,
                                                    unsigned long long *__restrict__ count,
                                                    const HotEnt *__restrict__ hot, int hotK) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    EmitAppend em{out, cap, count};
    int phase = SM_ITEM;
    const uint8_t *P = q;
    int64_t qi = 0, len = 0, x0 = 0, x1 = 0, i = 0, j = 0, e = 0, nxt = 0;
    bool first = false;
    BiInt x = {0, 0, V.n};
    uint32_t n_ext = 0, n_reads = 0;  // this lane's counts (rb3_search_stats)
    const int lg = V.log2D;
    for (;;) {
        // lanes without a chunk take the next ones (one atomic per warp)
        const unsigned need = __ballot_sync(0xffffffffu, phase == SM_ITEM);
        if (need) {
            const int leader = __ffs(need) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(next, (unsigned long long)__popc(need));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (phase == SM_ITEM) {
                const int64_t it = (int64_t)base + __popc(need & lt);
                if (it >= nitems) {
                    phase = SM_DONE;
                } else {
                    int64_t lo = 0, hi = nq;  // query of item it: largest i with item_off[i] <= it
                    while (hi - lo > 1) {
                        const int64_t mid = (lo + hi) >> 1;
                        if (item_off[mid] <= it) lo = mid;
                        else hi = mid;
                    }
                    qi = lo;
                    P = q + qoff[qi];
                    len = qoff[qi + 1] - qoff[qi];
                    x0 = (it - item_off[qi]) * chunk;
                    x1 = x0 + chunk < len ? x0 + chunk : len;
                    i = x0;
                    first = x0 > 0;
                    if (i >= x1 || i + ell > len) {
                        phase = SM_ITEM;  // nothing starts in this chunk
                    } else {
                        x = BiInt{0, 0, V.n};
                        j = i + ell - 1;
                        phase = SM_B1;
                    }
                }
            }
        }
        if (__ballot_sync(0xffffffffu, phase != SM_DONE) == 0) {
            // the warp leaves together: one atomic per counter
            const unsigned long long e = __reduce_add_sync(0xffffffffu, n_ext);
            const unsigned long long r = __reduce_add_sync(0xffffffffu, n_reads);
            if (lane == 0) {
                atomicAdd(&g_search_stats[0], e);
                atomicAdd(&g_search_stats[1], r);
            }
            break;
        }
        if (phase == SM_ITEM || phase == SM_DONE) continue;
        // A backward loop that starts from the whole index (B1, B2) takes its
        // first symbols from the hot-level table: the M symbols P[j-M+1, j]
        // (at most hotK, no N, and leaving the loop's last symbol to the step
        // below) in one read, when their interval still occurs >= smin times --
        // then every shorter one does too, so the loop would have taken all M.
        if (hotK > 0 && (phase == SM_B1 || phase == SM_B2) && x.s == V.n) {
            const int64_t room = phase == SM_B1 ? j - i : j - i - 1;
            const int M = room < hotK ? (int)room : hotK;
            uint32_t w = 0;
            int t = 0;
            for (; t < M; ++t) {
                const int c = P[j - t];
                if (c < 1 || c > 4) break;
                w |= (uint32_t)(c - 1) << (2 * t);
            }
            if (t >= 2) {
                const longlong2 *h = reinterpret_cast<const longlong2 *>(hot + hot_off(t) + w);
                const longlong2 a = __ldg(h), b = __ldg(h + 1);
                if (b.x >= smin) {
                    x = BiInt{a.x, a.y, b.x};
                    j -= t;
                    n_ext += (uint32_t)t;
                    ++n_reads;
                }
            }
        }
        // one extension per lane
        const int64_t at = phase == SM_CHK ? x0 - 1 : j;
        {
            const int64_t lo = phase == SM_F ? x.kp : x.k;  // the interval the extension ranks
            ++n_ext;
            n_reads += ((lo + x.s) >> lg) == (lo >> lg) ? 1u : 2u;
        }
        const BiInt y = ext_dir<NS>(V, x, P[at], phase == SM_F);
        bool to_start = false, after_f = false;
        if (phase == SM_B1) {
            if (y.s < smin) {
                i = j + 1;
                first = false;
                to_start = true;
            } else {
                x = y;
                if (j == i) {
                    j = i + ell;
                    if (j >= len) {
                        e = len;
                        after_f = true;
                    } else {
                        phase = SM_F;
                    }
                } else {
                    --j;
                }
            }
        } else if (phase == SM_F) {
            if (y.s < smin) {
                e = j;
                after_f = true;
            } else {
                x = y;
                if (++j == len) {
                    e = len;
                    after_f = true;
                }
            }
        } else if (phase == SM_CHK) {
            // chunk start x0 > 0: spurious if P[x0-1, e) still occurs >= smin times
            first = false;
            if (y.s < smin) em(qi, i, e, x);
            if (e == len) {
                phase = SM_ITEM;
            } else {
                x = BiInt{0, 0, V.n};
                j = e;
                nxt = i + 1;
                phase = SM_B2;
            }
        } else {  // SM_B2: the next start
            if (y.s < smin) {
                i = j + 1;
                to_start = true;
            } else {
                x = y;
                if (--j < i + 1) {
                    i = nxt;
                    to_start = true;
                }
            }
        }
        if (after_f) {
            if (first) {
                phase = SM_CHK;
            } else {
                em(qi, i, e, x);
                if (e == len) {
                    phase = SM_ITEM;
                } else {
                    x = BiInt{0, 0, V.n};
                    j = e;
                    nxt = i + 1;
                    phase = SM_B2;
                }
            }
        }
        if (to_start) {
            if (i >= x1 || i + ell > len) {
                phase = SM_ITEM;
            } else {
                x = BiInt{0, 0, V.n};
                j = i + ell - 1;
                phase = SM_B1;
            }
        }
    }
}

__global__ void k_smem_keys(const rb3_smem *__restrict__ r, int64_t n, uint64_t *__restrict__ key,
                            uint32_t *__restrict__ val) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    key[i] = ((uint64_t)r[i].qid << 32) | (uint32_t)r[i].start;
    val[i] = (uint32_t)i;
}

__global__ void k_smem_gather(const rb3_smem *__restrict__ in, const uint32_t *__restrict__ idx, int64_t n,
                              rb3_smem *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[idx[i]];
}

static inline unsigned nb_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

int search_stats(int64_t out[2], bool reset) {
    unsigned long long h[2];
    RB3_CUDA_TRY(cudaMemcpyFromSymbol(h, g_search_stats, sizeof(h)));
    for (int i = 0; i < 2; ++i) out[i] = (int64_t)h[i];
    if (reset) {
        const unsigned long long z[2] = {0, 0};
        RB3_CUDA_TRY(cudaMemcpyToSymbol(g_search_stats, z, sizeof(z)));
    }
    return RB3_OK;
}

int check_codes(const uint8_t *q, int64_t n, cudaStream_t st) {
    if (n <= 0) return RB3_OK;
    DevBuf bad;
    RB3_TRY(bad.alloc(sizeof(int), st));
    RB3_CUDA_TRY(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    unsigned grid = nb_for(n, 256);
    if (grid > (unsigned)num_sms() * 8) grid = (unsigned)num_sms() * 8;
    RB3_LAUNCH(k_check_codes, grid, 256, 0, st, q, n, bad.as<int>());
    int h = 0;
    RB3_CUDA_TRY(cudaMemcpyAsync(&h, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    if (h) {
        set_error("query symbol outside 1..5 (A,C,G,T,N codes)");
        return RB3_E_INVAL;
    }
    return RB3_OK;
}

int backward_search_impl(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, int64_t nq, int64_t total_q,
                         int64_t *lohi, cudaStream_t st) {
    RB3_TRY(check_codes(q, total_q, st));
    Phase ph("search.backward", st);
    if (nq > 0)
        RB3_WITH_NS(idx->D, RB3_LAUNCH(k_bsearch<NS>, nb_for(nq, 128), 128, 0, st, occ_view(idx), q, qoff, nq, lohi));
    return RB3_OK;
}

// ---- hot-level table ----------------------------------------------------------
// Level L from level L - 1: the string of digits w is its first symbol w >> 2(L-1)
// put before the string w mod 4^(L-1), so its interval is one BackwardExt of that
// string's (for L = 1, of the whole index).  One thread per string.
template <int NS>
__global__ void k_hot_level(OccView V, HotEnt *__restrict__ tab, int L) {
    const int64_t nw = int64_t(1) << (2 * L);
    const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w >= nw) return;
    BiInt x = {0, 0, V.n};
    if (L > 1) {
        const HotEnt &p = tab[hot_off(L - 1) + (w & ((nw >> 2) - 1))];
        x = BiInt{p.k, p.kp, p.s};
    }
    const BiInt y = backward_ext<NS>(V, x, (int)(w >> (2 * (L - 1))) + 1);
    tab[hot_off(L) + w] = HotEnt{y.k, y.kp, y.s, 0};
}

namespace {
std::mutex g_hot_mu;  // one builder at a time (server slots search from several threads)
const void *rank_arrays(const rb3_index *idx) { return idx->rle ? (const void *)idx->payload : idx->blocks; }
}  // namespace

void free_hot(rb3_index *x) {
    std::lock_guard<std::mutex> lk(g_hot_mu);
    if (x->hot) cudaFree(x->hot);
    for (void *p : x->hot_old) cudaFree(p);
    x->hot_old.clear();
    x->hot = nullptr;
    x->hot_k = 0;
    x->hot_n = -1;
    x->hot_src = nullptr;
}

// A table of depth K also serves every smaller depth (level L's place does not
// depend on K), so a deeper table is kept.
int hot_table(const rb3_index *idx, int K, cudaStream_t st, const HotEnt **out) {
    std::lock_guard<std::mutex> lk(g_hot_mu);
    const bool fresh = idx->hot && idx->hot_n == idx->n && idx->hot_src == rank_arrays(idx);
    if (fresh && idx->hot_k >= K) {
        *out = static_cast<const HotEnt *>(idx->hot);
        return RB3_OK;
    }
    if (idx->hot) {
        if (fresh) {
            idx->hot_old.push_back(idx->hot);  // shallower: other streams may still read it
        } else {
            // the index changed since (a merge), and no search runs beside a merge
            RB3_CUDA_TRY(cudaStreamSynchronize(st));
            cudaFree(idx->hot);
        }
        idx->hot = nullptr;
        idx->hot_k = 0;
    }
    // plain cudaMalloc: the table outlives the stream it is built on
    struct Guard {
        void *p = nullptr;
        ~Guard() {
            if (p) cudaFree(p);
        }
    } g;
    const size_t bytes = sizeof(HotEnt) * (size_t)hot_off(K + 1);
    RB3_CUDA_TRY(cudaMalloc(&g.p, bytes));
    const OccView V = occ_view(idx);
    for (int L = 1; L <= K; ++L) {
        const int64_t nw = int64_t(1) << (2 * L);
        RB3_WITH_NS(idx->D,
                    RB3_LAUNCH(k_hot_level<NS>, nb_for(nw, 256), 256, 0, st, V, static_cast<HotEnt *>(g.p), L));
    }
    RB3_CUDA_TRY(cudaStreamSynchronize(st));  // other streams may read it as soon as it is published
    idx->hot = g.p;
    g.p = nullptr;
    idx->hot_k = K;
    idx->hot_n = idx->n;
    idx->hot_src = rank_arrays(idx);
    *out = static_cast<const HotEnt *>(idx->hot);
    return RB3_OK;
}

int hot_depth_for(const rb3_index *idx, const rb3_opts &o, int64_t nq, int64_t total_q) {
    int K = o.hot_depth;
    if (K == 0) K = (int)tuned_hot_depth(idx, nq, total_q);
    if (K == 0) {
        K = idx->n > 1 ? ilog2(idx->n) / 2 - 3 : 0;
        if (K > 10) K = 10;
    }
    if (K < 2) return 0;  // a table of single symbols saves no step
    return K > HOT_MAX ? HOT_MAX : K;
}

int mem_search_impl(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, const int64_t *qoff_host,
                    int64_t nq, int64_t total_q, int32_t min_len, int64_t min_occ, const rb3_opts &o,
                    rb3_smem *out_dev, int64_t cap, int64_t *n_out, cudaStream_t st, bool codes_checked) {
    if (!codes_checked) RB3_TRY(check_codes(q, total_q, st));
    *n_out = 0;
    if (nq == 0) return RB3_OK;
    OccView V = occ_view(idx);
    int64_t chunk = o.chunk_len > 0 ? o.chunk_len : tuned_chunk_len(idx, nq, total_q);
    if (chunk <= 0) chunk = 256;
    const bool plain = o.search_form == 1;
    const bool loops = o.search_form == 2;  // chunked, each lane running FindSMEM1's loops
    const HotEnt *hot = nullptr;
    int hotK = plain || loops ? 0 : hot_depth_for(idx, o, nq, total_q);
    if (hotK > 0) RB3_TRY(hot_table(idx, hotK, st, &hot));
    std::vector<int64_t> item_off;
    int64_t nitems = nq;
    if (!plain) {
        item_off.resize(nq + 1);
        item_off[0] = 0;
        for (int64_t i = 0; i < nq; ++i) {
            int64_t len = qoff_host[i + 1] - qoff_host[i];
            int64_t c = len <= chunk ? 1 : (len + chunk - 1) / chunk;
            item_off[i + 1] = item_off[i] + c;
        }
        nitems = item_off[nq];
    }
    DevBuf items, ctr;
    RB3_TRY(ctr.alloc(2 * sizeof(unsigned long long), st));
    if (!plain) {
        RB3_TRY(items.alloc(sizeof(int64_t) * (nq + 1), st));
        RB3_CUDA_TRY(cudaMemcpyAsync(items.p, item_off.data(), sizeof(int64_t) * (nq + 1), cudaMemcpyHostToDevice, st));
    }
    // scratch for unsorted records: grows once if the first guess is short
    int64_t guess = total_q / 32 + 4096;
    int64_t scap = guess < cap ? guess : cap;
    if (scap < 1) scap = 1;
    DevBuf raw;
    unsigned long long count = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        raw.release();
        RB3_TRY(raw.alloc(sizeof(rb3_smem) * scap, st));
        RB3_CUDA_TRY(cudaMemsetAsync(ctr.p, 0, 2 * sizeof(unsigned long long), st));
        unsigned long long *d_next = ctr.as<unsigned long long>(), *d_count = d_next + 1;
        {
            Phase ph(plain ? "k.smem_plain" : (loops ? "k.smem_chunked" : "k.smem_steps"), st,
                     (double)total_q);  // bytes = query bases
            if (plain) {
                RB3_WITH_NS(idx->D, RB3_LAUNCH(k_smem_plain<NS>, nb_for(nq, 128), 128, 0, st, V, q, qoff, nq,
                                               (int)min_len, min_occ, raw.as<rb3_smem>(), scap, d_count));
            } else {
                int64_t resident = (int64_t)num_sms() * 2048;
                int64_t threads = nitems < resident ? nitems : resident;
                if (loops)
                    RB3_WITH_NS(idx->D, RB3_LAUNCH(k_smem_chunked<NS>, nb_for(threads, 256), 256, 0, st, V, q, qoff,
                                                   nq, items.as<int64_t>(), nitems, chunk, (int)min_len, min_occ,
                                                   d_next, raw.as<rb3_smem>(), scap, d_count));
                else  // one-warp CTAs: a warp's registers go back to the SM as soon as its lanes run out
                      // of chunks, not when the CTA's slowest warp does (micro-batches of other
                      // streams then get the SM)
                    RB3_WITH_NS(idx->D, RB3_LAUNCH(k_smem_steps<NS>, nb_for(threads, 32), 32, 0, st, V, q, qoff,
                                                   nq, items.as<int64_t>(), nitems, chunk, (int)min_len, min_occ,
                                                   d_next, raw.as<rb3_smem>(), scap, d_count, hot, hotK));
            }
        }
        RB3_CUDA_TRY(cudaMemcpyAsync(&count, d_count, sizeof(count), cudaMemcpyDeviceToHost, st));
        RB3_TRY(wait_stream_blocking(st));  // the search takes milliseconds: sleep, do not spin
        if ((int64_t)count <= scap || (int64_t)count > cap) break;
        scap = (int64_t)count;  // rerun with room for every record
    }
    *n_out = (int64_t)count;
    if ((int64_t)count > cap) {
        set_error("mem_search: %lld SMEMs found, output capacity %lld", (long long)count, (long long)cap);
        return RB3_E_CAPACITY;
    }
    if (count == 0) return RB3_OK;
    Phase ph("search.smem_sort", st);
    int64_t R = (int64_t)count;
    DevBuf k0, k1, v0, v1;
    RB3_TRY(k0.alloc(sizeof(uint64_t) * R, st));
    RB3_TRY(k1.alloc(sizeof(uint64_t) * R, st));
    RB3_TRY(v0.alloc(sizeof(uint32_t) * R, st));
    RB3_TRY(v1.alloc(sizeof(uint32_t) * R, st));
    RB3_LAUNCH(k_smem_keys, nb_for(R, 256), 256, 0, st, raw.as<rb3_smem>(), R, k0.as<uint64_t>(), v0.as<uint32_t>());
    bool alt = false;
    RB3_TRY(radix_sort_pairs(k0.as<uint64_t>(), v0.as<uint32_t>(), k1.as<uint64_t>(), v1.as<uint32_t>(), R, 0,
                             32 + ilog2(nq) + 1, st, &alt));
    RB3_LAUNCH(k_smem_gather, nb_for(R, 256), 256, 0, st, raw.as<rb3_smem>(),
               alt ? v1.as<uint32_t>() : v0.as<uint32_t>(), R, out_dev);
    return RB3_OK;
}

}  // namespace rb3
