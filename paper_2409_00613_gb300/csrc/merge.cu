// Merge of a batch BWT B2 into B1: Algorithm 1 (AppendBWT).
//
// For every B2 row k the merged row is pos[k] = k + l(k), where l(k) is the
// number of B1 suffixes smaller than the suffix of row k (the walk of
// Algorithm 1: l starts at m1 at each new string's sentinel and becomes
// pi_{B1}(a, l) one symbol back).  pos increases with k, so the inserts of
// Algorithm 1 are a stable merge: row q of the result takes the next B2
// symbol when q is the next pos, else the next B1 symbol.
//
// Forms of the walk (equal results):
//  * plain     -- one thread per new string, exactly as Algorithm 1: rows of
//                 B2 are followed by LF on B2 (pi_{B2}), l by pi_{B1}.
//  * segmented -- uses the batch's text T2 and inverse suffix array: the rows
//                 visited by Algorithm 1's walk for string i are ISA2 of the
//                 positions of P_i read right to left, and the symbol at each
//                 step is the text symbol.  Each string is cut into segments of
//                 about L symbols (by default each cut moved, within +-L/4, to a
//                 content anchor, so that the haplotypes' homologous segments
//                 start at the same locus); the exact l at a segment's right end (its seed) is
//                 found with ForwardExt (Algorithm 3) over B1 along the suffix
//                 that starts there, in the same persistent kernel that walks
//                 the segment; a walk that reaches a segment whose seed is not
//                 in yet takes that segment over (see k_merge_walk).  Segments
//                 are taken under warp-aggregated work stealing, ordered so that
//                 homologous segments of the batch's strings run together and
//                 share B1 blocks in L2.
#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace rb3 {

// ---- plain Algorithm 1 walk --------------------------------------------------
// own (optional): own[i] != 0 for the new strings this call walks (string i
// starts at B2 row i, its sentinel's row); the others are left alone.
template <int NS1, int NS2>
__global__ void k_walk_plain(OccView B1, OccView B2, int64_t m1, int64_t m2, const uint8_t *__restrict__ own,
                             int64_t *__restrict__ pos, unsigned int *__restrict__ err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m2) return;
    if (own && !own[i]) return;
    int64_t k = i, l = m1;
    for (int64_t steps = 0;; ++steps) {
        int a = sym_at(B2, k);
        pos[k] = k + l;
        if (a == 0) break;
        if (steps >= B2.n) {  // a BWT walk ends within n steps; guards a corrupt input
            atomicOr(err, 1u);
            break;
        }
        BlockLd<NS2> b2 = block_load<NS2>(B2, k);  // both blocks issued before use
        BlockLd<NS1> b1 = block_load<NS1>(B1, l);
        int64_t kn = C_of(B2, a) + block_rank<NS2>(b2, a);
        l = C_of(B1, a) + block_rank<NS1>(b1, a);
        k = kn;
    }
}

// ---- segmented walk with in-kernel seeds ------------------------------------------
// Segment w of a string covers positions [hi(w+1), hi(w)) (hi(w+1) = string
// start for its lowest segment); the top segment of a string starts at its
// sentinel, where l = m1 is known.  Every other segment first computes the exact
// l at hi(w) (its seed), then walks down.  A walk that has written position
// hi(w+1) either stops there, if segment w+1 has already resolved its seed, or
// claims segment w+1 and walks on through it.  state[w] goes 0 -> 1 when w's
// seed resolves and 0 -> 2 when the walk from above claims w; both moves are
// compare-and-swap, so exactly one walk covers every segment.  A seed whose
// segment was claimed stops at its next check.  No thread ever waits.
constexpr int ST_PENDING = 0, ST_RESOLVED = 1, ST_CLAIMED = 2;

__device__ __forceinline__ int load_state(const int *p) { return *reinterpret_cast<const volatile int *>(p); }

// Seed by ForwardExt (Algorithm 3) along X = T2[x, send)$ over a double-strand
// B1: extend until the count s is 0 (l = the k field of that failing extension:
// the B1 suffixes below X), or to X's sentinel (l = k + occ(Q$): the B1
// suffixes equal to Q up to a sentinel are older, hence smaller).  Returns -1
// if claimed from above or after cap steps.
// Rank block reads of the walks since the last reset (rb3_walk_stats):
// [0] seeds run, [1] block reads of seeds, [2] block reads of walk steps,
// [3] segments taken over from above.
__device__ unsigned long long g_walk_stats[4];

template <int NS>
__device__ __forceinline__ int64_t seed_forward(const OccView &B1, const uint8_t *__restrict__ T2, int64_t x,
                                                int64_t send, int64_t cap, const int *state_w, uint32_t *reads) {
    BiInt q = {0, 0, B1.n};
    int a = T2[x];
    const int lg = NS == 0 ? 5 : B1.log2D;
    for (int64_t t = 0;; ++t) {
        const int64_t p = x + t;
        if (p == send) {
            *reads += 2;
            return q.k + (rank1<NS>(B1, 0, q.kp + q.s) - rank1<NS>(B1, 0, q.kp));
        }
        if (t >= cap) return -1;
        if ((t & 15) == 15 && load_state(state_w) == ST_CLAIMED) return -1;
        const int an = T2[p + 1];  // next symbol (the sentinel at most), loaded ahead
        *reads += ((q.kp + q.s) >> lg) == (q.kp >> lg) ? 1u : 2u;  // ForwardExt reads the swapped interval's ends
        const BiInt y = forward_ext<NS>(B1, q, a);
        if (y.s == 0) return y.k;
        q = y;
        a = an;
    }
}

// Seed for any B1 (single strand has no ForwardExt): backward search over
// T2[x, y), y = min(x + cap, send).  From the sentinel the walk is exact at
// once (l = m1); otherwise the SA interval [lo, hi) of T2[p, y) is kept, and
// once it is empty every B1 suffix compares with T2[p..]$ as with T2[p, y), so
// l(p) = lo exactly.  Returns -1 if it never becomes exact or is claimed.
template <int NS>
__device__ __forceinline__ int64_t seed_backward(const OccView &B1, int64_t m1, const uint8_t *__restrict__ T2,
                                                 int64_t x, int64_t send, int64_t cap, const int *state_w,
                                                 uint32_t *reads) {
    const int64_t y = x + cap < send ? x + cap : send;
    bool exact = y == send;
    int64_t lo = exact ? m1 : 0, hi = exact ? m1 : B1.n;
    for (int64_t p = y - 1; p >= x; --p) {
        if (((y - p) & 15) == 0 && load_state(state_w) == ST_CLAIMED) return -1;
        const int a = T2[p];
        *reads += exact ? 1u : 2u;
        if (exact) {
            lo = C_of(B1, a) + rank1<NS>(B1, a, lo);
            hi = lo;
        } else {
            BlockLd<NS> bl = block_load<NS>(B1, lo), bh = block_load<NS>(B1, hi);
            lo = C_of(B1, a) + block_rank<NS>(bl, a);
            hi = C_of(B1, a) + block_rank<NS>(bh, a);
            exact = lo == hi;
        }
    }
    return exact ? lo : -1;
}

// One warp per CTA: a CTA's registers go back to the SM as soon as its 32
// walks are done, so work on other streams (the next batch's build) can use
// the SMs while the last long walks finish.
constexpr int WALK_THREADS = 32;

template <int NS, bool DS>
__global__ void __launch_bounds__(WALK_THREADS, 32) k_merge_walk(OccView B1, int64_t m1, const uint8_t *__restrict__ T2,
                                                    const int32_t *__restrict__ isa2,
                                                    const int64_t *__restrict__ w_hi,
                                                    const int64_t *__restrict__ w_send,
                                                    const int64_t *__restrict__ w_sstart,
                                                    const int32_t *__restrict__ w_next, int *__restrict__ state,
                                                    const int32_t *__restrict__ order, int64_t nw, int64_t cap,
                                                    unsigned long long *__restrict__ next,
                                                    int64_t *__restrict__ pos) {
    uint32_t n_seed = 0, r_seed = 0, r_walk = 0, n_claim = 0;  // this lane's counts (rb3_walk_stats)
    for (;;) {
        // warp-aggregated grab of one segment per active lane
        cg::coalesced_group grp = cg::coalesced_threads();
        unsigned long long base = 0;
        if (grp.thread_rank() == 0) base = atomicAdd(next, (unsigned long long)grp.size());
        base = grp.shfl(base, 0);
        const int64_t idx = (int64_t)base + grp.thread_rank();
        if (idx >= nw) {
            // the lanes leaving together add their counts with one atomic per counter
            cg::coalesced_group out = cg::coalesced_threads();
            const unsigned long long c0 = cg::reduce(out, (unsigned long long)n_seed, cg::plus<unsigned long long>());
            const unsigned long long c1 = cg::reduce(out, (unsigned long long)r_seed, cg::plus<unsigned long long>());
            const unsigned long long c2 = cg::reduce(out, (unsigned long long)r_walk, cg::plus<unsigned long long>());
            const unsigned long long c3 = cg::reduce(out, (unsigned long long)n_claim, cg::plus<unsigned long long>());
            if (out.thread_rank() == 0) {
                atomicAdd(&g_walk_stats[0], c0);
                atomicAdd(&g_walk_stats[1], c1);
                atomicAdd(&g_walk_stats[2], c2);
                atomicAdd(&g_walk_stats[3], c3);
            }
            break;
        }
        const int32_t w = order[idx];
        const int64_t hi = w_hi[w], send = w_send[w];
        int64_t l;
        if (hi == send) {  // top segment: starts at the string's sentinel, row isa2[hi]
            l = m1;
            const int64_t k = isa2[hi];
            pos[k] = k + l;
        } else {
            if (load_state(&state[w]) == ST_CLAIMED) continue;
            ++n_seed;
            l = DS ? seed_forward<NS>(B1, T2, hi, send, cap, &state[w], &r_seed)
                   : seed_backward<NS>(B1, m1, T2, hi, send, cap, &state[w], &r_seed);
            if (l < 0) continue;
            if (atomicCAS(&state[w], ST_PENDING, ST_RESOLVED) == ST_CLAIMED) continue;
        }
        const int64_t lo = w_sstart[w];
        int32_t nx = w_next[w];
        int64_t bnd = nx >= 0 ? w_hi[nx] : lo;
        int64_t p = hi - 1;
        if (p < lo) continue;
        int a = T2[p];
        int64_t k = isa2[p];
        for (;;) {
            // next position's symbol and row, loaded while this step's block is in flight
            int an = 0;
            int64_t kn = 0;
            if (p > lo) {
                an = T2[p - 1];
                kn = isa2[p - 1];
            }
            l = C_of(B1, a) + rank1<NS>(B1, a, l);
            pos[k] = k + l;
            ++r_walk;
            if (p == bnd && nx >= 0) {
                // reached the top of segment nx: stop if its seed is in, else take it over
                if (atomicCAS(&state[nx], ST_PENDING, ST_CLAIMED) == ST_RESOLVED) break;
                ++n_claim;
                nx = w_next[nx];
                bnd = nx >= 0 ? w_hi[nx] : lo;
            }
            if (--p < lo) break;
            a = an;
            k = kn;
        }
    }
}

// ---- segmented walk with bounded seeds: candidate tops, resolved afterwards ----------
// The takeover chain above is exact but its depth is the longest stretch of a
// new string that the index already holds (one dependent rank per symbol):
// when a new string equals an indexed one to its sentinel, every seed runs to
// the string end and the walk from above crosses the whole string.  Here no
// segment waits for another:
//  (1) k_walk_seeded: every segment's seed stops after `cap` extensions (and
//      once its interval holds at most CAND_MAX B1 suffixes).  Its bi-interval
//      (k, k', s) then says that the s B1 suffixes of rows [k, k+s) share the
//      seed's prefix with X, so l(X) is one of the s + 1 values k .. k+s.  The
//      segment walks all of them at once: the values stay s + 1 consecutive
//      rows' images under pi_{B1}(a, .), which is monotone and grows by
//      [B1[r] = a] from row r to r + 1, so they are held as the smallest value
//      v and a mask M (bit j - 1 set iff candidate j's value is candidate
//      j - 1's plus one).  One step reads the block of v (the rank) and the
//      symbols of rows v .. v + popcount(M) - 1, nearly always in the same
//      32-byte block: a step costs what a one-value step costs.  When M becomes
//      0 every candidate has the same value, which is then exact, and pos is
//      written from there on.  The segment stores its candidates' values at
//      its lower end (v, M).
//  (2) the resolve pass (k_res_chunk, k_res_carry, k_res_apply): the true
//      value at the top of segment w + 1 is the value of w's true candidate at
//      w's lower end, starting from the sentinel (exact); a scan along each
//      string of maps between candidate indexes (below).  An inconsistent
//      value (outside the next segment's candidates) is reported.
//  (3) k_rewalk: each segment whose walk did not converge before its end walks
//      its unwritten positions again from its true top value.
// Depth: cap + the longest segment, twice, plus the resolve pass; it does not
// grow with the length of a match.  A seed whose interval still holds more
// than CAND_MAX suffixes after cap extensions extends on until it holds at
// most CAND_MAX (or resolves): content held by more than CAND_MAX copies is
// the remaining case whose depth grows with the match.
constexpr int CAND_MAX = 63;  // candidates k .. k+s, s <= 63: the mask fits 64 bits
constexpr int REWALK_CK = 64;  // positions between checkpoints of the candidate walk (a power of two)

// bit t of the result = [B[r0 + t] == a] for t < d (1 <= d <= 63, r0 + d <= n);
// higher bits are unspecified.  D = 32: up to three blocks' planes; D >= 64:
// up to two 64-symbol payload sectors; run-length: the runs over [r0, r0 + d),
// decoded from the last mark before r0 (two spans at most).
template <int NS>
__device__ __forceinline__ uint64_t eq_bits(const OccView &v, int64_t r0, int d, int a) {
    if constexpr (NS == NS_RLE) {
        const int64_t rend = r0 + d;
        uint64_t e = 0;
        for (int64_t r = r0; r < rend;) {
            const int64_t sp = r >> v.log2D, s0 = sp << v.log2D;
            int64_t slen = v.n - s0;
            if (slen > ((int64_t)1 << v.log2D)) slen = (int64_t)1 << v.log2D;
            int64_t base[SIGMA], pos;
            uint64_t acc[2];
            RunRd rd;
            rd.init(rle_start(v, sp, r - s0, base, &pos, acc));
            while (pos < slen && s0 + pos < rend) {
                int b;
                int64_t len;
                rd.run(&b, &len);
                const int64_t lo = s0 + pos > r0 ? s0 + pos : r0, hi = s0 + pos + len < rend ? s0 + pos + len : rend;
                if (b == a && hi > lo) e |= ((1ull << (hi - lo)) - 1ull) << (lo - r0);
                pos += len;
            }
            r = s0 + slen;
        }
        return e;
    } else if constexpr (NS == 0) {
        const uint8_t *b = v.blocks + (r0 >> 5) * 32;
        const int o = (int)(r0 & 31);
        uint64_t e = (uint64_t)(s32_match(ld_sec64(b), a) >> o);
        int got = 32 - o;
        if (d > got) {
            e |= (uint64_t)s32_match(ld_sec64(b + 32), a) << got;
            got += 32;
            if (d > got) e |= (uint64_t)s32_match(ld_sec64(b + 64), a) << got;
        }
        return e;
    } else {
        const int D = 64 * NS;
        auto sec_of = [&](int64_t r) {
            return v.blocks + (r >> v.log2D) * (int64_t)v.bb + HEADER_BYTES + 32 * ((int)(r & (D - 1)) >> 6);
        };
        auto match64 = [&](const Sec &s) {
            const uint64_t p0 = sec_plane(s, 0), p1 = sec_plane(s, 1), p2 = sec_plane(s, 2);
            return ((a & 1) ? p0 : ~p0) & ((a & 2) ? p1 : ~p1) & ((a & 4) ? p2 : ~p2);
        };
        const int bit = (int)(r0 & 63);
        uint64_t e = match64(ld_sec64(sec_of(r0))) >> bit;
        const int got = 64 - bit;
        if (d > got) e |= match64(ld_sec64(sec_of((r0 | 63) + 1))) << got;
        return e;
    }
}

// Bits of e deposited, in order, at the set bits of m (bit t of e goes to the
// t-th set bit of m).
__device__ __forceinline__ uint64_t deposit_bits(uint64_t e, uint64_t m) {
    uint64_t r = 0;
    while (m) {
        const uint64_t b = m & (~m + 1ull);
        if (e & 1ull) r |= b;
        e >>= 1;
        m ^= b;
    }
    return r;
}

// Candidate seed over a double-strand B1: ForwardExt along X = T2[x, send)$
// until the count is 0 (exact: the k field), X's sentinel (exact: k +
// occ(Q$)), or, after cap extensions, an interval of at most CAND_MAX rows
// (candidates k .. k+s).  Returns k; *s_out = 0 when exact.
template <int NS>
__device__ __forceinline__ int64_t seed_forward_cand(const OccView &B1, const uint8_t *__restrict__ T2, int64_t x,
                                                     int64_t send, int64_t cap, int *s_out, uint32_t *reads) {
    BiInt q = {0, 0, B1.n};
    int a = T2[x];
    const int lg = NS == 0 ? 5 : B1.log2D;
    for (int64_t t = 0;; ++t) {
        const int64_t p = x + t;
        if (p == send) {
            *reads += 2;
            *s_out = 0;
            return q.k + (rank1<NS>(B1, 0, q.kp + q.s) - rank1<NS>(B1, 0, q.kp));
        }
        if (t >= cap && q.s <= CAND_MAX) {
            *s_out = (int)q.s;
            return q.k;
        }
        const int an = T2[p + 1];
        *reads += ((q.kp + q.s) >> lg) == (q.kp >> lg) ? 1u : 2u;
        const BiInt y = forward_ext<NS>(B1, q, a);
        if (y.s == 0) {
            *s_out = 0;
            return y.k;
        }
        q = y;
        a = an;
    }
}

// Candidate seed over any B1 (single strand: no ForwardExt): the SA interval
// [lo, hi) of T2[x, y), y = min(x + c, send), by backward search; exact once
// the interval is empty (l = lo) or when y = send (from the sentinel, l = m1);
// else the candidates are lo .. hi if hi - lo <= CAND_MAX, otherwise the
// window doubles.
template <int NS>
__device__ __forceinline__ int64_t seed_backward_cand(const OccView &B1, int64_t m1, const uint8_t *__restrict__ T2,
                                                      int64_t x, int64_t send, int64_t cap, int *s_out,
                                                      uint32_t *reads) {
    for (int64_t c = cap > 0 ? cap : 1;; c *= 2) {
        const int64_t y = x + c < send ? x + c : send;
        bool exact = y == send;
        int64_t lo = exact ? m1 : 0, hi = exact ? m1 : B1.n;
        for (int64_t p = y - 1; p >= x; --p) {
            const int a = T2[p];
            *reads += exact ? 1u : 2u;
            if (exact) {
                lo = C_of(B1, a) + rank1<NS>(B1, a, lo);
                hi = lo;
            } else {
                BlockLd<NS> bl = block_load<NS>(B1, lo), bh = block_load<NS>(B1, hi);
                lo = C_of(B1, a) + block_rank<NS>(bl, a);
                hi = C_of(B1, a) + block_rank<NS>(bh, a);
                exact = lo == hi;
            }
        }
        if (exact || hi - lo <= CAND_MAX) {
            *s_out = exact ? 0 : (int)(hi - lo);
            return lo;
        }
    }
}

// Walk counters of the bounded-seed form: [0] seeds, [1] seed block reads,
// [2] block reads of walk steps (both passes), [3] positions walked again.
template <int NS, bool DS>
__global__ void __launch_bounds__(WALK_THREADS, 32)
    k_walk_seeded(OccView B1, int64_t m1, const uint8_t *__restrict__ T2, const int32_t *__restrict__ isa2,
                  const int64_t *__restrict__ w_hi, const int64_t *__restrict__ w_send,
                  const int64_t *__restrict__ w_sstart, const int32_t *__restrict__ w_next,
                  const int32_t *__restrict__ order, int64_t nw, int64_t cap, unsigned long long *__restrict__ next,
                  int64_t *__restrict__ pos, int64_t *__restrict__ seg_lo, int32_t *__restrict__ seg_n,
                  int64_t *__restrict__ bot_v, uint64_t *__restrict__ bot_m, int64_t *__restrict__ unw_lo,
                  int64_t *__restrict__ ck_v, uint64_t *__restrict__ ck_m, int ck_per_seg,
                  unsigned int *__restrict__ err) {
    uint32_t n_seed = 0, r_seed = 0, r_walk = 0;
    for (;;) {
        cg::coalesced_group grp = cg::coalesced_threads();
        unsigned long long base = 0;
        if (grp.thread_rank() == 0) base = atomicAdd(next, (unsigned long long)grp.size());
        base = grp.shfl(base, 0);
        const int64_t idx = (int64_t)base + grp.thread_rank();
        if (idx >= nw) {
            cg::coalesced_group out = cg::coalesced_threads();
            const unsigned long long c0 = cg::reduce(out, (unsigned long long)n_seed, cg::plus<unsigned long long>());
            const unsigned long long c1 = cg::reduce(out, (unsigned long long)r_seed, cg::plus<unsigned long long>());
            const unsigned long long c2 = cg::reduce(out, (unsigned long long)r_walk, cg::plus<unsigned long long>());
            if (out.thread_rank() == 0) {
                atomicAdd(&g_walk_stats[0], c0);
                atomicAdd(&g_walk_stats[1], c1);
                atomicAdd(&g_walk_stats[2], c2);
            }
            break;
        }
        const int32_t w = order[idx];
        const int64_t hi = w_hi[w], send = w_send[w], lo = w_sstart[w];
        const int32_t nx = w_next[w];
        const int64_t bnd = nx >= 0 ? w_hi[nx] : lo;
        int64_t v;
        int s = 0;
        if (hi == send) {  // top segment: starts at the string's sentinel, row isa2[hi]
            v = m1;
            const int64_t k = isa2[hi];
            pos[k] = k + v;
        } else {
            ++n_seed;
            v = DS ? seed_forward_cand<NS>(B1, T2, hi, send, cap, &s, &r_seed)
                   : seed_backward_cand<NS>(B1, m1, T2, hi, send, cap, &s, &r_seed);
        }
        seg_lo[w] = v;
        seg_n[w] = s;
        if (hi - bnd >= (int64_t)ck_per_seg * REWALK_CK) {  // the plan bounds every segment below this
            atomicOr(err, 8u);
            continue;
        }
        uint64_t M = s ? (s == 64 ? ~0ull : ((1ull << s) - 1ull)) : 0ull;
        int64_t unw = M ? bnd : hi;  // lowest position not written (hi: none)
        int64_t p = hi - 1;
        if (p >= lo) {
            int a = T2[p];
            int64_t k = isa2[p];
            for (;;) {
                int an = 0;
                int64_t kn = 0;
                if (p > bnd) {
                    an = T2[p - 1];
                    kn = isa2[p - 1];
                }
                ++r_walk;
                if (M == 0) {
                    v = C_of(B1, a) + rank1<NS>(B1, a, v);
                    pos[k] = k + v;
                } else {
                    const int d = __popcll(M);
                    if (v + d > B1.n) {  // candidates are rows of B1: cannot happen on valid inputs
                        atomicOr(err, 2u);
                        break;
                    }
                    const int64_t vn = C_of(B1, a) + rank1<NS>(B1, a, v);
                    M = deposit_bits(eq_bits<NS>(B1, v, d, a), M);
                    v = vn;
                    if (M == 0) {  // the candidates met: exact from here down
                        pos[k] = k + v;
                        unw = p + 1;
                    } else if (((hi - p) & (REWALK_CK - 1)) == 0) {
                        // checkpoint t: the candidates' values at p = hi - t * REWALK_CK, from
                        // which the second walk restarts once the true candidate is known
                        const int64_t t = (hi - p) / REWALK_CK;
                        if (t < ck_per_seg) {
                            ck_v[(int64_t)w * ck_per_seg + t] = v;
                            ck_m[(int64_t)w * ck_per_seg + t] = M;
                        }
                    }
                }
                if (--p < bnd) break;
                a = an;
                k = kn;
            }
        }
        bot_v[w] = v;
        bot_m[w] = M;
        unw_lo[w] = unw;
    }
}

// ---- the resolve pass: which candidate of every segment top is the true one ----
// The true candidate j(w+1) at segment w+1's top is F_w(j(w)), where F_w maps a
// candidate index at w's top to the index, among w+1's candidates, of its value
// at w's lower end: F_w(j) = clamp(o + popcount(m & low_j), 0, n_{w+1}), o =
// (w's lowest bottom value) - (w+1's first candidate), m = w's bottom mask.
// Values outside w+1's candidates belong to false candidates only, so clamping
// them changes nothing that matters, and keeps F_w monotone with steps of 0 or
// 1: F_w is then (c, M): F(j) = c + popcount(M & low_j).  Such maps compose
// into maps of the same kind (G after F: c = G(F.c), M = the bits of G.M from
// F.c on, deposited at the set bits of F.M), so the j of every segment is an
// inclusive scan of the maps along its string, started from j = 0 at the
// string's top (its sentinel's value is exact):
//   k_res_chunk: one warp per chunk of up to 32 segments of one string, a warp
//     scan of the composition; prefix maps per segment, the chunk's aggregate;
//   k_res_carry: one warp per string, the chunks' aggregates in order (32
//     loaded at once, applied one after another): each chunk's entry j;
//   k_res_apply: one thread per segment, its j from its chunk's entry j and
//     the prefix map before it; top_l = first candidate + j, and the check
//     that the true value lies among the next segment's candidates.
struct CandMap {
    int c;
    uint64_t M;
};

__device__ __forceinline__ int cmap_at(const CandMap &f, int j) { return f.c + __popcll(f.M & prefix_mask(j)); }

// g after f
__device__ __forceinline__ CandMap cmap_then(const CandMap &f, const CandMap &g) {
    CandMap h;
    h.c = cmap_at(g, f.c);
    h.M = deposit_bits(f.c < 64 ? (g.M >> f.c) : 0ull, f.M);
    return h;
}

// F_w in (c, M) form from o, m and the next segment's candidate count nn
__device__ __forceinline__ CandMap cmap_of(int64_t o, uint64_t m, int nn) {
    CandMap f;
    f.c = o < 0 ? 0 : (o > nn ? nn : (int)o);
    // the t-th set bit of m moves the raw value from o + t to o + t + 1: it is a
    // step of the clamped map iff 0 <= o + t and o + t + 1 <= nn
    uint64_t r = 0;
    int64_t t = 0;
    while (m) {
        const uint64_t b = m & (~m + 1ull);
        if (o + t >= 0 && o + t + 1 <= nn) r |= b;
        m ^= b;
        ++t;
    }
    f.M = r;
    return f;
}

__device__ __forceinline__ CandMap cmap_shfl_up(const CandMap &f, int d) {
    CandMap g;
    g.c = __shfl_up_sync(0xffffffffu, f.c, d);
    g.M = __shfl_up_sync(0xffffffffu, f.M, d);
    return g;
}

// chunk q: segments [ch_w0[q], ch_w0[q] + ch_cnt[q]) of one string; seg_last[w]
// set for the last segment of a string (it has no next segment)
__global__ void k_res_chunk(const int32_t *__restrict__ ch_w0, const int32_t *__restrict__ ch_cnt, int64_t nch,
                            const int64_t *__restrict__ seg_lo, const int32_t *__restrict__ seg_n,
                            const int64_t *__restrict__ bot_v, const uint64_t *__restrict__ bot_m,
                            const uint8_t *__restrict__ seg_last, int32_t *__restrict__ pre_c,
                            uint64_t *__restrict__ pre_m, int32_t *__restrict__ agg_c, uint64_t *__restrict__ agg_m) {
    const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= nch) return;  // the warp leaves together
    const int64_t w = (int64_t)ch_w0[q] + lane;
    const int cnt = ch_cnt[q];
    CandMap f = {0, 0ull};
    if (lane < cnt && !seg_last[w]) f = cmap_of(bot_v[w] - seg_lo[w + 1], bot_m[w], seg_n[w + 1]);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const CandMap g = cmap_shfl_up(f, d);
        if (lane >= d) f = cmap_then(g, f);
    }
    if (lane < cnt) {
        pre_c[w] = f.c;
        pre_m[w] = f.M;
    }
    if (lane == cnt - 1) {
        agg_c[q] = f.c;
        agg_m[q] = f.M;
    }
}

// string s: chunks [choff[s], choff[s+1]); entry[q] = the true candidate at the
// top of chunk q's first segment
__global__ void k_res_carry(const int32_t *__restrict__ choff, int64_t ns, const int32_t *__restrict__ agg_c,
                            const uint64_t *__restrict__ agg_m, int32_t *__restrict__ entry) {
    const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= ns) return;
    const int64_t q0 = choff[s], q1 = choff[s + 1];
    int j = 0;
    for (int64_t b = q0; b < q1; b += 32) {
        const int64_t q = b + lane;
        CandMap f = {0, 0ull};
        if (q < q1) f = CandMap{agg_c[q], agg_m[q]};
        const int cnt = q1 - b < 32 ? (int)(q1 - b) : 32;
        int mine = 0;
        for (int i = 0; i < cnt; ++i) {
            const int ci = __shfl_sync(0xffffffffu, f.c, i);
            const uint64_t mi = __shfl_sync(0xffffffffu, f.M, i);
            if (lane == i) mine = j;
            j = ci + __popcll(mi & prefix_mask(j));
        }
        if (q < q1) entry[q] = mine;
    }
}

__global__ void k_res_apply(const int32_t *__restrict__ seg_chunk, const int32_t *__restrict__ ch_w0, int64_t nw,
                            const int32_t *__restrict__ entry, const int32_t *__restrict__ pre_c,
                            const uint64_t *__restrict__ pre_m, const int64_t *__restrict__ seg_lo,
                            const int32_t *__restrict__ seg_n, const int64_t *__restrict__ bot_v,
                            const uint64_t *__restrict__ bot_m, const uint8_t *__restrict__ seg_last,
                            int64_t *__restrict__ top_l, unsigned int *__restrict__ err) {
    const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w >= nw) return;
    const int32_t q = seg_chunk[w];
    const int e = entry[q];
    const int j = w == ch_w0[q] ? e : cmap_at(CandMap{pre_c[w - 1], pre_m[w - 1]}, e);
    top_l[w] = seg_lo[w] + j;
    bool bad = j < 0 || j > seg_n[w];
    if (!seg_last[w]) {  // the true value at the lower end must be one of the next top's candidates
        const int64_t v = bot_v[w] + __popcll(bot_m[w] & prefix_mask(j)) - seg_lo[w + 1];
        bad |= v < 0 || v > seg_n[w + 1];
    }
    if (bad) atomicOr(err, 1u);
}

// Positions [unw_lo[w], hi) of every segment, walked again from the exact
// value: in pieces of REWALK_CK positions, piece t starting at hi - t *
// REWALK_CK from the top value (t = 0) or from checkpoint t of the candidate
// walk, so that the pieces run side by side instead of one chain per segment.
// Unit u = (order position u / ck_per_seg, piece u % ck_per_seg).
template <int NS>
__global__ void __launch_bounds__(WALK_THREADS, 32)
    k_rewalk(OccView B1, const uint8_t *__restrict__ T2, const int32_t *__restrict__ isa2,
             const int64_t *__restrict__ w_hi, const int64_t *__restrict__ unw_lo, const int64_t *__restrict__ top_l,
             const int64_t *__restrict__ seg_lo, const int64_t *__restrict__ ck_v, const uint64_t *__restrict__ ck_m,
             int ck_per_seg, const int32_t *__restrict__ order, int64_t nw, unsigned long long *__restrict__ next,
             int64_t *__restrict__ pos, unsigned int *__restrict__ err) {
    uint32_t r_walk = 0, r_again = 0;
    const int64_t nu = nw * ck_per_seg;
    for (;;) {
        cg::coalesced_group grp = cg::coalesced_threads();
        unsigned long long base = 0;
        if (grp.thread_rank() == 0) base = atomicAdd(next, (unsigned long long)grp.size());
        base = grp.shfl(base, 0);
        const int64_t idx = (int64_t)base + grp.thread_rank();
        if (idx >= nu) {
            cg::coalesced_group out = cg::coalesced_threads();
            const unsigned long long c2 = cg::reduce(out, (unsigned long long)r_walk, cg::plus<unsigned long long>());
            const unsigned long long c3 = cg::reduce(out, (unsigned long long)r_again, cg::plus<unsigned long long>());
            if (out.thread_rank() == 0) {
                atomicAdd(&g_walk_stats[2], c2);
                atomicAdd(&g_walk_stats[3], c3);
            }
            break;
        }
        const int32_t w = order[idx / ck_per_seg];
        const int64_t t = idx % ck_per_seg;
        const int64_t hi = w_hi[w], u = unw_lo[w];
        const int64_t top = hi - t * REWALK_CK;  // this piece walks [max(u, top - REWALK_CK), top)
        if (top <= u) continue;
        const int64_t stop = top - REWALK_CK > u ? top - REWALK_CK : u;
        int64_t l;
        if (t == 0) {
            l = top_l[w];
        } else {
            const int j = (int)(top_l[w] - seg_lo[w]);
            l = ck_v[(int64_t)w * ck_per_seg + t] + __popcll(ck_m[(int64_t)w * ck_per_seg + t] & prefix_mask(j));
        }
        if (l < 0 || l > B1.n) {  // a value of B1's rows; anything else is reported, never read with
            atomicOr(err, 16u);
            continue;
        }
        int64_t p = top - 1;
        int a = T2[p];
        int64_t k = isa2[p];
        for (;;) {
            int an = 0;
            int64_t kn = 0;
            if (p > stop) {
                an = T2[p - 1];
                kn = isa2[p - 1];
            }
            l = C_of(B1, a) + rank1<NS>(B1, a, l);
            pos[k] = k + l;
            ++r_walk;
            ++r_again;
            if (--p < stop) break;
            a = an;
            k = kn;
        }
    }
}

// ---- scatter-merge (S4) + Occ rebuild ---------------------------------------------
// Tiles of MT output symbols.  kstart[t] = number of B2 rows with pos < t*MT.
constexpr int MT = 2048;
constexpr int MT_THREADS = MT / 8;
// CTAs per SM asked of the register allocator: a tile is short and latency-bound
// (its phases wait on pos, then on the input blocks), so residency is what hides it.
#ifndef RB3_SCATTER_MINB
#define RB3_SCATTER_MINB 8
#endif

__global__ void k_tile_starts(const int64_t *__restrict__ pos, int64_t n2, int64_t ntiles,
                              int64_t *__restrict__ kstart) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k > n2) return;
    int64_t tk = k < n2 ? pos[k] / MT : ntiles;           // tile of row k (ntiles past the end)
    int64_t tp = k > 0 ? pos[k - 1] / MT : -1;           // tile of row k-1
    for (int64_t t = tp + 1; t <= tk && t < ntiles + 1; ++t) kstart[t] = k;
}

// Plane bits of the cnt (<= 8) consecutive symbols starting at row `start`:
// out[b] bit j = bit b of the code of symbol start + j.  The run may cross
// into the next sector (of the same block or the next block).
__device__ __forceinline__ void plane_bits(const OccView &v, int64_t start, int cnt, uint32_t out[3]) {
    out[0] = out[1] = out[2] = 0u;
    if (cnt <= 0) return;
    if (v.log2D == 5) {  // D = 32: 32-bit planes at words 5..7 of each block
        const uint32_t *w = reinterpret_cast<const uint32_t *>(v.blocks + (start >> 5) * 32);
        const int bit = (int)(start & 31);
        const uint32_t m = (1u << cnt) - 1u;
#pragma unroll
        for (int b = 0; b < 3; ++b) out[b] = (__ldg(w + 5 + b) >> bit) & m;
        if (bit + cnt > 32) {
#pragma unroll
            for (int b = 0; b < 3; ++b) out[b] |= (__ldg(w + 8 + 5 + b) << (32 - bit)) & m;
        }
        return;
    }
    const int D = 1 << v.log2D;
    const int o = (int)(start & (D - 1));
    const uint8_t *sec = v.blocks + (start >> v.log2D) * (int64_t)v.bb + HEADER_BYTES + 32 * (o >> 6);
    const int bit = o & 63;
    const uint32_t m = (1u << cnt) - 1u;
#pragma unroll
    for (int b = 0; b < 3; ++b) out[b] = (uint32_t)(ldg_u64(sec + 8 * b) >> bit) & m;
    if (bit + cnt > 64) {
        const int64_t nxt = (start | 63) + 1;  // first row of the next sector
        const int on = (int)(nxt & (D - 1));
        const uint8_t *sec2 = v.blocks + (nxt >> v.log2D) * (int64_t)v.bb + HEADER_BYTES + 32 * (on >> 6);
#pragma unroll
        for (int b = 0; b < 3; ++b) out[b] |= (uint32_t)(ldg_u64(sec2 + 8 * b) << (64 - bit)) & m;
    }
}

// Rank of every symbol at each tile start of the merged BWT: rank_B1 at the
// number of B1 rows before it plus rank_B2 at the number of B2 rows before it.
__global__ void k_tile_bases(OccView B1, OccView B2, const int64_t *__restrict__ kstart, int64_t ntiles,
                             int64_t *__restrict__ base6) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const int64_t k0 = kstart[t], j0 = t * MT - k0;
    int64_t r1[SIGMA], r2[SIGMA];
    rank_all_any(B1, j0, r1);
    rank_all_any(B2, k0, r2);
#pragma unroll
    for (int a = 0; a < SIGMA; ++a) base6[t * SIGMA + a] = r1[a] + r2[a];
}

__global__ void __launch_bounds__(MT_THREADS, RB3_SCATTER_MINB) k_scatter(OccView B1, OccView B2, const int64_t *__restrict__ pos,
                                                        const int64_t *__restrict__ kstart,
                                                        const int64_t *__restrict__ tbase, int64_t nM, int64_t nbM,
                                                        int log2D, int bb, uint8_t *__restrict__ M) {
    __shared__ uint32_t flags[MT / 32];
    __shared__ uint32_t wtot[32];
    __shared__ int64_t base6[SIGMA];
    __shared__ uint32_t bcnt[MT / 32][SIGMA];  // per 32-symbol group counts
    const int64_t t = blockIdx.x;
    const int64_t q0 = t * MT;
    const int64_t k0 = kstart[t], k1 = kstart[t + 1];
    const int64_t j0 = q0 - k0;
    for (int i = threadIdx.x; i < MT / 32; i += MT_THREADS) flags[i] = 0;
    if (threadIdx.x < SIGMA) base6[threadIdx.x] = tbase[t * SIGMA + threadIdx.x];
    for (int i = threadIdx.x; i < (MT / 32) * SIGMA; i += MT_THREADS) (&bcnt[0][0])[i] = 0;
    __syncthreads();
    for (int64_t k = k0 + threadIdx.x; k < k1; k += MT_THREADS) {
        int d = (int)(pos[k] - q0);
        atomicOr(&flags[d >> 5], 1u << (d & 31));
    }
    __syncthreads();
    // thread owns output symbols [q0 + 8*tid, +8)
    const int o8 = threadIdx.x * 8;
    uint32_t fw = (flags[o8 >> 5] >> (o8 & 31)) & 0xFFu;
    uint32_t nf = __popc(fw);
    uint32_t before = block_excl<uint32_t>(nf, 0, wtot);
    int64_t kb = k0 + before;              // next B2 row
    int64_t jb = j0 + (o8 - (int64_t)before);  // next B1 row
    // symbols of this thread: the flagged ones are the next B2 rows, the others the next B1 rows
    const int64_t qt = q0 + o8;
    const int valid = qt >= nM ? 0 : (nM - qt < 8 ? (int)(nM - qt) : 8);
    const int n2t = (int)nf, n1t = valid - (int)nf;
    uint32_t s1[3], s2[3];
    plane_bits(B1, jb, n1t, s1);
    plane_bits(B2, kb, n2t, s2);
    uint32_t pl[3] = {0, 0, 0};  // plane bytes of these 8 output symbols
    int i1 = 0, i2 = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (j < valid) {
            const bool from2 = (fw >> j) & 1u;
            const int sh = from2 ? i2 : i1;
#pragma unroll
            for (int b = 0; b < 3; ++b) pl[b] |= (((from2 ? s2[b] : s1[b]) >> sh) & 1u) << j;
            i2 += from2;
            i1 += !from2;
        }
    }
    uint32_t c[SIGMA];
    {
        const uint32_t mv = (1u << valid) - 1u;
        const uint32_t b0 = pl[0], n0 = ~pl[0] & mv, t00 = ~pl[1] & ~pl[2] & mv, t10 = pl[1] & ~pl[2],
                       t01 = ~pl[1] & pl[2];
        c[0] = __popc(n0 & t00);
        c[1] = __popc(b0 & t00);
        c[2] = __popc(n0 & t10);
        c[3] = __popc(b0 & t10);
        c[4] = __popc(n0 & t01);
        c[5] = __popc(b0 & t01);
    }
    // counts per 32-symbol group (4 threads)
    const int grp = o8 >> 5;
#pragma unroll
    for (int a = 0; a < SIGMA; ++a)
        if (c[a]) atomicAdd(&bcnt[grp][a], c[a]);
    __syncthreads();
    // exclusive prefix over the groups, one thread per symbol: bcnt[g][a] = count
    // of a in the tile's symbols before group g
    if (threadIdx.x < SIGMA) {
        uint32_t run = 0;
        for (int g = 0; g < MT / 32; ++g) {
            const uint32_t v = bcnt[g][threadIdx.x];
            bcnt[g][threadIdx.x] = run;
            run += v;
        }
    }
    __syncthreads();
    // write payload word; headers at block starts
    const int D = 1 << log2D;
    const int64_t q = q0 + o8;
    const bool live = (q >> log2D) < nbM;  // past the last output block nothing is stored
    uint8_t *blk = M + (q >> log2D) * (int64_t)bb;
    const int o = (int)(q & (D - 1));
    if (log2D == 5) store_planes32(blk, pl[0], pl[1], pl[2], 0xffffffffu, live);
    else store_planes(blk + HEADER_BYTES + 32 * (o >> 6), pl[0], pl[1], pl[2], 0xffffffffu, live);
    if (!live) return;  // no barrier follows
    if (o == 0 && log2D == 5) {
        // D = 32: rank at q relative to the start of q's 2^32-symbol span, whose
        // absolute ranks are those of the tile that starts there
        const int ng = o8 >> 5;
        const int64_t gi = q >> GSPAN_LOG2;
        uint32_t *h32 = reinterpret_cast<uint32_t *>(blk);
#pragma unroll
        for (int a = 1; a < SIGMA; ++a) {
            int64_t r = base6[a] + bcnt[ng][a];
            if (gi) r -= tbase[((gi << GSPAN_LOG2) / MT) * SIGMA + a];
            h32[a - 1] = (uint32_t)r;
        }
    } else if (o == 0) {
        // rank at q = base + counts of the groups of this tile before q
        int ng = o8 >> 5;
        uint32_t *h32 = reinterpret_cast<uint32_t *>(blk);
        uint8_t hb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int a = 0; a < SIGMA; ++a) {
            int64_t r = base6[a] + bcnt[ng][a];
            h32[a] = (uint32_t)r;
            hb[a] = (uint8_t)(r >> 32);
        }
        *reinterpret_cast<uint2 *>(blk + 24) =
            make_uint2((uint32_t)hb[0] | ((uint32_t)hb[1] << 8) | ((uint32_t)hb[2] << 16) | ((uint32_t)hb[3] << 24),
                       (uint32_t)hb[4] | ((uint32_t)hb[5] << 8));
    }
}

static inline unsigned nb_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

int walk_stats(int64_t out[4], bool reset) {
    unsigned long long h[4];
    RB3_CUDA_TRY(cudaMemcpyFromSymbol(h, g_walk_stats, sizeof(h)));
    for (int i = 0; i < 4; ++i) out[i] = (int64_t)h[i];
    if (reset) {
        const unsigned long long z[4] = {0, 0, 0, 0};
        RB3_CUDA_TRY(cudaMemcpyToSymbol(g_walk_stats, z, sizeof(z)));
    }
    return RB3_OK;
}

// ---- sampled suffix array through a merge ---------------------------------------
// The merged rows come from B1 and B2 in the interleaving pos gives, so the
// merged sample set is the two inputs' sets interleaved the same way; a B2
// value's string index moves past B1's m1 strings.  Tiles as in k_scatter:
// thread owns merged rows [q0 + 8 tid, +8), the flagged ones being the next B2
// rows, the others the next B1 rows.
struct MergeRows {
    uint32_t fw;  // bit i: row i of the thread's 8 comes from B2
    int64_t kb, jb, q;
    int valid;
};

__device__ __forceinline__ MergeRows merge_rows(const int64_t *__restrict__ pos, const int64_t *__restrict__ kstart,
                                                int64_t nM, uint32_t *flags, uint32_t *wtot) {
    const int64_t t = blockIdx.x;
    const int64_t q0 = t * MT;
    const int64_t k0 = kstart[t], k1 = kstart[t + 1];
    for (int i = threadIdx.x; i < MT / 32; i += MT_THREADS) flags[i] = 0;
    __syncthreads();
    for (int64_t k = k0 + threadIdx.x; k < k1; k += MT_THREADS) {
        const int d = (int)(pos[k] - q0);
        atomicOr(&flags[d >> 5], 1u << (d & 31));
    }
    __syncthreads();
    MergeRows r;
    const int o8 = threadIdx.x * 8;
    r.fw = (flags[o8 >> 5] >> (o8 & 31)) & 0xFFu;
    const uint32_t before = block_excl<uint32_t>(__popc(r.fw), 0, wtot);
    r.kb = k0 + before;
    r.jb = (q0 - k0) + (o8 - (int64_t)before);
    r.q = q0 + o8;
    r.valid = r.q >= nM ? 0 : (nM - r.q < 8 ? (int)(nM - r.q) : 8);
    return r;
}

__device__ __forceinline__ bool sample_bit(const uint64_t *__restrict__ sdir, int64_t j) {
    return (sdir[2 * (j >> 6)] >> (j & 63)) & 1u;
}

// Merged bit words (64 rows = 8 threads) and their sample counts.
__global__ void __launch_bounds__(MT_THREADS) k_smerge_bits(const uint64_t *__restrict__ sd1,
                                                            const uint64_t *__restrict__ sd2,
                                                            const int64_t *__restrict__ pos,
                                                            const int64_t *__restrict__ kstart, int64_t nM,
                                                            int64_t nwords, uint64_t *__restrict__ sdo,
                                                            uint64_t *__restrict__ cnt) {
    __shared__ uint32_t flags[MT / 32];
    __shared__ uint32_t wtot[32];
    const MergeRows r = merge_rows(pos, kstart, nM, flags, wtot);
    uint32_t byte = 0;
    int64_t j = r.jb, k = r.kb;
    for (int i = 0; i < r.valid; ++i) {
        const bool from2 = (r.fw >> i) & 1u;
        const bool b = from2 ? sample_bit(sd2, k++) : sample_bit(sd1, j++);
        byte |= (uint32_t)b << i;
    }
    const int jj = threadIdx.x & 7;
    uint64_t v = (uint64_t)byte << (8 * jj);
#pragma unroll
    for (int d = 1; d < 8; d <<= 1) v |= __shfl_xor_sync(0xffffffffu, v, d);
    const int64_t word = r.q >> 6;
    if (jj == 0 && word < nwords) {
        sdo[2 * word] = v;
        cnt[word] = __popcll(v);
    }
}

__global__ void k_sdir_ranks(const uint64_t *__restrict__ excl, int64_t nwords, uint64_t *__restrict__ sdo) {
    const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w < nwords) sdo[2 * w + 1] = excl[w];
}

// Merged values: a sampled merged row takes its source row's value.
__global__ void __launch_bounds__(MT_THREADS) k_smerge_vals(const uint64_t *__restrict__ sd1,
                                                            const uint64_t *__restrict__ sv1,
                                                            const uint64_t *__restrict__ sd2,
                                                            const uint64_t *__restrict__ sv2, int64_t m1,
                                                            const int64_t *__restrict__ pos,
                                                            const int64_t *__restrict__ kstart, int64_t nM,
                                                            const uint64_t *__restrict__ sdo,
                                                            uint64_t *__restrict__ svo) {
    __shared__ uint32_t flags[MT / 32];
    __shared__ uint32_t wtot[32];
    const MergeRows r = merge_rows(pos, kstart, nM, flags, wtot);
    int64_t j = r.jb, k = r.kb;
    for (int i = 0; i < r.valid; ++i) {
        const bool from2 = (r.fw >> i) & 1u;
        int64_t si;
        const bool smp = from2 ? sample_at(sd2, k, &si) : sample_at(sd1, j, &si);
        if (smp) {
            int64_t oi;
            sample_at(sdo, r.q + i, &oi);
            svo[oi] = from2 ? sv2[si] + ((uint64_t)m1 << SVAL_OFF_BITS) : sv1[si];
        }
        if (from2) ++k;
        else ++j;
    }
}

int sample_merge(const rb3_index *dst, const rb3_index *src, const int64_t *pos, const int64_t *kstart,
                 int64_t ntiles, int64_t nM, int tile_rows, rb3_index *out, cudaStream_t st) {
    (void)tile_rows;
    const int64_t nwords = nM / 64 + 1;
    uint64_t *sdo = nullptr, *svo = nullptr;
    RB3_TRY(dev_alloc((void **)&sdo, sizeof(uint64_t) * 2 * nwords, st));
    DevBuf cnt, excl;
    RB3_TRY(cnt.alloc(sizeof(uint64_t) * nwords, st));
    RB3_TRY(excl.alloc(sizeof(uint64_t) * nwords, st));
    RB3_CUDA_TRY(cudaMemsetAsync(sdo, 0, sizeof(uint64_t) * 2 * nwords, st));
    RB3_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(uint64_t) * nwords, st));
    RB3_LAUNCH(k_smerge_bits, (unsigned)ntiles, MT_THREADS, 0, st, dst->sdir, src->sdir, pos, kstart, nM, nwords,
               sdo, cnt.as<uint64_t>());
    RB3_TRY(scan_u64(cnt.as<uint64_t>(), excl.as<uint64_t>(), nwords, false, st));
    RB3_LAUNCH(k_sdir_ranks, nb_for(nwords, 256), 256, 0, st, excl.as<uint64_t>(), nwords, sdo);
    int64_t tail[2];
    RB3_CUDA_TRY(cudaMemcpyAsync(&tail[0], excl.as<uint64_t>() + nwords - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaMemcpyAsync(&tail[1], cnt.as<uint64_t>() + nwords - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    const int64_t ns = tail[0] + tail[1];
    if (ns != dst->n_samples + src->n_samples) {
        dev_free(sdo, st);
        set_error("merge: sampled rows %lld, inputs %lld + %lld", (long long)ns, (long long)dst->n_samples,
                  (long long)src->n_samples);
        return RB3_E_CUDA;
    }
    int r = dev_alloc((void **)&svo, sizeof(uint64_t) * (ns > 0 ? ns : 1), st);
    if (r != RB3_OK) {
        dev_free(sdo, st);
        return r;
    }
    RB3_LAUNCH(k_smerge_vals, (unsigned)ntiles, MT_THREADS, 0, st, dst->sdir, dst->svals, src->sdir, src->svals,
               dst->m, pos, kstart, nM, sdo, svo);
    out->sdir = sdo;
    out->svals = svo;
    out->n_samples = ns;
    return RB3_OK;
}

// Bytes one rank needs: the symbol's count word(s) and, on average, the payload
// before the offset (D = 32: the count word and the three 4-byte planes).
static inline double rank_bytes(int D) { return D == 32 ? 16.0 : 5.0 + D / 4.0; }

// gbase[5 g + a - 1] = rank(a, g * 2^32) = the tile base of the tile starting there.
__global__ void k_span_bases(const int64_t *__restrict__ tbase, int64_t rows, int64_t *__restrict__ gb) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows * 5) return;
    const int64_t g = i / 5;
    const int a = (int)(i % 5) + 1;
    gb[i] = tbase[((g << GSPAN_LOG2) / MT) * SIGMA + a];
}

template <int NS1>
static int launch_walk_plain_1(int D2, OccView V1, OccView V2, int64_t m1, int64_t m2, const uint8_t *own,
                               int64_t *pos, unsigned int *err, cudaStream_t st) {
    unsigned grid = nb_for(m2, 32);
    if (D2 == 32) {
        auto kern = k_walk_plain<NS1, 0>;
        RB3_LAUNCH(kern, grid, 32, 0, st, V1, V2, m1, m2, own, pos, err);
    } else if (D2 == 64) {
        auto kern = k_walk_plain<NS1, 1>;
        RB3_LAUNCH(kern, grid, 32, 0, st, V1, V2, m1, m2, own, pos, err);
    } else if (D2 == 128) {
        auto kern = k_walk_plain<NS1, 2>;
        RB3_LAUNCH(kern, grid, 32, 0, st, V1, V2, m1, m2, own, pos, err);
    } else {
        auto kern = k_walk_plain<NS1, 4>;
        RB3_LAUNCH(kern, grid, 32, 0, st, V1, V2, m1, m2, own, pos, err);
    }
    return RB3_OK;
}

static int launch_walk_plain(int D1, int D2, OccView V1, OccView V2, int64_t m1, int64_t m2, const uint8_t *own,
                             int64_t *pos, unsigned int *err, cudaStream_t st) {
    if (D1 > 256) return launch_walk_plain_1<NS_RLE>(D2, V1, V2, m1, m2, own, pos, err, st);
    if (D1 == 32) return launch_walk_plain_1<0>(D2, V1, V2, m1, m2, own, pos, err, st);
    if (D1 == 64) return launch_walk_plain_1<1>(D2, V1, V2, m1, m2, own, pos, err, st);
    if (D1 == 128) return launch_walk_plain_1<2>(D2, V1, V2, m1, m2, own, pos, err, st);
    return launch_walk_plain_1<4>(D2, V1, V2, m1, m2, own, pos, err, st);
}

// Segment w of the plan: string s with segoff[s] <= w < segoff[s+1], r = w -
// segoff[s] segments below the string's sentinel: top hi = end - r*L, the next
// segment down (or -1 at the string start), and (r, w) as the sort key/value of
// the processing order.
// With anchors (T2 given), the top of segment r >= 1 moves within a window of
// +-L/4 around end - r*L to the position whose following 16 symbols hash
// lowest: the homologous segments of the batch's haplotypes (processed side by
// side) then start at the same locus, so their lanes step through homologous
// suffixes together and their rank reads and pos writes share blocks.  The
// windows of consecutive tops are disjoint, so segments stay in [L/2, 3L/2].
__device__ __forceinline__ uint64_t anchor_hash(uint32_t v) {
    uint64_t x = (uint64_t)v * 0x9E3779B97F4A7C15ull;
    x ^= x >> 29;
    x *= 0xBF58476D1CE4E5B9ull;
    return x ^ (x >> 32);
}

__device__ int64_t anchor_top(const uint8_t *__restrict__ T2, int64_t n2, int64_t start, int64_t q, int64_t L) {
    constexpr int K = 16;
#ifndef RB3_ANCHOR_W
#define RB3_ANCHOR_W 25  // window half-width, percent of L (below 50: windows stay disjoint)
#endif
    const int64_t W = L * RB3_ANCHOR_W / 100;
    const int64_t a = q - W > start + 1 ? q - W : start + 1, b = q + W;
    if (b + K > n2) return q;  // too close to the text's end to hash: the nominal top
    uint32_t v = 0;
    for (int64_t t = a; t < a + K - 1; ++t) v = (v << 2) | (((uint32_t)T2[t] - 1u) & 3u);
    uint64_t best = ~0ull;
    int64_t top = q;
    for (int64_t t = a; t <= b; ++t) {  // v = the 16 symbols from t
        v = (v << 2) | (((uint32_t)T2[t + K - 1] - 1u) & 3u);
        const uint64_t h = anchor_hash(v);
        if (h < best) {
            best = h;
            top = t;
        }
    }
    return top;
}

__global__ void k_seg_fill(const int64_t *__restrict__ str_end, const int64_t *__restrict__ str_start,
                           const int32_t *__restrict__ segoff, int64_t ns,
                           int64_t L, int64_t nw, const uint8_t *__restrict__ T2, int64_t n2,
                           int64_t *__restrict__ w_hi, int64_t *__restrict__ w_send,
                           int64_t *__restrict__ w_sstart, int32_t *__restrict__ w_next, uint32_t *__restrict__ key,
                           uint32_t *__restrict__ val) {
    const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w >= nw) return;
    int64_t lo = 0, hi = ns;  // largest s with segoff[s] <= w
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (segoff[mid] <= w) lo = mid;
        else hi = mid;
    }
    const int64_t s = lo, r = w - segoff[s], R = segoff[s + 1] - segoff[s];
    const int64_t end = str_end[s], start = str_start[s];
    w_hi[w] = (T2 && r > 0) ? anchor_top(T2, n2, start, end - r * L, L) : end - r * L;
    w_send[w] = end;
    w_sstart[w] = start;
    w_next[w] = r == R - 1 ? -1 : (int32_t)(w + 1);
    key[w] = (uint32_t)r;
    val[w] = (uint32_t)w;
}

__global__ void k_iota(int64_t *__restrict__ pos, int64_t n) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n) pos[k] = k;
}

// pos[k] = merged row of every B2 row k (the walk of Algorithm 1), into a
// caller-provided array of src->n entries; dst and src are not modified.
//
// merge_form 0 (default) and 2: bounded seeds and candidate tops (k_walk_seeded,
// the resolve pass, k_rewalk), segment tops at content anchors (0) or every L
// symbols (2); 3: anchored tops with uncapped seeds and the takeover chain
// (k_merge_walk); 1: plain Algorithm 1.  A consistency failure of the resolve
// pass is reported through *err_dev (bit 0: a segment's true value fell outside
// the next segment's candidates; bit 1: a candidate past B1's end) when given,
// else checked here before returning.
//
// owner (host, optional): owner[i] = the part that walks input string i of src
// (both of its strands); only the rows of strings with owner == part are
// written, every other entry of pos is set to 0, so that the parts' pos
// arrays add up to the whole.  With an empty dst, the part that owns string 0
// writes every row.
int merge_positions(const rb3_index *dst, const rb3_index *src, const rb3_opts &o, cudaStream_t st, int64_t *pos,
                    unsigned int *err_dev, const int32_t *owner, int32_t part) {
    RB3_CHECK_ARG(!src->rle, "the batch merged in must be a plain index");
    const int64_t n1 = dst->n, n2 = src->n;
    if (n2 == 0) return RB3_OK;
    OccView V1 = occ_view(dst), V2 = occ_view(src);
    const int64_t m1 = dst->m, m2 = src->m;
    // DS string s (the strings of src's text, in order) is input string s / 2, or s
    // with a single strand
    const int per = src->single_strand ? 1 : 2;
    auto owned = [&](int64_t s) { return owner == nullptr || owner[s / per] == part; };
    if (owner) RB3_CUDA_TRY(cudaMemsetAsync(pos, 0, sizeof(int64_t) * n2, st));
    {
        Phase ph("merge.walk", st);
        const bool chain = o.merge_form == 3;
        bool segmented = (o.merge_form == 0 || o.merge_form == 2 || chain) && src->text && src->isa;
        if (n1 == 0) {
            // empty B1: every l is 0 (there are no older suffixes), pos[k] = k
            if (owned(0)) RB3_LAUNCH(k_iota, nb_for(n2, 256), 256, 0, st, pos, n2);
        } else if (!segmented) {
            DevBuf err, own;
            RB3_TRY(err.alloc(sizeof(unsigned int), st));
            RB3_CUDA_TRY(cudaMemsetAsync(err.p, 0, sizeof(unsigned int), st));
            std::vector<uint8_t> own_h;
            if (owner) {
                own_h.resize(m2);
                for (int64_t s = 0; s < m2; ++s) own_h[s] = owned(s) ? 1 : 0;
                RB3_TRY(own.alloc(m2, st));
                RB3_CUDA_TRY(cudaMemcpyAsync(own.p, own_h.data(), m2, cudaMemcpyHostToDevice, st));
            }
            {
                // per new symbol: two ranks (B2 row, B1 l) and an 8 B pos
                Phase pk("k.walk_plain", st, (double)n2 * (rank_bytes(src->D) + rank_bytes(dst->D) + 8.0));
                RB3_TRY(launch_walk_plain(dst->D, src->D, V1, V2, m1, m2, owner ? own.as<uint8_t>() : nullptr, pos,
                                          err.as<unsigned int>(), st));
            }
            unsigned int herr = 0;
            RB3_CUDA_TRY(cudaMemcpyAsync(&herr, err.p, sizeof(herr), cudaMemcpyDeviceToHost, st));
            RB3_CUDA_TRY(cudaStreamSynchronize(st));
            if (herr) {
                set_error("merge: a walk over the batch BWT did not reach a sentinel (corrupt batch index)");
                return RB3_E_INVAL;
            }
        } else {
            // segment plan (host): strings of src from its sentinel positions
            int64_t L = o.seg_len;
            if (L <= 0) L = tuned_seg_len(dst, src);  // the autotuner's choice for this shape, if any
            if (L <= 0) {
                // about 512 segments per SM, length clamped to [512, 16384]
                int64_t target = (int64_t)num_sms() * 512;
                L = n2 / (target > 0 ? target : 1);
                if (L < 512) L = 512;
                if (L > 16384) L = 16384;
            }
            // chain form, double strand: seeds are self-limiting (claimed from above), so
            // no cap unless asked; single strand: the backward seed looks cap symbols
            // ahead.  Bounded form: 2L extensions (4L symbols ahead, single strand).
            int64_t cap = o.seed_cap > 0 ? o.seed_cap : (chain ? 0 : tuned_seed_cap(dst, src));
            if (cap <= 0) cap = dst->single_strand ? 4 * L : (chain ? (int64_t)1 << 62 : 2 * L);
            // the strings walked here (all, or the part's), and segments per string
            // (host, one number per string); the segments themselves and their
            // order are laid out on the device
            std::vector<int64_t> s_end, s_start;
            for (int64_t s = 0; s < (int64_t)src->str_end.size(); ++s)
                if (owned(s)) {
                    s_end.push_back(src->str_end[s]);
                    s_start.push_back(s == 0 ? 0 : src->str_end[s - 1] + 1);
                }
            const int64_t ns = (int64_t)s_end.size();
            if (ns == 0) return RB3_OK;  // nothing of this part's
            std::vector<int32_t> segoff(ns + 1, 0);
            int64_t nw = 0, maxr = 0;
            for (int64_t s = 0; s < ns; ++s) {
                const int64_t start = s_start[s];
                const int64_t len = s_end[s] - start;
                const int64_t R = len > L ? (len + L - 1) / L : 1;
                if (R - 1 > maxr) maxr = R - 1;
                nw += R;
                if (nw >= (int64_t(1) << 31)) {
                    set_error("merge: too many segments");
                    return RB3_E_INVAL;
                }
                segoff[s + 1] = (int32_t)nw;
            }
            DevBuf plan, sk0, sk1, sv1, ends, cand;
            size_t bytes = sizeof(int64_t) * (3 * nw) + sizeof(int32_t) * (3 * nw) + sizeof(unsigned long long) + 64;
            RB3_TRY(plan.alloc(bytes, st));
            RB3_TRY(sk0.alloc(sizeof(uint32_t) * nw, st));
            RB3_TRY(sk1.alloc(sizeof(uint32_t) * nw, st));
            RB3_TRY(sv1.alloc(sizeof(uint32_t) * nw, st));
            RB3_TRY(ends.alloc(sizeof(int64_t) * 2 * ns + sizeof(int32_t) * (ns + 1), st));
            int64_t *d_hi = plan.as<int64_t>(), *d_send = d_hi + nw, *d_sstart = d_send + nw;
            int32_t *d_next = reinterpret_cast<int32_t *>(d_sstart + nw), *d_state = d_next + nw, *d_order = d_state + nw;
            unsigned long long *d_ctr = reinterpret_cast<unsigned long long *>(
                (reinterpret_cast<uintptr_t>(d_order + nw) + 15) & ~uintptr_t(15));
            int64_t *d_end = ends.as<int64_t>(), *d_start = d_end + ns;
            int32_t *d_segoff = reinterpret_cast<int32_t *>(d_start + ns);
            RB3_CUDA_TRY(cudaMemcpyAsync(d_end, s_end.data(), sizeof(int64_t) * ns, cudaMemcpyHostToDevice, st));
            RB3_CUDA_TRY(cudaMemcpyAsync(d_start, s_start.data(), sizeof(int64_t) * ns, cudaMemcpyHostToDevice, st));
            RB3_CUDA_TRY(cudaMemcpyAsync(d_segoff, segoff.data(), sizeof(int32_t) * (ns + 1), cudaMemcpyHostToDevice, st));
            // order: by rank from the string end, then string (a stable sort by rank of
            // the segments in string order), so homologous segments of the batch's
            // strings run side by side
            uint32_t *ord_v0 = reinterpret_cast<uint32_t *>(d_order);
            RB3_LAUNCH(k_seg_fill, nb_for(nw, 256), 256, 0, st, d_end, d_start, d_segoff, ns, L, nw,
                       (o.merge_form == 0 || chain) ? src->text : (const uint8_t *)nullptr, src->n, d_hi, d_send,
                       d_sstart,
                       d_next, sk0.as<uint32_t>(), ord_v0);
            if (maxr > 0) {
                bool alt = false;
                RB3_TRY(radix_sort_pairs32(sk0.as<uint32_t>(), ord_v0, sk1.as<uint32_t>(), sv1.as<uint32_t>(), nw, 0,
                                           ilog2(maxr) + 1, st, &alt));
                if (alt)
                    RB3_CUDA_TRY(cudaMemcpyAsync(ord_v0, sv1.p, sizeof(uint32_t) * nw, cudaMemcpyDeviceToDevice, st));
            }
            RB3_CUDA_TRY(cudaMemsetAsync(d_ctr, 0, sizeof(unsigned long long), st));
            // the persistent walks: cps x 256 threads per SM (default 8, of which
            // registers let half be resident at once), in one-warp CTAs
            const int cps = o.walk_ctas_per_sm > 0 ? (o.walk_ctas_per_sm < 8 ? o.walk_ctas_per_sm : 8) : 8;
            const int64_t resident = (int64_t)num_sms() * 256 * cps;
            const int64_t threads = nw < resident ? nw : resident;
            const unsigned grid = nb_for(threads, WALK_THREADS);
            if (chain) {
                RB3_CUDA_TRY(cudaMemsetAsync(d_state, 0, sizeof(int32_t) * nw, st));
                // per new symbol: 1 B text, 4 B ISA, one rank, 8 B pos (seed steps not counted)
                Phase pw("k.merge_walk", st, (double)n2 * (13.0 + rank_bytes(dst->D)));
                if (dst->single_strand)
                    RB3_WITH_NS(dst->D, RB3_LAUNCH((k_merge_walk<NS, false>), grid, WALK_THREADS, 0, st, V1, m1,
                                                         src->text, src->isa, d_hi, d_send, d_sstart, d_next, d_state,
                                                         d_order, nw, cap, d_ctr, pos));
                else
                    RB3_WITH_NS(dst->D, RB3_LAUNCH((k_merge_walk<NS, true>), grid, WALK_THREADS, 0, st, V1, m1,
                                                         src->text, src->isa, d_hi, d_send, d_sstart, d_next, d_state,
                                                         d_order, nw, cap, d_ctr, pos));
            } else {
                // per segment: first candidate, candidate count, values and mask at the lower
                // end, lowest unwritten position, exact top value; a flag word and a counter
                // checkpoints of the candidate walks every REWALK_CK positions: a
                // segment holds at most L + 2 (anchor window) + 1 positions
                const int ck_per_seg = (int)((L + 2 * (L * RB3_ANCHOR_W / 100) + 2) / REWALK_CK + 1);
                RB3_TRY(cand.alloc(sizeof(int64_t) * (5 + 2 * (size_t)ck_per_seg) * nw + sizeof(int32_t) * nw + 64, st));
                int64_t *c_lo = cand.as<int64_t>(), *c_bv = c_lo + nw, *c_unw = c_bv + nw, *c_top = c_unw + nw;
                uint64_t *c_bm = reinterpret_cast<uint64_t *>(c_top + nw);
                int64_t *c_ckv = reinterpret_cast<int64_t *>(c_bm + nw);
                uint64_t *c_ckm = reinterpret_cast<uint64_t *>(c_ckv + (size_t)ck_per_seg * nw);
                int32_t *c_n = reinterpret_cast<int32_t *>(c_ckm + (size_t)ck_per_seg * nw);
                unsigned long long *c_ctr = reinterpret_cast<unsigned long long *>(
                    (reinterpret_cast<uintptr_t>(c_n + nw) + 15) & ~uintptr_t(15));
                unsigned int *c_err = reinterpret_cast<unsigned int *>(c_ctr + 1);
                RB3_CUDA_TRY(cudaMemsetAsync(c_ctr, 0, sizeof(unsigned long long) + sizeof(unsigned int), st));
                unsigned int *errp = err_dev ? err_dev : c_err;
                {
                    // per new symbol: 1 B text, 4 B ISA, one rank, 8 B pos (seed steps and the
                    // second walk of unconverged positions not counted)
                    Phase pw("k.merge_walk", st, (double)n2 * (13.0 + rank_bytes(dst->D)));
                    if (dst->single_strand)
                        RB3_WITH_NS(dst->D,
                                          RB3_LAUNCH((k_walk_seeded<NS, false>), grid, WALK_THREADS, 0, st, V1, m1,
                                                     src->text, src->isa, d_hi, d_send, d_sstart, d_next, d_order, nw,
                                                     cap, d_ctr, pos, c_lo, c_n, c_bv, c_bm, c_unw, c_ckv, c_ckm,
                                                     ck_per_seg, errp));
                    else
                        RB3_WITH_NS(dst->D,
                                          RB3_LAUNCH((k_walk_seeded<NS, true>), grid, WALK_THREADS, 0, st, V1, m1,
                                                     src->text, src->isa, d_hi, d_send, d_sstart, d_next, d_order, nw,
                                                     cap, d_ctr, pos, c_lo, c_n, c_bv, c_bm, c_unw, c_ckv, c_ckm,
                                                     ck_per_seg, errp));
                }
                {
                    // chunks of up to 32 segments of one string (host: from the
                    // segments per string), the string's chunks, each segment's chunk
                    std::vector<int32_t> h_w0, h_cnt, h_choff(ns + 1, 0), h_segch(nw);
                    std::vector<uint8_t> h_last(nw, 0);
                    for (int64_t s2 = 0; s2 < ns; ++s2) {
                        for (int64_t w = segoff[s2]; w < segoff[s2 + 1]; w += 32) {
                            const int64_t c = segoff[s2 + 1] - w < 32 ? segoff[s2 + 1] - w : 32;
                            for (int64_t i = 0; i < c; ++i) h_segch[w + i] = (int32_t)h_w0.size();
                            h_w0.push_back((int32_t)w);
                            h_cnt.push_back((int32_t)c);
                        }
                        h_choff[s2 + 1] = (int32_t)h_w0.size();
                        h_last[segoff[s2 + 1] - 1] = 1;
                    }
                    const int64_t nch = (int64_t)h_w0.size();
                    DevBuf rs;
                    RB3_TRY(rs.alloc(sizeof(int32_t) * (4 * nch + ns + 1 + 2 * nw) + sizeof(uint64_t) * (nw + nch) +
                                         nw + 64,
                                     st));
                    uint64_t *r_prem = rs.as<uint64_t>(), *r_aggm = r_prem + nw;
                    int32_t *r_prec = reinterpret_cast<int32_t *>(r_aggm + nch), *r_aggc = r_prec + nw,
                            *r_entry = r_aggc + nch, *r_w0 = r_entry + nch, *r_cnt = r_w0 + nch, *r_choff = r_cnt + nch,
                            *r_segch = r_choff + ns + 1;
                    uint8_t *r_last = reinterpret_cast<uint8_t *>(r_segch + nw);
                    RB3_CUDA_TRY(cudaMemcpyAsync(r_w0, h_w0.data(), sizeof(int32_t) * nch, cudaMemcpyHostToDevice, st));
                    RB3_CUDA_TRY(cudaMemcpyAsync(r_cnt, h_cnt.data(), sizeof(int32_t) * nch, cudaMemcpyHostToDevice, st));
                    RB3_CUDA_TRY(
                        cudaMemcpyAsync(r_choff, h_choff.data(), sizeof(int32_t) * (ns + 1), cudaMemcpyHostToDevice, st));
                    RB3_CUDA_TRY(cudaMemcpyAsync(r_segch, h_segch.data(), sizeof(int32_t) * nw, cudaMemcpyHostToDevice, st));
                    RB3_CUDA_TRY(cudaMemcpyAsync(r_last, h_last.data(), nw, cudaMemcpyHostToDevice, st));
                    Phase pr("k.seg_resolve", st);
                    RB3_LAUNCH(k_res_chunk, nb_for(nch * 32, 128), 128, 0, st, r_w0, r_cnt, nch, c_lo, c_n, c_bv, c_bm,
                               r_last, r_prec, r_prem, r_aggc, r_aggm);
                    RB3_LAUNCH(k_res_carry, nb_for(ns * 32, 128), 128, 0, st, r_choff, ns, r_aggc, r_aggm, r_entry);
                    RB3_LAUNCH(k_res_apply, nb_for(nw, 256), 256, 0, st, r_segch, r_w0, nw, r_entry, r_prec, r_prem,
                               c_lo, c_n, c_bv, c_bm, r_last, c_top, errp);
                }
                {
                    Phase pr("k.rewalk", st);
                    RB3_WITH_NS(dst->D, RB3_LAUNCH((k_rewalk<NS>), grid, WALK_THREADS, 0, st, V1, src->text,
                                                         src->isa, d_hi, c_unw, c_top, c_lo, c_ckv, c_ckm, ck_per_seg,
                                                         d_order, nw, c_ctr, pos, errp));
                }
                if (!err_dev) {
                    unsigned int herr = 0;
                    RB3_CUDA_TRY(cudaMemcpyAsync(&herr, c_err, sizeof(herr), cudaMemcpyDeviceToHost, st));
                    RB3_CUDA_TRY(cudaStreamSynchronize(st));
                    if (herr) {
                        set_error("merge: segment seeds and walks disagree (flags %u)", herr);
                        return RB3_E_CUDA;
                    }
                }
            }
        }
    }
    return RB3_OK;
}

static int merge_check(const rb3_index *dst, const rb3_index *src) {
    RB3_CHECK_ARG(dst != src, "dst and src must differ");
    RB3_CHECK_ARG(!src->rle, "the batch merged in must be a plain index");
    RB3_CHECK_ARG(dst->single_strand == src->single_strand || dst->n == 0,
                  "cannot merge a single-strand index with a double-strand one");
    if ((dst->n + src->n) >= (int64_t(1) << 40)) {
        set_error("merged index would exceed 2^40 symbols");
        return RB3_E_INVAL;
    }
    return RB3_OK;
}

int merge_impl(rb3_index *dst, const rb3_index *src, const rb3_opts &o, cudaStream_t st) {
    RB3_TRY(merge_check(dst, src));
    if (src->n == 0) return RB3_OK;
    DevBuf posb, errb;
    RB3_TRY(posb.alloc(sizeof(int64_t) * src->n, st));
    RB3_TRY(errb.alloc(sizeof(unsigned int), st));
    RB3_CUDA_TRY(cudaMemsetAsync(errb.p, 0, sizeof(unsigned int), st));
    RB3_TRY(merge_positions(dst, src, o, st, posb.as<int64_t>(), errb.as<unsigned int>()));
    return merge_apply(dst, src, posb.as<int64_t>(), errb.as<unsigned int>(), st);
}

// pos[k] < pos[k+1], 0 <= pos[0], pos[n2-1] < n1 + n2: the rows of a stable
// interleave of B1 and B2 (bit 2 of *bad otherwise).
__global__ void k_check_pos(const int64_t *__restrict__ pos, int64_t n2, int64_t nM, unsigned int *__restrict__ bad) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n2) return;
    const int64_t p = pos[k];
    if (p < 0 || p >= nM || (k + 1 < n2 && pos[k + 1] <= p)) atomicOr(bad, 4u);
}

// A run-length dst: the merged spans are written from its runs and src's
// symbols (rle_merge_arrays), with the sampled suffix array merged as for a
// plain one; dst is replaced only when everything succeeded.
static int merge_apply_rle(rb3_index *dst, const rb3_index *src, const int64_t *pos, const unsigned int *errb,
                           int64_t *kst, int64_t ntiles, cudaStream_t st) {
    const int64_t n1 = dst->n, n2 = src->n, nM = n1 + n2;
    struct Owned {
        rb3_index *p = new rb3_index();
        ~Owned() {
            if (p) rb3_index_free(p);
        }
    } R;
    RB3_TRY(rle_merge_arrays(dst, src, pos, st, R.p));
    const bool keep_samples = src->sa_s > 0 && src->sdir && (n1 == 0 || (dst->sa_s == src->sa_s && dst->sdir));
    if (keep_samples) {
        Phase ph("merge.sample", st);
        RB3_LAUNCH(k_tile_starts, nb_for(n2 + 1, 256), 256, 0, st, pos, n2, ntiles, kst);
        if (n1 == 0) {
            const int64_t nw = n2 / 64 + 1;
            RB3_TRY(dev_alloc((void **)&R.p->sdir, sizeof(uint64_t) * 2 * nw, st));
            RB3_TRY(dev_alloc((void **)&R.p->svals, sizeof(uint64_t) * (src->n_samples > 0 ? src->n_samples : 1), st));
            RB3_CUDA_TRY(cudaMemcpyAsync(R.p->sdir, src->sdir, sizeof(uint64_t) * 2 * nw, cudaMemcpyDeviceToDevice, st));
            if (src->n_samples > 0)
                RB3_CUDA_TRY(cudaMemcpyAsync(R.p->svals, src->svals, sizeof(uint64_t) * src->n_samples,
                                             cudaMemcpyDeviceToDevice, st));
            R.p->n_samples = src->n_samples;
        } else {
            RB3_TRY(sample_merge(dst, src, pos, kst, ntiles, nM, MT, R.p, st));
        }
        R.p->sa_s = src->sa_s;
    }
    unsigned int herr = 0;
    RB3_CUDA_TRY(cudaMemcpyAsync(&herr, errb, sizeof(herr), cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr) {
        set_error("merge: segment seeds and walks disagree (flags %u); dst unchanged", herr);
        return RB3_E_CUDA;
    }
    int64_t Cw[SIGMA + 1];
    for (int a = 0; a <= SIGMA; ++a) Cw[a] = R.p->C[a];
    RB3_TRY(finalize_counts(R.p, st));
    for (int a = 0; a <= SIGMA; ++a)
        if (R.p->C[a] != Cw[a]) {
            set_error("merge: merged counts differ from the inputs' (symbol %d)", a);
            return RB3_E_CUDA;
        }
    std::swap(*dst, *R.p);  // dst's old arrays leave with R
    return RB3_OK;
}

int merge_apply(rb3_index *dst, const rb3_index *src, const int64_t *pos, const unsigned int *walk_err,
                cudaStream_t st) {
    RB3_TRY(merge_check(dst, src));
    if (src->n == 0) return RB3_OK;
    const int64_t n1 = dst->n, n2 = src->n, nM = n1 + n2;
    // output layout: D of dst (or of src when a plain dst is empty)
    int D = n1 || dst->rle ? dst->D : src->D;
    int log2D = ilog2(D), bb = block_bytes_for(D);
    int64_t nbM = nM / D + 1;
    int64_t ntiles = (nbM * D + MT - 1) / MT;
    DevBuf kst, Mb, tbase, errb;
    RB3_TRY(errb.alloc(sizeof(unsigned int), st));
    if (walk_err)
        RB3_CUDA_TRY(cudaMemcpyAsync(errb.p, walk_err, sizeof(unsigned int), cudaMemcpyDeviceToDevice, st));
    else
        RB3_CUDA_TRY(cudaMemsetAsync(errb.p, 0, sizeof(unsigned int), st));
    RB3_TRY(kst.alloc(sizeof(int64_t) * (ntiles + 2), st));
    OccView V1 = occ_view(dst), V2 = occ_view(src);
    const int64_t m1 = dst->m, m2 = src->m;
    if (!walk_err) {
        // positions from the caller: a valid interleave, or nothing is written
        RB3_LAUNCH(k_check_pos, nb_for(n2, 256), 256, 0, st, pos, n2, nM, errb.as<unsigned int>());
        unsigned int herr = 0;
        RB3_CUDA_TRY(cudaMemcpyAsync(&herr, errb.p, sizeof(herr), cudaMemcpyDeviceToHost, st));
        RB3_CUDA_TRY(cudaStreamSynchronize(st));
        if (herr) {
            set_error("merge: pos is not an increasing list of rows of the merged index");
            return RB3_E_INVAL;
        }
    }
    if (dst->rle) return merge_apply_rle(dst, src, pos, errb.as<unsigned int>(), kst.as<int64_t>(), ntiles, st);
    RB3_TRY(tbase.alloc(sizeof(int64_t) * SIGMA * (ntiles + 1), st));
    RB3_TRY(Mb.alloc((size_t)nbM * bb, st));
    {
        Phase ph("merge.scatter", st);
        RB3_LAUNCH(k_tile_starts, nb_for(n2 + 1, 256), 256, 0, st, pos, n2, ntiles, kst.as<int64_t>());
        {
            // every input block read once, every output block written once, 8 B pos per new symbol
            double bytes = (double)dst->nblocks * dst->block_bytes + (double)src->nblocks * src->block_bytes +
                           (double)nbM * bb + 8.0 * n2;
            RB3_LAUNCH(k_tile_bases, nb_for(ntiles, 128), 128, 0, st, V1, V2, kst.as<int64_t>(), ntiles,
                       tbase.as<int64_t>());
            Phase pk("k.scatter", st, bytes);
            RB3_LAUNCH(k_scatter, (unsigned)ntiles, MT_THREADS, 0, st, V1, V2, pos, kst.as<int64_t>(),
                       tbase.as<int64_t>(), nM, nbM, log2D, bb, Mb.as<uint8_t>());
        }
    }
    // sampled suffix array: kept when both inputs have one at the same rate
    rb3_index smp;
    const bool keep_samples = src->sa_s > 0 && src->sdir && (n1 == 0 || (dst->sa_s == src->sa_s && dst->sdir));
    if (keep_samples) {
        Phase ph("merge.sample", st);
        if (n1 == 0) {  // the result is src: a copy of its sample
            const int64_t nw = n2 / 64 + 1;
            RB3_TRY(dev_alloc((void **)&smp.sdir, sizeof(uint64_t) * 2 * nw, st));
            RB3_TRY(dev_alloc((void **)&smp.svals, sizeof(uint64_t) * (src->n_samples > 0 ? src->n_samples : 1), st));
            RB3_CUDA_TRY(cudaMemcpyAsync(smp.sdir, src->sdir, sizeof(uint64_t) * 2 * nw, cudaMemcpyDeviceToDevice, st));
            if (src->n_samples > 0)
                RB3_CUDA_TRY(cudaMemcpyAsync(smp.svals, src->svals, sizeof(uint64_t) * src->n_samples,
                                             cudaMemcpyDeviceToDevice, st));
            smp.n_samples = src->n_samples;
        } else {
            RB3_TRY(sample_merge(dst, src, pos, kst.as<int64_t>(), ntiles, nM, MT, &smp, st));
        }
    }
    // D = 32 past 2^32 symbols: the span bases are the ranks at the tiles where spans start
    int64_t *gb = nullptr;
    if (D == 32 && nM >> GSPAN_LOG2) {
        const int64_t rows = gbase_rows(nM);
        RB3_TRY(dev_alloc((void **)&gb, sizeof(int64_t) * 5 * rows, st));
        RB3_LAUNCH(k_span_bases, nb_for(rows * 5, 128), 128, 0, st, tbase.as<int64_t>(), rows, gb);
    }
    // the walk's own consistency check (segment seeds against the walks from above),
    // before dst is touched
    {
        unsigned int herr = 0;
        RB3_CUDA_TRY(cudaMemcpyAsync(&herr, errb.p, sizeof(herr), cudaMemcpyDeviceToHost, st));
        RB3_CUDA_TRY(cudaStreamSynchronize(st));
        if (herr) {
            if (gb) dev_free(gb, st);
            if (smp.sdir) dev_free(smp.sdir, st);
            if (smp.svals) dev_free(smp.svals, st);
            smp.sdir = nullptr;
            smp.svals = nullptr;
            set_error("merge: segment seeds and walks disagree (flags %u); dst unchanged", herr);
            return RB3_E_CUDA;
        }
    }
    // install
    free_samples(dst);
    dst->sa_s = keep_samples ? src->sa_s : 0;
    dst->sdir = smp.sdir;
    dst->svals = smp.svals;
    dst->n_samples = smp.n_samples;
    smp.sdir = nullptr;
    smp.svals = nullptr;
    if (dst->gbase) dev_free(dst->gbase, st);
    dst->gbase = gb;
    if (dst->blocks) dev_free(dst->blocks, st);
    if (dst->text) dev_free(dst->text, st);
    if (dst->isa) dev_free(dst->isa, st);
    dst->text = nullptr;
    dst->isa = nullptr;
    dst->str_end.clear();
    dst->blocks = static_cast<uint8_t *>(Mb.detach());
    dst->n = nM;
    dst->m = m1 + m2;
    for (int a = 0; a <= SIGMA; ++a) dst->C[a] = dst->C[a] + src->C[a];
    // the merged blocks must hold exactly the symbols of both inputs (read back from the device)
    int64_t Cw[SIGMA + 1];
    for (int a = 0; a <= SIGMA; ++a) Cw[a] = dst->C[a];
    dst->D = D;
    dst->log2D = log2D;
    dst->block_bytes = bb;
    dst->nblocks = nbM;
    dst->single_strand = src->single_strand;
    RB3_TRY(finalize_counts(dst, st));
    for (int a = 0; a <= SIGMA; ++a)
        if (dst->C[a] != Cw[a]) {
            set_error("merge: merged counts differ from the inputs' (symbol %d)", a);
            return RB3_E_CUDA;
        }
    return RB3_OK;
}

}  // namespace rb3
