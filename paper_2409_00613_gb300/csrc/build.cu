// Batch BWT builder: S0 encode (both strands), S1 prefix-doubling suffix sort,
// S2 BWT extraction, 4-bit packing and Occ checkpoints.
//
// What is computed (Section "Basic concepts", Table 1; Section "BWT
// construction" for the sentinel order; Section "Double-strand BWT" for the
// text): T = P0 $ rc(P0) $ P1 $ ..., S its suffix array under
// $_0 < ... < $_{m-1} < A < C < G < T < N, B[i] = T[S(i)-1] with T[-1] = T[n-1].
// The paper runs libsais on the integer alphabet; here the suffix array comes
// from prefix doubling with radix passes (how), which reaches the same S.
//
// Prefix doubling, Larsson-Sadakane style:
//   round 0   key(p) = T[p..p+18) as an 18-digit base-6 number (47 bits),
//             cut after the first sentinel.  A window holding a sentinel makes its suffix's
//             order final (sentinels are distinct and ordered by position, and
//             the stable sort by key keeps position order among equal keys).
//             A window holds a sentinel iff its last digit is 0.
//             Stable radix sort of (key, p); ranks = group start positions.
//   round h   for every suffix still in a group of >= 2, key = rank[p + h];
//             sort inside the group; split; new rank = start of the sub-group.
//             Groups are processed in the order of their first member's text
//             position (locality of the rank reads and writes).
// Rank writes of a round are applied only after every key of that round has
// been read, so all keys of a round see the same (h-level) ranks.
#include "common.cuh"

namespace rb3 {

constexpr int H0 = 18;            // symbols in the round-0 key (base-6 digits; 6^18 < 2^47)
constexpr int H0_BITS = 47;
// Batches without N: H4 symbols as 2-bit digits (A..T = 0..3) and a field
// counting them.  By default 14 symbols and a 4-bit count, 32 bits: four radix
// passes over (uint32 key, uint32 value) pairs, 8 bytes each, instead of six
// over 12-byte pairs for the base-6 key (RB3_KEY4_32 = 0: 17 symbols and a
// 5-bit count in a uint64 key, five passes).
#ifndef RB3_KEY4_32
#define RB3_KEY4_32 1
#endif
#if RB3_KEY4_32
constexpr int H4 = 14;
constexpr int K4_CNT_BITS = 4;
using Key4 = uint32_t;
#else
constexpr int H4 = 17;
constexpr int K4_CNT_BITS = 5;
using Key4 = uint64_t;
#endif
constexpr int H4_BITS = 2 * H4 + K4_CNT_BITS;
constexpr int SMALL_MAX = 1024;   // groups up to this size are sorted in shared memory
constexpr int RT_TILE = 2048;     // round-kernel tile (entries)
constexpr int RT_THREADS = 256;
constexpr int RT_MAXR = RT_TILE + SMALL_MAX;
constexpr uint32_t SURV = 0x80000000u;

// ---- S0: encode ------------------------------------------------------------
__global__ void k_encode(const uint8_t *__restrict__ seq, const int64_t *__restrict__ in_off,
                         const int64_t *__restrict__ out_off, int64_t n_seq, int64_t total_in, int both,
                         uint8_t *__restrict__ T, int *__restrict__ bad) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total_in;
         g += (int64_t)gridDim.x * blockDim.x) {
        // string s with in_off[s] <= g < in_off[s+1]
        int64_t lo = 0, hi = n_seq;  // count of in_off[1..] <= g
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (in_off[mid + 1] <= g) lo = mid + 1;
            else hi = mid;
        }
        int64_t s = lo;
        int64_t o = g - in_off[s], L = in_off[s + 1] - in_off[s];
        int x = seq[g];
        if (x < 1 || x > 5) {
            atomicOr(bad, 1);
            x = 5;
        }
        // bit 1: the batch holds N (one atomic per warp that sees one)
        const unsigned nm = __ballot_sync(__activemask(), x == 5);
        if (nm && (threadIdx.x & 31) == __ffs(nm) - 1) atomicOr(bad, 2);
        int64_t base = out_off[s];
        T[base + o] = (uint8_t)x;
        if (both) T[base + L + 1 + (L - 1 - o)] = (uint8_t)comp_sym(x);
    }
}

__global__ void k_sentinels(const int64_t *__restrict__ in_off, const int64_t *__restrict__ out_off, int64_t n_seq,
                            int both, uint8_t *__restrict__ T) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n_seq) return;
    int64_t L = in_off[s + 1] - in_off[s], base = out_off[s];
    T[base + L] = 0;
    if (both) T[base + 2 * L + 1] = 0;
}

// ---- S1: round 0 ------------------------------------------------------------
__global__ void k_init_keys(const uint8_t *__restrict__ T, int64_t n, uint64_t *__restrict__ key,
                            uint32_t *__restrict__ val) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    uint64_t k = 0;
    bool stop = false;
#pragma unroll
    for (int j = 0; j < H0; ++j) {
        uint32_t c = stop ? 0u : (uint32_t)T[p + j];  // T ends with a sentinel: reads stop at n-1
        stop = stop || c == 0;
        k = k * 6u + c;
    }
    key[p] = k;
    val[p] = (uint32_t)p;
}

// Round-0 key of an N-free batch.  The window's symbols up to its first
// sentinel (at most H4) as 2-bit digits, padded with zeros, then the number of
// those symbols (H4 if the window holds no sentinel).  Ordering by (digits,
// count) is the suffix order of the windows: a window U$ sorts before every
// window starting with U and a letter, and the padding ties U$ only with
// windows U A..A, which the count puts after it.  Windows with the same digits
// and count are equal (or both end at a sentinel after the same prefix: then
// the stable sort keeps them in position order, the order of their sentinels).
constexpr int K4_PER = 16;  // positions per thread of k_init_keys4

// One thread per K4_PER consecutive positions p0 + r: the window bytes
// T[p0, p0 + 32) in registers (two 16-byte loads), the digits of position r + 1
// rolled from those of r, the count from a mask of the window's sentinels.
__global__ void k_init_keys4(const uint8_t *__restrict__ T, int64_t n, Key4 *__restrict__ key,
                             uint32_t *__restrict__ val) {
    const int64_t p0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * K4_PER;
    if (p0 >= n) return;
    uint32_t w[8];
    if (p0 + 32 <= n) {  // T is 16-byte aligned and p0 a multiple of 16
        const uint4 a = __ldg(reinterpret_cast<const uint4 *>(T + p0));
        const uint4 b = __ldg(reinterpret_cast<const uint4 *>(T + p0) + 1);
        w[0] = a.x, w[1] = a.y, w[2] = a.z, w[3] = a.w, w[4] = b.x, w[5] = b.y, w[6] = b.z, w[7] = b.w;
    } else {  // past the text: zero bytes, read as sentinels (the text ends with one anyway)
#pragma unroll
        for (int k = 0; k < 8; ++k) w[k] = 0;
#pragma unroll
        for (int b = 0; b < 32; ++b)
            if (p0 + b < n) w[b >> 2] |= (uint32_t)T[p0 + b] << (8 * (b & 3));
    }
    uint32_t z = 0;  // bit b: byte b of the window is a sentinel
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t e = __vcmpeq4(w[k], 0u);
        z |= (((e >> 7) & 1u) | ((e >> 14) & 2u) | ((e >> 21) & 4u) | ((e >> 28) & 8u)) << (4 * k);
    }
    constexpr uint64_t MD = (1ull << (2 * H4)) - 1ull;
    uint64_t raw = 0;  // digits of T[p0 + r + j], j < H4, as (symbol - 1) & 3
#pragma unroll
    for (int j = 0; j < H4; ++j) raw = (raw << 2) | (((w[j >> 2] >> (8 * (j & 3))) - 1u) & 3u);
    Key4 kk[K4_PER];
#pragma unroll
    for (int r = 0; r < K4_PER; ++r) {
        const uint32_t zr = z >> r;
        const uint32_t len = zr ? min((uint32_t)H4, (uint32_t)(__ffs(zr) - 1)) : (uint32_t)H4;
        const int drop = 2 * (H4 - (int)len);  // digits at and after the first sentinel are zero
        kk[r] = (Key4)((((raw >> drop) << drop) << K4_CNT_BITS) | len);
        if (r + 1 < K4_PER) {
            const int b = r + H4;
            raw = ((raw << 2) | (((w[b >> 2] >> (8 * (b & 3))) - 1u) & 3u)) & MD;
        }
    }
    if (p0 + K4_PER <= n) {
        if constexpr (sizeof(Key4) == 8) {
            ulonglong2 *ko = reinterpret_cast<ulonglong2 *>(key + p0);
#pragma unroll
            for (int r = 0; r < K4_PER; r += 2) ko[r / 2] = make_ulonglong2(kk[r], kk[r + 1]);
        } else {
            uint4 *ko = reinterpret_cast<uint4 *>(key + p0);
#pragma unroll
            for (int r = 0; r < K4_PER; r += 4)
                ko[r / 4] = make_uint4((uint32_t)kk[r], (uint32_t)kk[r + 1], (uint32_t)kk[r + 2], (uint32_t)kk[r + 3]);
        }
        uint4 *vo = reinterpret_cast<uint4 *>(val + p0);
#pragma unroll
        for (int r = 0; r < K4_PER; r += 4)
            vo[r / 4] = make_uint4((uint32_t)(p0 + r), (uint32_t)(p0 + r + 1), (uint32_t)(p0 + r + 2),
                                   (uint32_t)(p0 + r + 3));
    } else {
#pragma unroll
        for (int r = 0; r < K4_PER; ++r)
            if (p0 + r < n) {
                key[p0 + r] = kk[r];
                val[p0 + r] = (uint32_t)(p0 + r);
            }
    }
}

// A group starts at i if its key differs from the previous one, or if its
// window holds a sentinel (then its order is final: singleton).  A base-6
// window holds a sentinel iff its last digit is 0; a 2-bit one iff its count
// field is below H4.
template <bool B4, class KT>
__global__ void k_heads(const KT *__restrict__ K, int64_t n, uint32_t *__restrict__ hv) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool sent = B4 ? (K[i] & ((1u << K4_CNT_BITS) - 1u)) < (KT)H4 : (K[i] % 6u) == 0;
    bool head = i == 0 || K[i] != K[i - 1] || sent;
    hv[i] = head ? (uint32_t)i : 0u;
}

// Round-0 groups, a tile of IG_TILE entries per block.  Singletons and the
// members of groups above SMALL_MAX get their rank now (members of smaller
// groups get theirs from k_expand_groups, in locus order); a small group's size
// is kept at its head.  The head of each group of 2..SMALL_MAX is listed as
// (its SA value, its index) and every member of a larger group as (its SA
// value, its group start), each list filled through one counter per tile:
// their order does not matter (the head list is sorted by SA value next, the
// large list by (group, key) in every round).  The groups of 2..SMALL_MAX are
// then laid out in the order of their first member's text position (the
// stable sort keeps members in position order, so that is the head's SA
// value): a pangenome's groups are mostly homologous copies of one locus, so
// neighbouring groups are neighbouring loci and the rank[p + h] reads and rank
// writes of a round touch nearby addresses.
constexpr int IG_ITEMS = 8;
constexpr int IG_THREADS = 256;
constexpr int IG_TILE = IG_THREADS * IG_ITEMS;
constexpr int IG_WARPS = IG_THREADS / 32;
static_assert(IG_ITEMS * IG_WARPS == 64, "one warp scans two counts per lane");

__global__ void __launch_bounds__(IG_THREADS) k_init_groups(const uint32_t *__restrict__ SA,
                                                            const uint32_t *__restrict__ gstart, int64_t n,
                                                            int32_t *__restrict__ rank, uint32_t *__restrict__ gsize,
                                                            uint32_t *__restrict__ cnt, uint32_t *__restrict__ hkey,
                                                            uint32_t *__restrict__ hval, uint32_t *__restrict__ lp,
                                                            uint32_t *__restrict__ lg) {
    __shared__ uint32_t wc[2][IG_ITEMS * IG_WARPS];  // per (list, pass, warp): counts, then offsets
    __shared__ uint32_t tb[2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t t0 = (int64_t)blockIdx.x * IG_TILE;
    uint32_t sv[IG_ITEMS], gv[IG_ITEMS];
    unsigned hm = 0, lm = 0;  // bit j: entry j heads a small group / is a member of a large one
#pragma unroll
    for (int j = 0; j < IG_ITEMS; ++j) {
        const int64_t i = t0 + j * IG_THREADS + threadIdx.x;
        bool hd = false, lgm = false;
        sv[j] = gv[j] = 0;
        if (i < n) {
            const uint32_t g = gstart[i], s = SA[i];
            const bool last = i + 1 == n || gstart[i + 1] != g;
            const bool single = g == (uint32_t)i && last;
            const bool large = (int64_t)g + SMALL_MAX < n && gstart[g + SMALL_MAX] == g;
            if (single || large) rank[s] = (int32_t)g;
            if (last && !single && !large) gsize[g] = (uint32_t)(i - g + 1);
            hd = g == (uint32_t)i && !single && !large;
            lgm = large;
            sv[j] = s;
            gv[j] = g;
        }
        const unsigned hb = __ballot_sync(0xFFFFFFFFu, hd), lb = __ballot_sync(0xFFFFFFFFu, lgm);
        if (lane == 0) {
            wc[0][j * IG_WARPS + w] = __popc(hb);
            wc[1][j * IG_WARPS + w] = __popc(lb);
        }
        hm |= (unsigned)hd << j;
        lm |= (unsigned)lgm << j;
    }
    __syncthreads();
    if (w < 2) {  // warp L: exclusive offsets of list L in (pass, warp) order, and the tile's place in it
        uint32_t *c = wc[w];
        const uint32_t c0 = c[2 * lane], c1 = c[2 * lane + 1];
        const uint32_t inc = warp_incl(c0 + c1, 0);
        const uint32_t ex = inc - c0 - c1;
        c[2 * lane] = ex;
        c[2 * lane + 1] = ex + c0;
        uint32_t base = 0;
        if (lane == 31 && inc) base = atomicAdd(&cnt[w], inc);
        if (lane == 31) tb[w] = base;
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < IG_ITEMS; ++j) {
        const int64_t i = t0 + j * IG_THREADS + threadIdx.x;
        const bool hd = (hm >> j) & 1u, lgm = (lm >> j) & 1u;
        const unsigned hb = __ballot_sync(0xFFFFFFFFu, hd), lb = __ballot_sync(0xFFFFFFFFu, lgm);
        if (hd) {
            const uint32_t o = tb[0] + wc[0][j * IG_WARPS + w] + __popc(hb & lt);
            hkey[o] = sv[j];
            hval[o] = (uint32_t)i;
        }
        if (lgm) {
            const uint32_t o = tb[1] + wc[1][j * IG_WARPS + w] + __popc(lb & lt);
            lp[o] = sv[j];
            lg[o] = gv[j];
        }
    }
}

// Small group j in locus order: its size, kept at its head by k_init_groups.
__global__ void k_group_sizes(const uint32_t *__restrict__ hval, int64_t G, const uint32_t *__restrict__ gsize,
                              uint32_t *__restrict__ gsz) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= G) return;
    gsz[j] = gsize[hval[j]];
}

// A warp lays out 32 consecutive groups, whose places in the list are one
// contiguous range: lanes stride over that range (coalesced list writes and
// SA reads), each finding its group among the warp's 32 by a shuffle search.
__global__ void k_expand_groups(const uint32_t *__restrict__ hval, const uint32_t *__restrict__ gsz,
                                const uint32_t *__restrict__ goff, int64_t G, const uint32_t *__restrict__ SA,
                                uint32_t *__restrict__ sp, uint32_t *__restrict__ sg, int32_t *__restrict__ rank) {
    const int lane = threadIdx.x & 31;
    const int64_t j0 = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * 32;
    if (j0 >= G) return;  // the whole warp
    const int nvalid = G - j0 < 32 ? (int)(G - j0) : 32;
    const bool ok = lane < nvalid;
    const uint32_t h = ok ? hval[j0 + lane] : 0u, o = ok ? goff[j0 + lane] : 0u, z = ok ? gsz[j0 + lane] : 0u;
    const uint32_t first = __shfl_sync(0xffffffffu, o, 0);
    const uint32_t end = __shfl_sync(0xffffffffu, o + z, nvalid - 1);
    for (uint32_t base = first; base < end; base += 32) {
        const uint32_t x = base + lane;
        int g = 0;  // the last of the warp's groups that starts at or before x
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const int mid = g + step;
            const uint32_t om = __shfl_sync(0xffffffffu, o, mid < 32 ? mid : 31);
            if (mid < nvalid && om <= x) g = mid;
        }
        const uint32_t hg = __shfl_sync(0xffffffffu, h, g), og = __shfl_sync(0xffffffffu, o, g);
        if (x < end) {
            const uint32_t p = SA[hg + (x - og)];
            sp[x] = p;
            sg[x] = hg;
            rank[p] = (int32_t)hg;
        }
    }
}

// out[0] = excl[n-1] + flag[n-1] (+ out[0] when accumulate)
__global__ void k_tally(const uint32_t *__restrict__ excl, const uint32_t *__restrict__ flag, int64_t n,
                        uint32_t *__restrict__ out, int accumulate) {
    uint32_t v = n > 0 ? excl[n - 1] + flag[n - 1] : 0u;
    out[0] = accumulate ? out[0] + v : v;
}

// ---- S1: doubling rounds, groups of <= SMALL_MAX -----------------------------
// Tiles of RT_TILE list entries, moved to group boundaries.  Keys are gathered
// into shared memory; each entry counts the keys of its group that are smaller
// (less) and equal before it (eqb): its new place is group start + less + eqb,
// its new rank group start + less.
__device__ __forceinline__ int64_t run_start_at(const uint32_t *__restrict__ wg, int64_t x, int64_t N) {
    while (x > 0 && x < N && wg[x] == wg[x - 1]) ++x;
    return x;
}

__global__ void __launch_bounds__(RT_THREADS) k_round_small(const uint32_t *__restrict__ wp,
                                                            const uint32_t *__restrict__ wg, int64_t N,
                                                            const int32_t *__restrict__ rank, uint32_t h, int64_t n,
                                                            uint32_t *__restrict__ err,
                                                            int32_t *__restrict__ SA, uint32_t *__restrict__ tp,
                                                            uint32_t *__restrict__ tg,
                                                            uint32_t *__restrict__ tile_surv,
                                                            uint32_t *__restrict__ tile_begin) {
    __shared__ uint32_t sp[RT_MAXR], sg[RT_MAXR], sk[RT_MAXR];
    __shared__ int64_t rb, re;
    __shared__ uint32_t wtot[32];
    int64_t b0 = (int64_t)blockIdx.x * RT_TILE;
    int64_t e0 = b0 + RT_TILE < N ? b0 + RT_TILE : N;
    if (threadIdx.x == 0) {
        rb = run_start_at(wg, b0, N);
        tile_begin[blockIdx.x] = (uint32_t)rb;
    }
    if (threadIdx.x == 32) re = run_start_at(wg, e0, N);
    __syncthreads();
    int64_t b = rb;
    int cnt = (int)(re - rb);
    for (int i = threadIdx.x; i < cnt; i += RT_THREADS) {
        uint32_t p = wp[b + i];
        sp[i] = p;
        sg[i] = wg[b + i];
        int64_t ph = (int64_t)p + h;
        if (ph < n) {
            sk[i] = (uint32_t)rank[ph];
        } else {  // cannot happen for a sentinel-terminated text; recorded, never read
            atomicOr(err, 1u);
            sk[i] = 0u;
        }
    }
    __syncthreads();
    uint32_t surv = 0;
    for (int i = threadIdx.x; i < cnt; i += RT_THREADS) {
        // the lanes of a warp hold consecutive entries (a prefix of the warp on
        // the last pass): a group's bounds inside the warp come from ballots of
        // its first and last entries; only groups that cross the warp's edge
        // are followed in shared memory
        const int lane = threadIdx.x & 31, w0 = i - lane;
        const unsigned act = cnt - w0 >= 32 ? 0xFFFFFFFFu : (1u << (cnt - w0)) - 1u;
        uint32_t g = sg[i], k = sk[i];
        const bool first = i == 0 || sg[i - 1] != g;
        const bool last = i + 1 == cnt || sg[i + 1] != g;
        const unsigned fb = __ballot_sync(act, first) & (0xFFFFFFFFu >> (31 - lane));  // lanes 0..lane
        const unsigned lb = __ballot_sync(act, last) & (0xFFFFFFFFu << lane);          // lanes lane..31
        int rs, rend;
        if (fb) {
            rs = w0 + (31 - __clz(fb));
        } else {
            rs = w0;
            while (rs > 0 && sg[rs - 1] == g) --rs;
        }
        if (lb) {
            rend = w0 + __ffs(lb);
        } else {
            rend = w0 + 32;
            while (rend < cnt && sg[rend] == g) ++rend;
        }
        int less = 0, eqb = 0, eqt = 0;
        for (int j = rs; j < rend; ++j) {
            uint32_t kj = sk[j];
            less += kj < k;
            int e = kj == k;
            eqt += e;
            eqb += e & (j < i);
        }
        int off = less + eqb;
        if (off != i - rs) SA[g + off] = (int32_t)sp[i];  // unchanged places are not rewritten
        uint32_t gn = g + (uint32_t)less;
        bool sv = eqt >= 2;
        tp[b + rs + off] = sp[i];
        tg[b + rs + off] = gn | (sv ? SURV : 0u);
        surv += sv;
    }
    // block sum of survivors
    uint32_t ex = block_excl<uint32_t>(surv, 0, wtot);
    if (threadIdx.x == RT_THREADS - 1) tile_surv[blockIdx.x] = ex + surv;
}

// Applies the new ranks of a tile and compacts its survivors (order kept, so
// every group stays contiguous).
__global__ void __launch_bounds__(RT_THREADS) k_compact_small(const uint32_t *__restrict__ tp,
                                                              const uint32_t *__restrict__ tg,
                                                              const uint32_t *__restrict__ wg_old,
                                                              const uint32_t *__restrict__ tile_begin,
                                                              const uint32_t *__restrict__ tile_off, int64_t ntiles,
                                                              int64_t N, int32_t *__restrict__ rank,
                                                              uint32_t *__restrict__ op,
                                                              uint32_t *__restrict__ og) {
    __shared__ uint32_t wtot[32];
    __shared__ uint32_t tot;
    int64_t b = tile_begin[blockIdx.x];
    int64_t e = blockIdx.x + 1 < ntiles ? (int64_t)tile_begin[blockIdx.x + 1] : N;
    uint32_t base = tile_off[blockIdx.x];
    uint32_t running = 0;
    for (int64_t c0 = b; c0 < e; c0 += RT_THREADS) {
        int64_t i = c0 + threadIdx.x;
        uint32_t p = 0, g = 0, sv = 0;
        if (i < e) {
            p = tp[i];
            g = tg[i];
            // entry i of the new order lies in the same old group as entry i of the
            // old list; its rank changes only if its sub-group does not start there
            if ((g & ~SURV) != wg_old[i]) rank[p] = (int32_t)(g & ~SURV);
            sv = g >> 31;
        }
        uint32_t ex = block_excl<uint32_t>(sv, 0, wtot);
        if (sv) {
            op[base + running + ex] = p;
            og[base + running + ex] = g & ~SURV;
        }
        if (threadIdx.x == RT_THREADS - 1) tot = ex + sv;
        __syncthreads();
        running += tot;
        __syncthreads();
    }
}

// ---- S1: doubling rounds, groups > SMALL_MAX (radix sort by (group, key)) ----
__global__ void k_large_keys(const uint32_t *__restrict__ lp, const uint32_t *__restrict__ lg, int64_t NL,
                             const int32_t *__restrict__ rank, uint32_t h, int64_t n, uint32_t *__restrict__ err,
                             uint64_t *__restrict__ ck, uint32_t *__restrict__ cv) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= NL) return;
    int64_t ph = (int64_t)lp[i] + h;
    uint32_t r = 0;
    if (ph < n) r = (uint32_t)rank[ph];
    else atomicOr(err, 1u);
    ck[i] = ((uint64_t)lg[i] << 32) | r;
    cv[i] = (uint32_t)i;
}

__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t *__restrict__ a, int64_t n, uint64_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_large_assign(const uint64_t *__restrict__ ck, const uint32_t *__restrict__ cv, int64_t NL,
                               const uint32_t *__restrict__ lp, int32_t *__restrict__ SA,
                               uint32_t *__restrict__ tp, uint32_t *__restrict__ tg,
                               uint32_t *__restrict__ gsize) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= NL) return;
    uint64_t c = ck[j];
    uint32_t g = (uint32_t)(c >> 32);
    uint32_t p = lp[cv[j]];
    int64_t fg = lower_bound_u64(ck, NL, (uint64_t)g << 32);
    int64_t fe = lower_bound_u64(ck, NL, c);
    int64_t ee = lower_bound_u64(ck, NL, c + 1);
    SA[g + (j - fg)] = (int32_t)p;
    uint32_t gn = g + (uint32_t)(fe - fg);
    int64_t eqt = ee - fe;
    tp[j] = p;
    tg[j] = gn | (eqt >= 2 ? SURV : 0u);
    if (j == fe) gsize[gn] = (uint32_t)eqt;
}

__global__ void k_large_flags(const uint32_t *__restrict__ tp, const uint32_t *__restrict__ tg, int64_t NL,
                              int32_t *__restrict__ rank, const uint32_t *__restrict__ gsize,
                              uint32_t *__restrict__ fs, uint32_t *__restrict__ fl) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= NL) return;
    uint32_t g = tg[j], gn = g & ~SURV;
    rank[tp[j]] = (int32_t)gn;
    uint32_t sz = (g & SURV) ? gsize[gn] : 0u;
    fs[j] = (sz >= 2 && sz <= (uint32_t)SMALL_MAX) ? 1u : 0u;
    fl[j] = sz > (uint32_t)SMALL_MAX ? 1u : 0u;
}

__global__ void k_large_scatter(const uint32_t *__restrict__ tp, const uint32_t *__restrict__ tg,
                                const uint32_t *__restrict__ fs, const uint32_t *__restrict__ fl,
                                const uint32_t *__restrict__ ps, const uint32_t *__restrict__ pl, int64_t NL,
                                const uint32_t *__restrict__ small_base, uint32_t *__restrict__ sp,
                                uint32_t *__restrict__ sg, uint32_t *__restrict__ lp2, uint32_t *__restrict__ lg2) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= NL) return;
    uint32_t gn = tg[j] & ~SURV;
    if (fs[j]) {
        uint32_t o = small_base[0] + ps[j];
        sp[o] = tp[j];
        sg[o] = gn;
    } else if (fl[j]) {
        lp2[pl[j]] = tp[j];
        lg2[pl[j]] = gn;
    }
}

// ---- S2: BWT extraction, packing, Occ ------------------------------------------
// One thread packs 8 consecutive BWT symbols into a 32-bit payload word and
// counts them; the D/8 threads of a block reduce their counts with shuffles.
__global__ void k_pack(const uint8_t *__restrict__ T, const int32_t *__restrict__ SA, int64_t n, int log2D, int bb,
                       int64_t nblocks, uint8_t *__restrict__ blocks, uint32_t *__restrict__ cnt) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t total = nblocks << (log2D - 3);
    if (t >= total) return;  // total is a multiple of 32 when D >= 256 ... guarded reduce below
    int64_t q0 = t << 3;
    int64_t b = q0 >> log2D;
    uint32_t pl[3] = {0, 0, 0};  // plane bytes of these 8 symbols
    uint32_t c[SIGMA] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        int64_t i = q0 + j;
        if (i < n) {
            int32_t s = SA[i];
            uint32_t sym = s ? T[s - 1] : T[n - 1];
            pl[0] |= (sym & 1u) << j;
            pl[1] |= ((sym >> 1) & 1u) << j;
            pl[2] |= ((sym >> 2) & 1u) << j;
            c[sym]++;
        }
    }
    int o = (int)(q0 & ((1 << log2D) - 1));
    uint8_t *blk = blocks + b * bb;
    if (log2D == 5) store_planes32(blk, pl[0], pl[1], pl[2], __activemask(), true);
    else store_planes(blk + HEADER_BYTES + 32 * (o >> 6), pl[0], pl[1], pl[2], __activemask(), true);
    // segmented reduce over the D/8 lanes of this block (D/8 in {4,8,16,32})
    int seg = 1 << (log2D - 3);
    unsigned full = __activemask();
#pragma unroll
    for (int a = 0; a < SIGMA; ++a) {
        uint32_t v = c[a];
        for (int d = seg >> 1; d >= 1; d >>= 1) v += __shfl_down_sync(full, v, d, seg);
        c[a] = v;
    }
    if ((t & (seg - 1)) == 0)
        for (int a = 0; a < SIGMA; ++a) cnt[(int64_t)a * nblocks + b] = c[a];
}

// Header of block b: rank(a, b*D) = (exclusive prefix of row a at b).  The
// scan ran over the whole [6][nblocks] array, so subtract the row's start.  A
// batch has fewer than 2^31 symbols, so D = 32 counts need no span base.
__global__ void k_headers(const uint32_t *__restrict__ ex, int64_t nblocks, int bb, uint8_t *__restrict__ blocks) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    uint8_t *h = blocks + b * bb;
    uint32_t *h32 = reinterpret_cast<uint32_t *>(h);
    if (bb == 32) {  // D = 32: words 0..4 = A..N; words 5..7 hold the planes
#pragma unroll
        for (int a = 1; a < SIGMA; ++a) h32[a - 1] = ex[(int64_t)a * nblocks + b] - ex[(int64_t)a * nblocks];
        return;
    }
#pragma unroll
    for (int a = 0; a < SIGMA; ++a) h32[a] = ex[(int64_t)a * nblocks + b] - ex[(int64_t)a * nblocks];
    *reinterpret_cast<uint32_t *>(h + 24) = 0;  // high bytes 0..3
    *reinterpret_cast<uint32_t *>(h + 28) = 0;  // high bytes 4..5, reserved
}

static inline unsigned nb_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

int build_batch_impl(const uint8_t *seq_dev, const int64_t *lens, int64_t n_seq, const rb3_opts &o,
                     cudaStream_t st, rb3_index *out) {
    const int both = o.single_strand ? 0 : 1;
    const int mult = both ? 2 : 1;
    int D = o.occ_interval ? o.occ_interval : kDefaultOccInterval;
    RB3_CHECK_ARG(valid_occ_interval(D), "occ_interval must be 32, 64, 128 or 256");
    RB3_CHECK_ARG(o.sa_sample == 0 || (o.sa_sample >= 2 && o.sa_sample <= 1024 && (o.sa_sample & (o.sa_sample - 1)) == 0),
                  "sa_sample must be 0 or a power of two in [2, 1024]");
    std::vector<int64_t> in_off(n_seq + 1, 0), out_off(n_seq + 1, 0);
    for (int64_t s = 0; s < n_seq; ++s) {
        RB3_CHECK_ARG(lens[s] >= 0, "negative string length");
        in_off[s + 1] = in_off[s] + lens[s];
        out_off[s + 1] = out_off[s] + mult * (lens[s] + 1);
    }
    const int64_t total_in = in_off[n_seq], n = out_off[n_seq];
    if (n >= (int64_t(1) << 31) - 64) {
        set_error("batch too large: %lld symbols (limit 2^31 - 64 per batch)", (long long)n);
        return RB3_E_INVAL;
    }
    out->D = D;
    out->log2D = ilog2(D);
    out->block_bytes = block_bytes_for(D);
    out->single_strand = !both;
    out->n = n;
    out->m = n_seq * mult;
    out->nblocks = n / D + 1;
    out->str_end.clear();
    for (int64_t s = 0; s < n_seq; ++s) {
        out->str_end.push_back(out_off[s] + lens[s]);
        if (both) out->str_end.push_back(out_off[s] + 2 * lens[s] + 1);
    }
    DevBuf blocks_buf;
    RB3_TRY(blocks_buf.alloc((size_t)out->nblocks * out->block_bytes, st));
    RB3_CUDA_TRY(cudaMemsetAsync(blocks_buf.p, 0, (size_t)out->nblocks * out->block_bytes, st));
    DevBuf Tb, isab;
    RB3_TRY(Tb.alloc((size_t)n + 64, st));
    RB3_CUDA_TRY(cudaMemsetAsync(Tb.p, 0, (size_t)n + 64, st));
    RB3_TRY(isab.alloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1), st));
    uint8_t *T = Tb.as<uint8_t>();
    int32_t *rank = isab.as<int32_t>();

    if (n > 0) {
        bool has_n = false;  // N-free batches take the 2-bit round-0 key
        // ---- S0 ----
        {
            Phase ph("build.encode", st);
            DevBuf offs, bad;
            RB3_TRY(offs.alloc(sizeof(int64_t) * 2 * (n_seq + 1), st));
            RB3_TRY(bad.alloc(sizeof(int), st));
            int64_t *d_in = offs.as<int64_t>(), *d_out = d_in + (n_seq + 1);
            RB3_CUDA_TRY(cudaMemcpyAsync(d_in, in_off.data(), sizeof(int64_t) * (n_seq + 1), cudaMemcpyHostToDevice, st));
            RB3_CUDA_TRY(cudaMemcpyAsync(d_out, out_off.data(), sizeof(int64_t) * (n_seq + 1), cudaMemcpyHostToDevice, st));
            RB3_CUDA_TRY(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
            if (total_in > 0) {
                unsigned grid = nb_for(total_in, 256);
                if (grid > 65535u * 16) grid = 65535u * 16;
                RB3_LAUNCH(k_encode, grid, 256, 0, st, seq_dev, d_in, d_out, n_seq, total_in, both, T, bad.as<int>());
            }
            RB3_LAUNCH(k_sentinels, nb_for(n_seq, 256), 256, 0, st, d_in, d_out, n_seq, both, T);
            int hbad = 0;
            RB3_CUDA_TRY(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
            RB3_CUDA_TRY(cudaStreamSynchronize(st));
            if (hbad & 1) {
                set_error("input symbol outside 1..5 (A,C,G,T,N codes)");
                return RB3_E_INVAL;
            }
            has_n = (hbad & 2) != 0;
        }
        // ---- S1 round 0 ----
        DevBuf SAb, gsizeb;
        RB3_TRY(SAb.alloc(sizeof(int32_t) * n, st));
        RB3_TRY(gsizeb.alloc(sizeof(uint32_t) * n, st));
        int32_t *SA = SAb.as<int32_t>();
        uint32_t *gsize = gsizeb.as<uint32_t>();
        DevBuf sp, sg, sp2, sg2, tp, tg, lp, lg;
        int64_t NS = 0, NL = 0;
        DevBuf counters;
        RB3_TRY(counters.alloc(sizeof(uint32_t) * 4, st));
        RB3_CUDA_TRY(cudaMemsetAsync(counters.p, 0, sizeof(uint32_t) * 4, st));
        uint32_t *d_cnt = counters.as<uint32_t>();
        uint32_t *d_err = d_cnt + 2;
        {
            Phase ph("build.sort0", st);
            DevBuf k0, k1, v1;
            RB3_TRY(k0.alloc(sizeof(uint64_t) * n, st));
            RB3_TRY(k1.alloc(sizeof(uint64_t) * n, st));
            RB3_TRY(v1.alloc(sizeof(uint32_t) * n, st));
            uint32_t *v0 = reinterpret_cast<uint32_t *>(SA);
            // The sort starts from (ka, va) and ends in (k0, SA): the six base-6 passes
            // return to their input, the five 2-bit ones end in the other buffer.
            // the sort starts from the (A) buffers and ends in (k0, SA): an even number
            // of passes returns to its input, an odd one ends in the other buffer
            const int passes = ((has_n ? H0_BITS : H4_BITS) + 7) / 8;
            uint32_t *vA = (passes & 1) ? v1.as<uint32_t>() : v0, *vB = (passes & 1) ? v0 : v1.as<uint32_t>();
            bool alt = false;
            DevBuf hv;
            RB3_TRY(hv.alloc(sizeof(uint32_t) * n, st));
            if (has_n) {
                uint64_t *kA = (passes & 1) ? k1.as<uint64_t>() : k0.as<uint64_t>();
                uint64_t *kB = (passes & 1) ? k0.as<uint64_t>() : k1.as<uint64_t>();
                {
                    Phase pk("k.init_keys", st, 13.0 * n);  // 1 text byte in, 8-byte key + 4-byte value out
                    RB3_LAUNCH(k_init_keys, nb_for(n, 256), 256, 0, st, T, n, kA, vA);
                }
                RB3_TRY(radix_sort_pairs(kA, vA, kB, vB, n, 0, H0_BITS, st, &alt));
                RB3_LAUNCH((k_heads<false, uint64_t>), nb_for(n, 256), 256, 0, st, alt ? kB : kA, n,
                           hv.as<uint32_t>());
            } else {
                Key4 *kA = (passes & 1) ? k1.as<Key4>() : k0.as<Key4>();
                Key4 *kB = (passes & 1) ? k0.as<Key4>() : k1.as<Key4>();
                {
                    Phase pk("k.init_keys", st, (1.0 + sizeof(Key4) + 4.0) * n);  // text in, key + value out
                    RB3_LAUNCH(k_init_keys4, nb_for((n + K4_PER - 1) / K4_PER, 256), 256, 0, st, T, n, kA, vA);
                }
                if constexpr (sizeof(Key4) == 4)
                    RB3_TRY(radix_sort_pairs32(reinterpret_cast<uint32_t *>(kA), vA, reinterpret_cast<uint32_t *>(kB),
                                               vB, n, 0, H4_BITS, st, &alt));
                else
                    RB3_TRY(radix_sort_pairs(reinterpret_cast<uint64_t *>(kA), vA, reinterpret_cast<uint64_t *>(kB),
                                             vB, n, 0, H4_BITS, st, &alt));
                RB3_LAUNCH((k_heads<true, Key4>), nb_for(n, 256), 256, 0, st, alt ? kB : kA, n, hv.as<uint32_t>());
            }
            if ((alt ? vB : vA) != v0)
                RB3_CUDA_TRY(cudaMemcpyAsync(SA, alt ? vB : vA, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st));
            RB3_TRY(scan_u32(hv.as<uint32_t>(), hv.as<uint32_t>(), n, true, 1, st));  // gstart
            k0.release();
            k1.release();
            v1.release();
            // the head list holds at most n / 2 groups; the large list at most n entries
            const int64_t hcap = n / 2 + 2;
            DevBuf hk0, hk1, hv0, hv1, gsz, goff;
            RB3_TRY(hk0.alloc(sizeof(uint32_t) * hcap, st));
            RB3_TRY(hv0.alloc(sizeof(uint32_t) * hcap, st));
            RB3_TRY(lp.alloc(sizeof(uint32_t) * (n + 1), st));
            RB3_TRY(lg.alloc(sizeof(uint32_t) * (n + 1), st));
            RB3_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, sizeof(uint32_t) * 2, st));
            RB3_LAUNCH(k_init_groups, nb_for((n + IG_TILE - 1) / IG_TILE, 1), IG_THREADS, 0, st,
                       reinterpret_cast<uint32_t *>(SA), hv.as<uint32_t>(), n, rank, gsize, d_cnt, hk0.as<uint32_t>(),
                       hv0.as<uint32_t>(), lp.as<uint32_t>(), lg.as<uint32_t>());
            uint32_t hc[2];
            RB3_CUDA_TRY(cudaMemcpyAsync(hc, d_cnt, sizeof(hc), cudaMemcpyDeviceToHost, st));
            RB3_CUDA_TRY(cudaStreamSynchronize(st));
            const int64_t G = hc[0];  // groups of 2..SMALL_MAX
            NL = hc[1];
            if (G >= hcap || NL > n) {
                set_error("round 0: group lists overflow (%lld heads, %lld large)", (long long)G, (long long)NL);
                return RB3_E_CUDA;
            }
            // small groups in order of their first member's text position
            RB3_TRY(hk1.alloc(sizeof(uint32_t) * (G + 1), st));
            RB3_TRY(hv1.alloc(sizeof(uint32_t) * (G + 1), st));
            RB3_TRY(gsz.alloc(sizeof(uint32_t) * (G + 1), st));
            RB3_TRY(goff.alloc(sizeof(uint32_t) * (G + 1), st));
            bool halt = false;
            RB3_TRY(radix_sort_pairs32(hk0.as<uint32_t>(), hv0.as<uint32_t>(), hk1.as<uint32_t>(), hv1.as<uint32_t>(),
                                       G, 0, ilog2(n) + 1, st, &halt));
            const uint32_t *hval = halt ? hv1.as<uint32_t>() : hv0.as<uint32_t>();
            if (G > 0)
                RB3_LAUNCH(k_group_sizes, nb_for(G, 256), 256, 0, st, hval, G, gsize, gsz.as<uint32_t>());
            RB3_TRY(scan_u32(gsz.as<uint32_t>(), goff.as<uint32_t>(), G, false, 0, st));
            RB3_LAUNCH(k_tally, 1, 1, 0, st, goff.as<uint32_t>(), gsz.as<uint32_t>(), G, d_cnt, 0);
            RB3_CUDA_TRY(cudaMemcpyAsync(hc, d_cnt, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            RB3_CUDA_TRY(cudaStreamSynchronize(st));
            NS = hc[0];
            RB3_TRY(sp.alloc(sizeof(uint32_t) * (NS + NL + 1), st));
            RB3_TRY(sg.alloc(sizeof(uint32_t) * (NS + NL + 1), st));
            RB3_TRY(sp2.alloc(sizeof(uint32_t) * (NS + NL + 1), st));
            RB3_TRY(sg2.alloc(sizeof(uint32_t) * (NS + NL + 1), st));
            RB3_TRY(tp.alloc(sizeof(uint32_t) * (NS + NL + 1), st));
            RB3_TRY(tg.alloc(sizeof(uint32_t) * (NS + NL + 1), st));
            if (G > 0)
                RB3_LAUNCH(k_expand_groups, nb_for(G, 256), 256, 0, st, hval, gsz.as<uint32_t>(), goff.as<uint32_t>(),
                           G, reinterpret_cast<uint32_t *>(SA), sp.as<uint32_t>(), sg.as<uint32_t>(), rank);
        }
        // ---- S1 doubling rounds ----
        const int64_t capS = NS + NL + 1;
        DevBuf lp2, lg2, ltp, ltg, lck0, lck1, lcv0, lcv1, lfs, lfl, lps, lpl;
        if (NL > 0) {
            RB3_TRY(lp2.alloc(sizeof(uint32_t) * (NL + 1), st));
            RB3_TRY(lg2.alloc(sizeof(uint32_t) * (NL + 1), st));
            RB3_TRY(ltp.alloc(sizeof(uint32_t) * (NL + 1), st));
            RB3_TRY(ltg.alloc(sizeof(uint32_t) * (NL + 1), st));
            RB3_TRY(lck0.alloc(sizeof(uint64_t) * (NL + 1), st));
            RB3_TRY(lck1.alloc(sizeof(uint64_t) * (NL + 1), st));
            RB3_TRY(lcv0.alloc(sizeof(uint32_t) * (NL + 1), st));
            RB3_TRY(lcv1.alloc(sizeof(uint32_t) * (NL + 1), st));
            RB3_TRY(lfs.alloc(sizeof(uint32_t) * (NL + 1), st));
            RB3_TRY(lfl.alloc(sizeof(uint32_t) * (NL + 1), st));
            RB3_TRY(lps.alloc(sizeof(uint32_t) * (NL + 1), st));
            RB3_TRY(lpl.alloc(sizeof(uint32_t) * (NL + 1), st));
        }
        const int64_t max_tiles = (capS + RT_TILE - 1) / RT_TILE + 1;
        DevBuf tsurv, tbeg, toff;
        RB3_TRY(tsurv.alloc(sizeof(uint32_t) * max_tiles, st));
        RB3_TRY(tbeg.alloc(sizeof(uint32_t) * max_tiles, st));
        RB3_TRY(toff.alloc(sizeof(uint32_t) * max_tiles, st));
        int gbits = ilog2(n) + 1;
        uint32_t h = has_n ? H0 : H4;  // symbols the round-0 order is exact to
        int round = 0;
        static const char *kRoundNames[] = {
            "round.00", "round.01", "round.02", "round.03", "round.04", "round.05", "round.06", "round.07",
            "round.08", "round.09", "round.10", "round.11", "round.12", "round.13", "round.14", "round.15",
            "round.16", "round.17", "round.18", "round.19", "round.20", "round.21", "round.22", "round.23",
            "round.24", "round.25", "round.26", "round.27", "round.28", "round.29", "round.30", "round.31",
            "round.32", "round.33", "round.34", "round.35", "round.36", "round.37", "round.38", "round.39",
            "round.40"};
        while (NS + NL > 0) {
            Phase ph("build.round", st);
            // "bytes" of a per-round record = entries still unresolved at its start
            Phase pr_(kRoundNames[round < 40 ? round : 40], st, (double)(NS + NL));
            if (++round > 40 || h >= (uint32_t)n) {
                set_error("prefix doubling did not converge (round %d, h=%u)", round, h);
                return RB3_E_CUDA;
            }
            int64_t ntiles = (NS + RT_TILE - 1) / RT_TILE;
            if (NS > 0) {
                // per entry: 8 B list in, 4 B rank gather, 4 B SA out, 8 B (p, rank) out
                Phase pr("k.round_small", st, 24.0 * NS);
                RB3_LAUNCH(k_round_small, (unsigned)ntiles, RT_THREADS, 0, st, sp.as<uint32_t>(), sg.as<uint32_t>(), NS,
                           rank, h, n, d_err, SA, tp.as<uint32_t>(), tg.as<uint32_t>(), tsurv.as<uint32_t>(),
                           tbeg.as<uint32_t>());
            }
            if (NL > 0) {
                RB3_LAUNCH(k_large_keys, nb_for(NL, 256), 256, 0, st, lp.as<uint32_t>(), lg.as<uint32_t>(), NL, rank, h, n,
                           d_err, lck0.as<uint64_t>(), lcv0.as<uint32_t>());
                bool alt = false;
                RB3_TRY(radix_sort_pairs(lck0.as<uint64_t>(), lcv0.as<uint32_t>(), lck1.as<uint64_t>(),
                                         lcv1.as<uint32_t>(), NL, 0, 32 + gbits, st, &alt));
                const uint64_t *ck = alt ? lck1.as<uint64_t>() : lck0.as<uint64_t>();
                const uint32_t *cv = alt ? lcv1.as<uint32_t>() : lcv0.as<uint32_t>();
                RB3_LAUNCH(k_large_assign, nb_for(NL, 256), 256, 0, st, ck, cv, NL, lp.as<uint32_t>(), SA,
                           ltp.as<uint32_t>(), ltg.as<uint32_t>(), gsize);
            }
            // all keys of this round are read; now apply ranks and compact
            if (NS > 0) {
                RB3_TRY(scan_u32(tsurv.as<uint32_t>(), toff.as<uint32_t>(), ntiles, false, 0, st));
                RB3_LAUNCH(k_tally, 1, 1, 0, st, toff.as<uint32_t>(), tsurv.as<uint32_t>(), ntiles, d_cnt, 0);
                Phase pc("k.compact_small", st, 12.0 * NS);  // 8 B in, 4 B rank out (survivor writes not counted)
                RB3_LAUNCH(k_compact_small, (unsigned)ntiles, RT_THREADS, 0, st, tp.as<uint32_t>(), tg.as<uint32_t>(),
                           sg.as<uint32_t>(), tbeg.as<uint32_t>(), toff.as<uint32_t>(), ntiles, NS, rank, sp2.as<uint32_t>(),
                           sg2.as<uint32_t>());
            } else {
                RB3_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, sizeof(uint32_t), st));
            }
            RB3_CUDA_TRY(cudaMemsetAsync(d_cnt + 1, 0, sizeof(uint32_t), st));
            if (NL > 0) {
                RB3_LAUNCH(k_large_flags, nb_for(NL, 256), 256, 0, st, ltp.as<uint32_t>(), ltg.as<uint32_t>(), NL,
                           rank, gsize, lfs.as<uint32_t>(), lfl.as<uint32_t>());
                RB3_TRY(scan_u32(lfs.as<uint32_t>(), lps.as<uint32_t>(), NL, false, 0, st));
                RB3_TRY(scan_u32(lfl.as<uint32_t>(), lpl.as<uint32_t>(), NL, false, 0, st));
                RB3_LAUNCH(k_large_scatter, nb_for(NL, 256), 256, 0, st, ltp.as<uint32_t>(), ltg.as<uint32_t>(),
                           lfs.as<uint32_t>(), lfl.as<uint32_t>(), lps.as<uint32_t>(), lpl.as<uint32_t>(), NL,
                           d_cnt, sp2.as<uint32_t>(), sg2.as<uint32_t>(), lp2.as<uint32_t>(), lg2.as<uint32_t>());
                RB3_LAUNCH(k_tally, 1, 1, 0, st, lps.as<uint32_t>(), lfs.as<uint32_t>(), NL, d_cnt, 1);
                RB3_LAUNCH(k_tally, 1, 1, 0, st, lpl.as<uint32_t>(), lfl.as<uint32_t>(), NL, d_cnt + 1, 0);
            }
            uint32_t hc[3];
            RB3_CUDA_TRY(cudaMemcpyAsync(hc, d_cnt, sizeof(hc), cudaMemcpyDeviceToHost, st));
            RB3_CUDA_TRY(cudaStreamSynchronize(st));
            NS = hc[0];
            NL = hc[1];
            if (hc[2]) {
                set_error("prefix doubling: internal error (rank gather past the text end)");
                return RB3_E_CUDA;
            }
            if (NS > capS) {
                set_error("prefix doubling list overflow");
                return RB3_E_CUDA;
            }
            std::swap(sp.p, sp2.p);
            std::swap(sg.p, sg2.p);
            std::swap(lp.p, lp2.p);
            std::swap(lg.p, lg2.p);
            h *= 2;
        }
        // ---- S2 ----
        {
            Phase ph("build.pack", st);
            int64_t nb = out->nblocks;
            DevBuf cnt;
            RB3_TRY(cnt.alloc(sizeof(uint32_t) * SIGMA * nb, st));
            int64_t threads = nb << (out->log2D - 3);
            {
                // per symbol: 4 B SA in, 1 B text gather, payload out; per block 24 B of counts
                Phase pp("k.pack", st, n * (5.0 + 0.5) + 24.0 * nb);
                RB3_LAUNCH(k_pack, nb_for(threads, 256), 256, 0, st, T, SA, n, out->log2D, out->block_bytes, nb,
                           blocks_buf.as<uint8_t>(), cnt.as<uint32_t>());
            }
            RB3_TRY(scan_u32(cnt.as<uint32_t>(), cnt.as<uint32_t>(), SIGMA * nb, false, 0, st));
            RB3_LAUNCH(k_headers, nb_for(nb, 256), 256, 0, st, cnt.as<uint32_t>(), nb, out->block_bytes,
                       blocks_buf.as<uint8_t>());
        }
        // ---- sampled suffix array (optional) ----
        if (o.sa_sample) {
            Phase ps_("build.sample", st);
            out->sa_s = o.sa_sample;
            RB3_TRY(sample_batch(out, SA, st));
        }
    }
    out->blocks = static_cast<uint8_t *>(blocks_buf.detach());
    out->text = static_cast<uint8_t *>(Tb.detach());
    out->isa = static_cast<int32_t *>(isab.detach());
    RB3_TRY(finalize_counts(out, st));
    return RB3_OK;
}

}  // namespace rb3
