// Cell tables of Algorithm 5 (the revised BWA-SW of Section "Finding inexact
// matches with BWA-SW"): one warp's table of (bi-interval, H, E, F) cells in
// shared memory, the children of a cell by BackwardExt (Algorithm 3), and the
// band order.  Shared by the linear-query kernel (haplotype diversity) and the
// query-DAWG kernel (BWA-SW).
#pragma once

#include <climits>
#include <cstdint>

#include "common.cuh"

namespace rb3 {
namespace dv {

constexpr int32_t DV_NEG = -(1 << 30);
constexpr unsigned DV_FULL = 0xffffffffu;
constexpr int DV_CAP_G = 65534;  // cells of the global-memory tier (indexes + 1 fit 16 bits)

// Hash slots of a table of cap cells: twice the next power of two.
__host__ __device__ constexpr int dv_hash_slots(int cap) {
    int h = 1;
    while (h < cap) h <<= 1;
    return 2 * h;
}
// A table of cap cells (structure of arrays: k, k', s, H, E, F, a worklist
// ring of cell indexes, a flag byte) and its hash index (cell index + 1, 0 =
// empty; open addressing with linear probing), rounded to 16 bytes.
constexpr int DV_HIST = 256;  // score bins of the band selection
__host__ __device__ constexpr size_t dv_warp_bytes(int cap) {
    return DV_HIST * 4 + ((size_t)cap * (3 * 8 + 3 * 4 + 2 + 1) + (size_t)dv_hash_slots(cap) * 2 + 15) / 16 * 16;
}

struct DvParams {
    int32_t a, b, q, e, W, redundancy;
};

// One warp's cells.
struct DvTab {
    int64_t *k, *kp, *s;
    int32_t *H, *E, *F;
    unsigned short *queue;  // worklist ring of the cells to extend by deletions
    uint8_t *flag;          // bit 0: in the worklist; bit 1: taken into the band
    unsigned short *slot;   // hash index over (k, k', s)
    uint32_t *hist;         // [DV_HIST] scratch of the band selection
};

// The table's counters (warp-uniform): cells, worklist head and tail.
struct DvSt {
    int tn, qh, qt;
};

template <int CAP> __device__ __forceinline__ DvTab dv_tab(uint8_t *base) {
    static_assert(CAP % 2 == 0 && CAP <= DV_CAP_G, "cell count: even, indexes + 1 in 16 bits");
    DvTab t;
    t.k = reinterpret_cast<int64_t *>(base);
    t.kp = t.k + CAP;
    t.s = t.kp + CAP;
    t.H = reinterpret_cast<int32_t *>(t.s + CAP);
    t.E = t.H + CAP;
    t.F = t.E + CAP;
    t.queue = reinterpret_cast<unsigned short *>(t.F + CAP);
    t.flag = reinterpret_cast<uint8_t *>(t.queue + CAP);
    t.slot = reinterpret_cast<unsigned short *>(t.flag + CAP);  // CAP is even: 2-byte aligned
    t.hist = reinterpret_cast<uint32_t *>(base + dv_warp_bytes(CAP) - DV_HIST * 4);
    return t;
}

__device__ __forceinline__ uint32_t dv_hash(int64_t k, int64_t kp, int64_t s);

// Clears the whole hash index (a table in memory not yet used).
template <int CAP> __device__ __forceinline__ void dv_clear_all(const DvTab &T, DvSt &st, int lane) {
    for (int i = lane; i < dv_hash_slots(CAP); i += 32) T.slot[i] = 0;
    st.tn = st.qh = st.qt = 0;
    __syncwarp();
}

// Empties the table (the warp together).  Small hash indexes are cleared
// whole; a large one only at the slots of the st.tn cells in use (each cell's
// slot found first, then all cleared, so no probe crosses a cleared slot).
template <int CAP> __device__ __forceinline__ void dv_clear(const DvTab &T, DvSt &st, int lane) {
    constexpr int HS = dv_hash_slots(CAP);
    if (HS <= 8192 || st.tn * 4 > HS) {
        for (int i = lane; i < HS; i += 32) T.slot[i] = 0;
    } else {
        for (int j0 = 0; j0 < st.tn; j0 += 32) {
            const int j = j0 + lane;
            uint32_t pos = 0;
            if (j < st.tn) {
                pos = dv_hash(T.k[j], T.kp[j], T.s[j]) & (HS - 1);
                while (T.slot[pos] != (unsigned short)(j + 1)) pos = (pos + 1) & (HS - 1);
            }
            __syncwarp();
            if (j < st.tn) T.slot[pos] = 0;
            __syncwarp();
        }
    }
    st.tn = 0;
    st.qh = 0;
    st.qt = 0;
    __syncwarp();
}

__device__ __forceinline__ uint32_t dv_hash(int64_t k, int64_t kp, int64_t s) {
    uint64_t x = (uint64_t)k * 0x9E3779B97F4A7C15ull ^ (uint64_t)kp * 0xC2B2AE3D27D4EB4Full ^
                 (uint64_t)s * 0x165667B19E3779F9ull;
    x ^= x >> 29;
    x *= 0xBF58476D1CE4E5B9ull;
    return (uint32_t)(x >> 32);
}

// BackwardExt (Algorithm 3) of (k, k', s) by A, C, G and T at once, from the
// ranks of every symbol at k and at k + s: child a has s = d(a),
// k = C(a) + rank(a, k), k' = k' + the d of the complements of the symbols
// below comp(a).
template <int NS>
__device__ __forceinline__ void dv_children(const OccView &V, int64_t k, int64_t kp, int64_t s, int64_t ck[4],
                                            int64_t ckp[4], int64_t cs[4]) {
    int64_t r0[SIGMA], r1[SIGMA], d[SIGMA];
    rank_all<NS>(V, k, r0);
    rank_all<NS>(V, k + s, r1);
#pragma unroll
    for (int i = 0; i < SIGMA; ++i) d[i] = r1[i] - r0[i];
#pragma unroll
    for (int a = 1; a <= 4; ++a) {
        const int ac = comp_sym(a);
        int64_t add = 0;
#pragma unroll
        for (int b = 0; b < SIGMA; ++b)
            if (b < ac) add += d[comp_sym(b)];
        ck[a - 1] = V.C[a] + r0[a];
        ckp[a - 1] = kp + add;
        cs[a - 1] = d[a];
    }
}

// Raises the cells offered by the lanes with `want` -- (k, k', s) to H =
// max(H, h), E = max(E, ev), F = max(F, fv) -- adding those absent; a cell
// that is new, or whose H or F rises, joins the worklist unless it is in it.
// Lanes offering the same cell are combined first (the maxima, one leader),
// so the leaders hold distinct keys: each looks its key up in the hash index,
// raises the cell it finds, or, absent, takes a new cell (numbered in lane
// order after st.tn) and claims a free slot for it.  Called by the whole warp;
// st stays warp-uniform; sets overflow, changing nothing, when the new cells
// do not fit.
template <int CAP>
__device__ __forceinline__ void dv_upsert_batch(const DvTab &T, DvSt &st, bool want, int64_t k, int64_t kp, int64_t s,
                                                int32_t h, int32_t ev, int32_t fv, int lane, bool &overflow) {
    const unsigned vm = __ballot_sync(DV_FULL, want);
    if (!vm) return;
    const unsigned g = __match_any_sync(DV_FULL, k) & __match_any_sync(DV_FULL, kp) & __match_any_sync(DV_FULL, s) & vm;
    if (want) {
        h = __reduce_max_sync(g, h);
        ev = __reduce_max_sync(g, ev);
        fv = __reduce_max_sync(g, fv);
    }
    const bool lead = want && (__ffs(g) - 1) == lane;
    constexpr uint32_t HM = dv_hash_slots(CAP) - 1;
    uint32_t pos = dv_hash(k, kp, s) & HM;
    int found = -1;
    if (lead) {
        for (;;) {
            const int sl = T.slot[pos];
            if (sl == 0) break;
            const int j = sl - 1;
            if (T.s[j] == s && T.k[j] == k && T.kp[j] == kp) {
                found = j;
                break;
            }
            pos = (pos + 1) & HM;
        }
    }
    __syncwarp();
    const unsigned nm = __ballot_sync(DV_FULL, lead && found < 0);
    const int nnew = __popc(nm);
    if (st.tn + nnew > CAP) {
        overflow = true;
        return;
    }
    int cell = -1;  // the cell to put on the worklist
    if (lead && found >= 0) {
        bool up = false;
        if (ev > T.E[found]) T.E[found] = ev;
        if (fv > T.F[found]) {
            T.F[found] = fv;
            up = true;
        }
        if (h > T.H[found]) {
            T.H[found] = h;
            up = true;
        }
        if (up && !(T.flag[found] & 1)) {
            T.flag[found] |= 1;
            cell = found;
        }
    } else if (lead) {
        const int j = st.tn + __popc(nm & ((1u << lane) - 1u));
        T.k[j] = k;
        T.kp[j] = kp;
        T.s[j] = s;
        T.H[j] = h;
        T.E[j] = ev;
        T.F[j] = fv;
        T.flag[j] = 1;
        cell = j;
        // a free slot from where the lookup stopped (other leaders may take some)
        while (atomicCAS(&T.slot[pos], (unsigned short)0, (unsigned short)(j + 1)) != 0) pos = (pos + 1) & HM;
    }
    const unsigned pm = __ballot_sync(DV_FULL, cell >= 0);
    if (cell >= 0) T.queue[(st.qt + __popc(pm & ((1u << lane) - 1u))) % CAP] = (unsigned short)cell;
    st.tn += nnew;
    st.qt += __popc(pm);
    __syncwarp();
}

// x[a] for a warp-uniform a in 0..3, by selects (the array stays in registers).
__device__ __forceinline__ int64_t dv_pick(const int64_t x[4], int a) {
    return a == 0 ? x[0] : (a == 1 ? x[1] : (a == 2 ? x[2] : x[3]));
}

// Band order: larger H first, then smaller k, k', s.
__device__ __forceinline__ bool dv_before(int32_t h1, int64_t k1, int64_t kp1, int64_t s1, int32_t h2, int64_t k2,
                                          int64_t kp2, int64_t s2) {
    if (h1 != h2) return h1 > h2;
    if (k1 != k2) return k1 < k2;
    if (kp1 != kp2) return kp1 < kp2;
    return s1 < s2;
}

// Lanes each holding a cell index (or -1) end up holding them in band order
// (-1 last): a bitonic sort across the warp (cells are distinct, so the order
// is total).
__device__ __forceinline__ int dv_sort_lanes(const DvTab &T, int idx, int lane) {
    const bool v = idx >= 0;
    int32_t h = v ? T.H[idx] : INT32_MIN;
    int64_t k = v ? T.k[idx] : INT64_MAX, kp = v ? T.kp[idx] : INT64_MAX, s = v ? T.s[idx] : INT64_MAX;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1)
#pragma unroll
        for (int j = size >> 1; j > 0; j >>= 1) {
            const int32_t oh = __shfl_xor_sync(DV_FULL, h, j);
            const int64_t ok = __shfl_xor_sync(DV_FULL, k, j), okp = __shfl_xor_sync(DV_FULL, kp, j),
                          os = __shfl_xor_sync(DV_FULL, s, j);
            const int oi = __shfl_xor_sync(DV_FULL, idx, j);
            // the lower lane of a pair keeps the earlier cell in an ascending run, the later one in a descending run
            const bool lower = (lane & j) == 0, asc = (lane & size) == 0;
            const bool other_first = oi >= 0 && (idx < 0 || dv_before(oh, ok, okp, os, h, k, kp, s));
            if (other_first == (lower == asc)) {
                h = oh;
                k = ok;
                kp = okp;
                s = os;
                idx = oi;
            }
        }
    return idx;
}

// Band by rounds: round r takes the first cell in band order among those of
// list[0 .. n) (list = null: cells 0 .. n) not yet taken (flag bit 1); lane
// r returns round r's cell.
__device__ __forceinline__ int dv_band_rounds(const DvTab &T, const unsigned short *list, int n, int keep,
                                              int lane) {
    int mine = -1;
    for (int r = 0; r < keep; ++r) {
        int bj = -1;
        int32_t bH = 0;
        int64_t bk = 0, bkp = 0, bs = 0;
        for (int x = lane; x < n; x += 32) {
            const int j = list ? list[x] : x;
            if (T.flag[j] & 2) continue;
            if (bj < 0 || dv_before(T.H[j], T.k[j], T.kp[j], T.s[j], bH, bk, bkp, bs)) {
                bj = j;
                bH = T.H[j];
                bk = T.k[j];
                bkp = T.kp[j];
                bs = T.s[j];
            }
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            const int oj = __shfl_xor_sync(DV_FULL, bj, off);
            const int32_t oH = __shfl_xor_sync(DV_FULL, bH, off);
            const int64_t ok = __shfl_xor_sync(DV_FULL, bk, off);
            const int64_t okp = __shfl_xor_sync(DV_FULL, bkp, off);
            const int64_t os = __shfl_xor_sync(DV_FULL, bs, off);
            if (oj >= 0 && (bj < 0 || dv_before(oH, ok, okp, os, bH, bk, bkp, bs))) {
                bj = oj;
                bH = oH;
                bk = ok;
                bkp = okp;
                bs = os;
            }
        }
        // keys are distinct, so every lane holds the same cell
        if (lane == r) mine = bj;
        __syncwarp();
        if (lane == 0) T.flag[bj] |= 2;
        __syncwarp();
    }
    return mine;
}

// The band: the W <= 32 cells of largest H (ties: smaller k, k', s) of the
// table's tn cells; lane r returns the r-th (-1 past min(tn, W)).  A table that
// fits the lanes is sorted across the warp.  A larger one: the largest H, a
// histogram of how far below it every H lies (DV_HIST bins), the bin b where
// the count from the top reaches W; the cells above bin b (fewer than W) are
// all in the band and are sorted across the warp, and the cells of bin b (one
// score) fill the remaining places by (k, k', s) -- sorted across the warp
// when they fit the lanes, else by rounds.  When the top DV_HIST scores hold
// fewer than W cells, or bin b holds more cells than the list can take, the
// band is taken by rounds over the whole table.
template <int CAP> __device__ __forceinline__ int dv_band(const DvTab &T, int tn, int W, int lane) {
    const int keep = tn < W ? tn : W;
    if (tn <= 32) {
        const int j = dv_sort_lanes(T, lane < tn ? lane : -1, lane);
        return lane < keep ? j : -1;
    }
    int32_t mh = INT32_MIN;
    for (int j = lane; j < tn; j += 32) mh = max(mh, T.H[j]);
    mh = __reduce_max_sync(DV_FULL, mh);
    for (int i = lane; i < DV_HIST; i += 32) T.hist[i] = 0;
    __syncwarp();
    for (int j = lane; j < tn; j += 32) {
        const int64_t d = (int64_t)mh - T.H[j];
        if (d < DV_HIST) atomicAdd(&T.hist[d], 1u);
    }
    __syncwarp();
    // bins 8 a lane: the first bin where the count from the top reaches W
    constexpr int PB = DV_HIST / 32;
    uint32_t c[PB], lt = 0;
#pragma unroll
    for (int i = 0; i < PB; ++i) {
        c[i] = T.hist[lane * PB + i];
        lt += c[i];
    }
    uint32_t incl = lt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t u = __shfl_up_sync(DV_FULL, incl, d);
        if (lane >= d) incl += u;
    }
    uint32_t before = incl - lt;  // cells in the bins of lower lanes
    int bstar = -1;
    uint32_t above = 0;
#pragma unroll
    for (int i = 0; i < PB; ++i) {
        if (bstar < 0 && before + c[i] >= (uint32_t)W) {
            bstar = lane * PB + i;
            above = before;
        }
        before += c[i];
    }
    const unsigned found = __ballot_sync(DV_FULL, bstar >= 0);
    if (!found) return dv_band_rounds(T, nullptr, tn, keep, lane);
    const int src = __ffs(found) - 1;
    bstar = __shfl_sync(DV_FULL, bstar, src);
    const int nabove = (int)__shfl_sync(DV_FULL, above, src);
    const int nties = (int)T.hist[bstar];
    if (nties > CAP - 32) return dv_band_rounds(T, nullptr, tn, keep, lane);
    // the cells above bin b to list[0 ..), those of bin b to list[32 ..)
    unsigned short *list = T.queue;
    int na = 0, nt = 0;
    for (int j0 = 0; j0 < tn; j0 += 32) {
        const int j = j0 + lane;
        const int64_t d = j < tn ? (int64_t)mh - T.H[j] : DV_HIST;
        const unsigned ma = __ballot_sync(DV_FULL, d < bstar), mt = __ballot_sync(DV_FULL, d == bstar);
        const unsigned lt_mask = (1u << lane) - 1u;
        if (d < bstar) list[na + __popc(ma & lt_mask)] = (unsigned short)j;
        if (d == bstar) list[32 + nt + __popc(mt & lt_mask)] = (unsigned short)j;
        na += __popc(ma);
        nt += __popc(mt);
    }
    __syncwarp();
    const int ia = dv_sort_lanes(T, lane < nabove ? (int)list[lane] : -1, lane);
    const int need = keep - nabove;  // places for bin b's cells
    int it;
    if (nties <= 32) {
        it = dv_sort_lanes(T, lane < nties ? (int)list[32 + lane] : -1, lane);
    } else {
        it = dv_band_rounds(T, list + 32, nties, need, lane);
    }
    // lane r: the r-th cell above bin b, else bin b's (r - nabove)-th
    const int from_t = __shfl_sync(DV_FULL, it, (lane - nabove) & 31);
    return lane < nabove ? ia : (lane < keep ? from_t : -1);
}

// The deletion closure: cells are taken off the worklist 32 at a time; each
// with H or F still giving a positive F to its children extends them (F =
// max(H - q, F) - e); a child that is new or whose H or F rises joins the
// worklist again.  The recurrences are monotone, so the closure is the same in
// any order.
template <int NS, int CAP>
__device__ __forceinline__ void dv_close(const OccView &V, const DvTab &T, DvSt &st, const DvParams &p, int lane,
                                         bool &overflow, unsigned long long &n_ext) {
    while (!overflow && st.qh < st.qt) {
        const int cnt = st.qt - st.qh < 32 ? st.qt - st.qh : 32;
        int32_t fv = DV_NEG;
        int64_t yk[4] = {0, 0, 0, 0}, ykp[4] = {0, 0, 0, 0}, ys[4] = {0, 0, 0, 0};
        if (lane < cnt) {
            const int j = T.queue[(st.qh + lane) % CAP];
            T.flag[j] &= (uint8_t)~1u;
            fv = max(T.H[j] - p.q, T.F[j]) - p.e;
            if (fv > 0) dv_children<NS>(V, T.k[j], T.kp[j], T.s[j], yk, ykp, ys);
        }
        st.qh += cnt;
        const bool ext = lane < cnt && fv > 0;
        n_ext += __popc(__ballot_sync(DV_FULL, ext));
        __syncwarp();
        // one call site for the four children (a smaller kernel: the upsert is long)
#pragma unroll 1
        for (int a = 0; a < 4 && !overflow; ++a) {
            const int64_t k = dv_pick(yk, a), kp = dv_pick(ykp, a), s = dv_pick(ys, a);
            dv_upsert_batch<CAP>(T, st, ext && s > 0, k, kp, s, fv, DV_NEG, fv, lane, overflow);
        }
    }
}

}  // namespace dv
}  // namespace rb3
