// Cell tables of Algorithm 5 (the revised BWA-SW of Section "Finding inexact
// matches with BWA-SW"): one warp's table of (bi-interval, H, E, F) cells in
// shared memory, the children of a cell by BackwardExt (Algorithm 3), and the
// band order.  Shared by the linear-query kernel (haplotype diversity) and the
// query-DAWG kernel (BWA-SW).
#pragma once

#include "common.cuh"

namespace rb3 {
namespace dv {

constexpr int32_t DV_NEG = -(1 << 30);
constexpr unsigned DV_FULL = 0xffffffffu;
__host__ __device__ constexpr size_t dv_warp_bytes(int cap) { return (size_t)cap * (3 * 8 + 3 * 4 + 1); }

struct DvParams {
    int32_t a, b, q, e, W, redundancy;
};

// One warp's cells, structure of arrays.
struct DvTab {
    int64_t *k, *kp, *s;
    int32_t *H, *E, *F;
    uint8_t *flag;  // bit 0: to be extended by deletions; bit 1: taken into the band
};

template <int CAP> __device__ __forceinline__ DvTab dv_tab(uint8_t *base) {
    DvTab t;
    t.k = reinterpret_cast<int64_t *>(base);
    t.kp = t.k + CAP;
    t.s = t.kp + CAP;
    t.H = reinterpret_cast<int32_t *>(t.s + CAP);
    t.E = t.H + CAP;
    t.F = t.E + CAP;
    t.flag = reinterpret_cast<uint8_t *>(t.F + CAP);
    return t;
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

// Finds (k, k', s) among the first tn cells: its index or -1 (warp-uniform).
__device__ __forceinline__ int dv_find(const DvTab &T, int tn, int64_t k, int64_t kp, int64_t s, int lane) {
    for (int j0 = 0; j0 < tn; j0 += 32) {
        const int j = j0 + lane;
        const bool hit = j < tn && T.s[j] == s && T.k[j] == k && T.kp[j] == kp;
        const unsigned m = __ballot_sync(DV_FULL, hit);
        if (m) return j0 + __ffs(m) - 1;
    }
    return -1;
}

// Raises the cell (k, k', s) to H = max(H, h), E = max(E, ev), F = max(F, fv),
// adding it when absent; a cell whose H or F rises is marked for deletion
// extension.  Warp-uniform; returns the new cell count.
template <int CAP>
__device__ __forceinline__ int dv_upsert(const DvTab &T, int tn, int64_t k, int64_t kp, int64_t s, int32_t h,
                                         int32_t ev, int32_t fv, int lane, bool &overflow) {
    const int j = dv_find(T, tn, k, kp, s, lane);
    if (j >= 0) {
        if (lane == 0) {
            bool up = false;
            if (ev > T.E[j]) T.E[j] = ev;
            if (fv > T.F[j]) {
                T.F[j] = fv;
                up = true;
            }
            if (h > T.H[j]) {
                T.H[j] = h;
                up = true;
            }
            if (up) T.flag[j] |= 1;
        }
        __syncwarp();
        return tn;
    }
    if (tn >= CAP) {
        overflow = true;
        return tn;
    }
    if (lane == 0) {
        T.k[tn] = k;
        T.kp[tn] = kp;
        T.s[tn] = s;
        T.H[tn] = h;
        T.E[tn] = ev;
        T.F[tn] = fv;
        T.flag[tn] = 1;
    }
    __syncwarp();
    return tn + 1;
}

// Band order: larger H first, then smaller k, k', s.
__device__ __forceinline__ bool dv_before(int32_t h1, int64_t k1, int64_t kp1, int64_t s1, int32_t h2, int64_t k2,
                                          int64_t kp2, int64_t s2) {
    if (h1 != h2) return h1 > h2;
    if (k1 != k2) return k1 < k2;
    if (kp1 != kp2) return kp1 < kp2;
    return s1 < s2;
}


}  // namespace dv
}  // namespace rb3
