// Algorithm 4 (FindSMEM1 / FindSMEM) over the extensions of Algorithm 3, for
// the starts of one query that lie in [x0, x1).  The way a found SMEM is
// handed on is a template parameter (appended under an atomic counter, counted,
// or written at a known offset); the search itself is the same for all.
#pragma once

#include "common.cuh"

namespace rb3 {

// Appends records under a global atomic counter; writes only below cap.
struct EmitAppend {
    rb3_smem *out;
    int64_t cap;
    unsigned long long *count;
    __device__ __forceinline__ void operator()(int64_t qid, int64_t st, int64_t en, const BiInt &x) const {
        unsigned long long at = atomicAdd(count, 1ull);
        if ((int64_t)at < cap) {
            rb3_smem r;
            r.qid = qid;
            r.start = (int32_t)st;
            r.end = (int32_t)en;
            r.k = x.k;
            r.kp = x.kp;
            r.s = x.s;
            out[at] = r;
        }
    }
};

// FindSMEM loop over starts in [x0, x1) of one query.
template <int NS, class Emit>
__device__ void smem_range(const OccView &V, const uint8_t *__restrict__ P, int64_t len, int64_t qid, int64_t x0,
                           int64_t x1, int ell, int64_t smin, Emit &emit) {
    int64_t i = x0;
    bool first = x0 > 0;
    while (i < x1) {
        if (i + ell > len) break;
        BiInt x = {0, 0, V.n};
        int64_t j;
        bool fail = false;
        for (j = i + ell - 1; j >= i; --j) {
            x = backward_ext<NS>(V, x, P[j]);
            if (x.s < smin) {
                fail = true;
                break;
            }
        }
        if (fail) {
            i = j + 1;
            first = false;
            continue;
        }
        for (j = i + ell; j < len; ++j) {
            BiInt y = forward_ext<NS>(V, x, P[j]);
            if (y.s < smin) break;
            x = y;
        }
        const int64_t e = j;
        bool keep = true;
        if (first) {  // i == x0 > 0: spurious if P[x0-1, e) still occurs >= smin times
            BiInt y = backward_ext<NS>(V, x, P[x0 - 1]);
            if (y.s >= smin) keep = false;
        }
        first = false;
        if (keep) emit(qid, i, e, x);
        if (e == len) break;
        BiInt z = {0, 0, V.n};
        int64_t nxt = i + 1;
        for (j = e; j >= i + 1; --j) {
            z = backward_ext<NS>(V, z, P[j]);
            if (z.s < smin) {
                nxt = j + 1;
                break;
            }
        }
        i = nxt;
    }
}

}  // namespace rb3
