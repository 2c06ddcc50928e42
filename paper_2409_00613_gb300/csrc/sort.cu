// Device-wide primitives used by the batch builder and the search output:
// reduce-then-scan prefix sums and a stable LSD radix sort of (uint64 or
// uint32 key, uint32 value) pairs.  Both are written for this library; no CUB.
#include "common.cuh"

namespace rb3 {

// ---------------------------------------------------------------------------
// Scan: tiles of 2048 elements (256 threads x 8).  A tile is staged through
// shared memory so global loads and stores stay coalesced.
// ---------------------------------------------------------------------------
constexpr int SC_ITEMS = 8;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

template <class T> __global__ void k_scan_reduce(const T *__restrict__ in, int64_t n, T *__restrict__ part, int op) {
    __shared__ T wtot[32];
    int64_t base = (int64_t)blockIdx.x * SC_TILE;
    T acc = 0;
    for (int i = threadIdx.x; i < SC_TILE; i += SC_THREADS) {
        int64_t g = base + i;
        if (g < n) acc = op2(acc, in[g], op);
    }
    // block reduce via inclusive warp scans
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = warp_incl(acc, op);
    if (lane == 31) wtot[w] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
        T t = 0;
        for (int j = 0; j < SC_THREADS / 32; ++j) t = op2(t, wtot[j], op);
        part[blockIdx.x] = t;
    }
}

__device__ __forceinline__ int pad_idx(int i) { return i + (i >> 5); }

template <class T>
__global__ void k_scan_apply(const T *__restrict__ in, T *__restrict__ out, int64_t n, const T *__restrict__ part,
                             int inclusive, int op) {
    __shared__ T s[SC_TILE + SC_TILE / 32];
    __shared__ T wtot[32];
    int64_t base = (int64_t)blockIdx.x * SC_TILE;
    for (int i = threadIdx.x; i < SC_TILE; i += SC_THREADS) {
        int64_t g = base + i;
        s[pad_idx(i)] = g < n ? in[g] : T(0);
    }
    __syncthreads();
    T v[SC_ITEMS];
    T run = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        v[j] = s[pad_idx(threadIdx.x * SC_ITEMS + j)];
        run = op2(run, v[j], op);
    }
    T ex = block_excl(run, op, wtot);
    T acc = op2(part ? part[blockIdx.x] : T(0), ex, op);
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        if (inclusive) {
            acc = op2(acc, v[j], op);
            s[pad_idx(threadIdx.x * SC_ITEMS + j)] = acc;
        } else {
            s[pad_idx(threadIdx.x * SC_ITEMS + j)] = acc;
            acc = op2(acc, v[j], op);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SC_TILE; i += SC_THREADS) {
        int64_t g = base + i;
        if (g < n) out[g] = s[pad_idx(i)];
    }
}

// Vector forms for 16-byte-aligned uint32 arrays, same tiles: the reduce reads
// each tile as 16-byte words (order does not matter for + and max); the apply
// gives thread t elements [8t, 8t + 8) of its tile straight from two 16-byte
// loads and writes them back the same way, without staging in shared memory.
__global__ void k_scan_reduce_v(const uint32_t *__restrict__ in, int64_t n, uint32_t *__restrict__ part, int op) {
    __shared__ uint32_t wtot[32];
    const int64_t base = (int64_t)blockIdx.x * SC_TILE;
    uint32_t acc = 0;
    if (base + SC_TILE <= n) {
        const uint4 *v = reinterpret_cast<const uint4 *>(in + base);
#pragma unroll
        for (int j = 0; j < SC_ITEMS / 4; ++j) {
            const uint4 x = __ldg(v + threadIdx.x + j * SC_THREADS);
            acc = op2(op2(acc, x.x, op), op2(op2(x.y, x.z, op), x.w, op), op);
        }
    } else {
        for (int i = threadIdx.x; i < SC_TILE; i += SC_THREADS)
            if (base + i < n) acc = op2(acc, in[base + i], op);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t inc = warp_incl(acc, op);
    if (lane == 31) wtot[w] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int j = 0; j < SC_THREADS / 32; ++j) t = op2(t, wtot[j], op);
        part[blockIdx.x] = t;
    }
}

__global__ void k_scan_apply_v(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int64_t n,
                               const uint32_t *__restrict__ part, int inclusive, int op) {
    __shared__ uint32_t wtot[32];
    const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
    uint32_t v[SC_ITEMS];
    const bool full = base + SC_ITEMS <= n;
    if (full) {
        const uint4 a = __ldg(reinterpret_cast<const uint4 *>(in + base));
        const uint4 b = __ldg(reinterpret_cast<const uint4 *>(in + base) + 1);
        v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
    } else {
#pragma unroll
        for (int j = 0; j < SC_ITEMS; ++j) v[j] = base + j < n ? in[base + j] : 0u;
    }
    uint32_t run = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) run = op2(run, v[j], op);
    const uint32_t ex = block_excl(run, op, wtot);
    uint32_t acc = op2(part ? part[blockIdx.x] : 0u, ex, op);
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        const uint32_t x = v[j];
        if (inclusive) {
            acc = op2(acc, x, op);
            v[j] = acc;
        } else {
            v[j] = acc;
            acc = op2(acc, x, op);
        }
    }
    if (full) {
        uint4 *o = reinterpret_cast<uint4 *>(out + base);
        o[0] = make_uint4(v[0], v[1], v[2], v[3]);
        o[1] = make_uint4(v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
        for (int j = 0; j < SC_ITEMS; ++j)
            if (base + j < n) out[base + j] = v[j];
    }
}

template <class T> static int scan_impl(const T *in, T *out, int64_t n, bool inclusive, int op, cudaStream_t st) {
    if (n <= 0) return RB3_OK;
    int64_t ntiles = (n + SC_TILE - 1) / SC_TILE;
    if constexpr (sizeof(T) == 4) {
        if (ntiles > 1 && ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0) {
            DevBuf part;
            RB3_TRY(part.alloc(sizeof(T) * ntiles, st));
            const uint32_t *vin = reinterpret_cast<const uint32_t *>(in);
            uint32_t *vout = reinterpret_cast<uint32_t *>(out), *vp = part.as<uint32_t>();
            RB3_LAUNCH(k_scan_reduce_v, (unsigned)ntiles, SC_THREADS, 0, st, vin, n, vp, op);
            RB3_TRY(scan_impl<T>(part.as<T>(), part.as<T>(), ntiles, false, op, st));
            RB3_LAUNCH(k_scan_apply_v, (unsigned)ntiles, SC_THREADS, 0, st, vin, vout, n, (const uint32_t *)vp,
                       (int)inclusive, op);
            return RB3_OK;
        }
    }
    if (ntiles == 1) {
        RB3_LAUNCH(k_scan_apply<T>, 1, SC_THREADS, 0, st, in, out, n, (const T *)nullptr, (int)inclusive, op);
        return RB3_OK;
    }
    DevBuf part;
    RB3_TRY(part.alloc(sizeof(T) * ntiles, st));
    RB3_LAUNCH(k_scan_reduce<T>, (unsigned)ntiles, SC_THREADS, 0, st, in, n, part.as<T>(), op);
    RB3_TRY(scan_impl<T>(part.as<T>(), part.as<T>(), ntiles, false, op, st));
    RB3_LAUNCH(k_scan_apply<T>, (unsigned)ntiles, SC_THREADS, 0, st, in, out, n, (const T *)part.as<T>(),
               (int)inclusive, op);
    return RB3_OK;
}

int scan_u32(const uint32_t *in, uint32_t *out, int64_t n, bool inclusive, int op, cudaStream_t st) {
    return scan_impl<uint32_t>(in, out, n, inclusive, op, st);
}
// Sum scan whose tile partials go to a caller-provided workspace instead of a
// fresh allocation: n <= SC_TILE * SC_TILE and part_cap >= ceil(n / SC_TILE).
int scan_u32_ws(const uint32_t *in, uint32_t *out, int64_t n, bool inclusive, uint32_t *part_ws, int64_t part_cap,
                cudaStream_t st) {
    if (n <= 0) return RB3_OK;
    int64_t ntiles = (n + SC_TILE - 1) / SC_TILE;
    if (ntiles == 1) {
        RB3_LAUNCH(k_scan_apply<uint32_t>, 1, SC_THREADS, 0, st, in, out, n, (const uint32_t *)nullptr, (int)inclusive,
                   0);
        return RB3_OK;
    }
    if (ntiles > SC_TILE || ntiles > part_cap) {
        set_error("scan workspace too small (%lld tiles)", (long long)ntiles);
        return RB3_E_INVAL;
    }
    RB3_LAUNCH(k_scan_reduce<uint32_t>, (unsigned)ntiles, SC_THREADS, 0, st, in, n, part_ws, 0);
    RB3_LAUNCH(k_scan_apply<uint32_t>, 1, SC_THREADS, 0, st, part_ws, part_ws, ntiles, (const uint32_t *)nullptr, 0,
               0);
    RB3_LAUNCH(k_scan_apply<uint32_t>, (unsigned)ntiles, SC_THREADS, 0, st, in, out, n, (const uint32_t *)part_ws,
               (int)inclusive, 0);
    return RB3_OK;
}

int scan_u64(const uint64_t *in, uint64_t *out, int64_t n, bool inclusive, cudaStream_t st) {
    return scan_impl<unsigned long long>(reinterpret_cast<const unsigned long long *>(in),
                                         reinterpret_cast<unsigned long long *>(out), n, inclusive, 0, st);
}

// ---------------------------------------------------------------------------
// Radix sort: 8-bit digits, tiles of 4096 pairs (warp w takes items
// [512w, 512w + 512) of the tile, lane-interleaved over 16 iterations, so item
// order = (warp, iteration, lane) = input order).  One pass over the keys
// counts the digits of every pass (a digit's global count does not depend on
// the order); then each pass is one kernel: a tile takes the next tile number
// from a counter, ranks its pairs by warp multi-split (__match_any_sync),
// publishes its digit counts, adds up the counts of the tiles before it
// (decoupled look-back: a tile's flag is either its own count or the count of
// everything up to it), and writes its pairs out in runs through shared
// memory.  A tile only waits for tiles that took their numbers before it, so
// they are running or done; every wait has an iteration limit, after which
// the tile records an error (read by the host after the sort).
// The keys stay in registers with their ranks; a pair's value is loaded after
// the tile's ranks are known and goes straight to its place in shared memory.
// Tile shape: RS_ITERS keys per thread, RS_MINB CTAs per SM asked of the
// register allocator; with RS_ALIAS the values reuse the keys' shared-memory
// staging after the keys are written out (a one-byte digit per pair kept for
// their places).  Default 16 / 4 / aliased: 64 registers and 46 KB, four CTAs
// per SM (against three with separate staging at 80 registers and 58 KB:
// 22 % less time per pass on the pangenome builds).
// ---------------------------------------------------------------------------
#ifndef RB3_RS_ITERS
#define RB3_RS_ITERS 16
#endif
#ifndef RB3_RS_MINB
#define RB3_RS_MINB 4
#endif
#ifndef RB3_RS_ALIAS
#define RB3_RS_ALIAS 1
#endif
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITERS = RB3_RS_ITERS;
constexpr int RS_MINB = RB3_RS_MINB;
constexpr bool RS_ALIAS = RB3_RS_ALIAS != 0;
constexpr int RS_TILE = RS_THREADS * RS_ITERS;
constexpr int RS_BINS = 256;
constexpr int RS_MAXPASS = 8;
constexpr uint64_t RS_AGG = 1ull << 62, RS_INC = 2ull << 62, RS_VAL = (1ull << 62) - 1;
constexpr int RS_SPIN_LIMIT = 1 << 22;

template <class K>
__global__ void __launch_bounds__(RS_THREADS) k_rs_allhist(const K *__restrict__ keys, int64_t n, int begin_bit,
                                                           int end_bit, uint32_t *__restrict__ counts) {
    __shared__ uint32_t h[RS_MAXPASS][RS_BINS];
    const int npass = (end_bit - begin_bit + 7) / 8;
    for (int i = threadIdx.x; i < RS_MAXPASS * RS_BINS; i += RS_THREADS) (&h[0][0])[i] = 0;
    __syncthreads();
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const K k = keys[g];
        for (int p = 0; p < npass; ++p) {
            const int sh = begin_bit + 8 * p;
            const int nb = end_bit - sh < 8 ? end_bit - sh : 8;
            atomicAdd(&h[p][(uint32_t)(k >> sh) & ((1u << nb) - 1u)], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npass * RS_BINS; i += RS_THREADS) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&counts[i], c);
    }
}

// base[p][d] = number of keys whose digit p is below d (one block per pass).
__global__ void k_rs_bases(const uint32_t *__restrict__ counts, uint32_t *__restrict__ base) {
    __shared__ uint32_t wtot[32];
    const int p = blockIdx.x;
    base[p * RS_BINS + threadIdx.x] = block_excl<uint32_t>(counts[p * RS_BINS + threadIdx.x], 0, wtot);
}

__device__ __forceinline__ void rs_flag_store(uint64_t *p, uint64_t v) {
    asm volatile("st.volatile.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t rs_flag_load(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Bounded wait for a tile's look-back flag: polls until its status bits are
// set or `limit` polls have passed; a time-out is recorded in err (read by the
// host after the launch, reported as RB3_E_TIMEOUT) and an empty inclusive
// flag is returned, so the tile finishes and the context stays usable.
__device__ __forceinline__ uint64_t rs_wait_flag(const uint64_t *G, int limit, unsigned int *err) {
    uint64_t v = rs_flag_load(G);
    int spins = 0;
    while ((v >> 62) == 0) {
        if (++spins > limit) {
            atomicOr(err, 1u);
            return RS_INC;
        }
        __nanosleep(32);
        v = rs_flag_load(G);
    }
    return v;
}

// Self-test of the bounded wait: one thread waits on a flag that nothing sets.
__global__ void k_wait_selftest(const uint64_t *flag, int limit, unsigned int *err) {
    if (blockIdx.x == 0 && threadIdx.x == 0) rs_wait_flag(flag, limit, err);
}

template <class K, bool ALIAS> struct RsStage {
    K k[RS_TILE];
    uint32_t v[RS_TILE];
};
template <class K> struct RsStage<K, true> {
    union {
        K k[RS_TILE];
        uint32_t v[RS_TILE];
    };
    uint8_t dg[RS_TILE];
};
template <class K> struct RsSmem : RsStage<K, RS_ALIAS> {
    uint32_t wh[RS_WARPS][RS_BINS];
    uint32_t dstart[RS_BINS];
    uint32_t goff[RS_BINS];
    uint32_t wtot[32];
    uint32_t tile;
};

template <class K>
__global__ void __launch_bounds__(RS_THREADS, RS_MINB) k_rs_onesweep(const K *__restrict__ kin,
                                                               const uint32_t *__restrict__ vin,
                                                               K *__restrict__ kout, uint32_t *__restrict__ vout,
                                                               int64_t n, int shift, uint32_t mask,
                                                               const uint32_t *__restrict__ dbase,
                                                               unsigned int *__restrict__ tile_ctr,
                                                               uint64_t *__restrict__ flags,
                                                               unsigned int *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smraw[];
    RsSmem<K> &S = *reinterpret_cast<RsSmem<K> *>(smraw);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&S.wh[0][0])[i] = 0;
    if (threadIdx.x == 0) S.tile = atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const int64_t t = S.tile;
    const int64_t tb = t * RS_TILE;
    int64_t base = tb + w * (RS_ITERS * 32);
    unsigned lt = (1u << lane) - 1u;
    K kk[RS_ITERS];
    uint32_t lr[RS_ITERS];
    // the whole tile's keys are loaded before any is ranked
#pragma unroll
    for (int it = 0; it < RS_ITERS; ++it) {
        int64_t g = base + it * 32 + lane;
        kk[it] = g < n ? kin[g] : K(0);
    }
#pragma unroll
    for (int it = 0; it < RS_ITERS; ++it) {
        int64_t g = base + it * 32 + lane;
        bool valid = g < n;
        K k = kk[it];
        uint32_t d = valid ? ((uint32_t)(k >> shift) & mask) : (RS_BINS + lane);
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int leader = 31 - __clz(peers);
        uint32_t c0 = valid ? S.wh[w][d] : 0u;
        __syncwarp();
        if (valid && lane == leader) S.wh[w][d] = c0 + __popc(peers);
        __syncwarp();
        lr[it] = c0 + __popc(peers & lt);
    }
    __syncthreads();
    // per digit (thread = digit): warp-exclusive offsets and tile total
    const int d = threadIdx.x;
    uint32_t tot = 0;
#pragma unroll
    for (int j = 0; j < RS_WARPS; ++j) {
        uint32_t c = S.wh[j][d];
        S.wh[j][d] = tot;
        tot += c;
    }
    // publish, look back over the tiles before this one, publish the inclusive count
    uint64_t *F = flags + t * RS_BINS + d;
    uint64_t excl = 0;
    if (t == 0) {
        rs_flag_store(F, RS_INC | tot);
    } else {
        rs_flag_store(F, RS_AGG | tot);
        for (int64_t tt = t - 1; tt >= 0; --tt) {
            const uint64_t v = rs_wait_flag(flags + tt * RS_BINS + d, RS_SPIN_LIMIT, err);
            excl += v & RS_VAL;
            if ((v >> 62) == 2) break;
        }
        rs_flag_store(F, RS_INC | (excl + tot));
    }
    S.goff[d] = dbase[d] + (uint32_t)excl;
    uint32_t ds = block_excl<uint32_t>(tot, 0, S.wtot);
    S.dstart[d] = ds;
    __syncthreads();
#pragma unroll
    for (int it = 0; it < RS_ITERS; ++it) {
        int64_t g = base + it * 32 + lane;
        if (g < n) {
            uint32_t dd = (uint32_t)(kk[it] >> shift) & mask;
            lr[it] += S.dstart[dd] + S.wh[w][dd];
            S.k[lr[it]] = kk[it];
        }
    }
    const int cnt = (int)((n - tb) < RS_TILE ? (n - tb) : RS_TILE);
    if constexpr (RS_ALIAS) {
        uint32_t vv[RS_ITERS];  // values requested before the keys go out
#pragma unroll
        for (int it = 0; it < RS_ITERS; ++it) {
            int64_t g = base + it * 32 + lane;
            vv[it] = g < n ? vin[g] : 0u;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += RS_THREADS) {
            K k = S.k[i];
            uint32_t dd = (uint32_t)(k >> shift) & mask;
            S.dg[i] = (uint8_t)dd;
            kout[(int64_t)S.goff[dd] + (i - (int64_t)S.dstart[dd])] = k;
        }
        __syncthreads();  // the keys' staging is free: the values take it
#pragma unroll
        for (int it = 0; it < RS_ITERS; ++it) {
            int64_t g = base + it * 32 + lane;
            if (g < n) S.v[lr[it]] = vv[it];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += RS_THREADS) {
            const uint32_t dd = S.dg[i];
            vout[(int64_t)S.goff[dd] + (i - (int64_t)S.dstart[dd])] = S.v[i];
        }
    } else {
        // values: loaded now, stored at their pair's place
#pragma unroll
        for (int it = 0; it < RS_ITERS; ++it) {
            int64_t g = base + it * 32 + lane;
            if (g < n) S.v[lr[it]] = vin[g];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += RS_THREADS) {
            K k = S.k[i];
            uint32_t dd = (uint32_t)(k >> shift) & mask;
            int64_t gp = (int64_t)S.goff[dd] + (i - (int64_t)S.dstart[dd]);
            kout[gp] = k;
            vout[gp] = S.v[i];
        }
    }
}

template <class K>
static int radix_sort_impl(K *k0, uint32_t *v0, K *k1, uint32_t *v1, int64_t n, int begin_bit, int end_bit,
                           cudaStream_t st, bool *in_alt) {
    *in_alt = false;
    if (n <= 1 || end_bit <= begin_bit) return RB3_OK;
    if (n > 0xFFFFFFFFll) {
        set_error("radix sort: too many elements (%lld)", (long long)n);
        return RB3_E_INVAL;
    }
    const int npass = (end_bit - begin_bit + 7) / 8;
    if (npass > RS_MAXPASS) {
        set_error("radix sort: %d key bits", end_bit - begin_bit);
        return RB3_E_INVAL;
    }
    static const cudaError_t attr = cudaFuncSetAttribute(k_rs_onesweep<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)sizeof(RsSmem<K>));  // once, thread-safe
    RB3_CUDA_TRY(attr);
    const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    // one buffer: digit counts and bases of every pass, tile counters, error flag, look-back flags
    const size_t head = sizeof(uint32_t) * (2 * RS_MAXPASS * RS_BINS + RS_MAXPASS + 2);
    const size_t head_al = (head + 255) & ~size_t(255);
    DevBuf work;
    RB3_TRY(work.alloc(head_al + sizeof(uint64_t) * RS_BINS * ntiles, st));
    uint32_t *counts = work.as<uint32_t>(), *bases = counts + RS_MAXPASS * RS_BINS;
    unsigned int *ctr = bases + RS_MAXPASS * RS_BINS, *err = ctr + RS_MAXPASS;
    uint64_t *flags = reinterpret_cast<uint64_t *>(work.as<uint8_t>() + head_al);
    RB3_CUDA_TRY(cudaMemsetAsync(work.p, 0, head, st));
    {
        Phase ph("k.rs_hist", st, (double)sizeof(K) * n);  // reads the keys once for every pass
        unsigned grid = (unsigned)((n + RS_THREADS * 16 - 1) / (RS_THREADS * 16));
        if (grid > (unsigned)num_sms() * 8) grid = (unsigned)num_sms() * 8;
        RB3_LAUNCH(k_rs_allhist<K>, grid, RS_THREADS, 0, st, k0, n, begin_bit, end_bit, counts);
        RB3_LAUNCH(k_rs_bases, (unsigned)npass, RS_BINS, 0, st, counts, bases);
    }
    K *ka = k0, *kb = k1;
    uint32_t *va = v0, *vb = v1;
    bool alt = false;
    const double kv = (double)sizeof(K) + 4.0;
    for (int p = 0; p < npass; ++p) {
        const int shift = begin_bit + 8 * p;
        const int nb = end_bit - shift < 8 ? end_bit - shift : 8;
        const uint32_t mask = (1u << nb) - 1u;
        RB3_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(uint64_t) * RS_BINS * ntiles, st));
        {
            Phase ph("k.rs_scatter", st, 2.0 * kv * n);  // reads and writes (key, 4-byte value)
            RB3_LAUNCH(k_rs_onesweep<K>, (unsigned)ntiles, RS_THREADS, sizeof(RsSmem<K>), st, ka, va, kb, vb, n,
                       shift, mask, bases + p * RS_BINS, ctr + p, flags, err);
        }
        K *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
        alt = !alt;
    }
    unsigned int herr = 0;
    RB3_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr) {
        set_error("radix sort: a tile gave up waiting for the counts of the tiles before it");
        return RB3_E_TIMEOUT;
    }
    *in_alt = alt;
    return RB3_OK;
}

int radix_sort_pairs(uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1, int64_t n, int begin_bit, int end_bit,
                     cudaStream_t st, bool *in_alt) {
    return radix_sort_impl<unsigned long long>(reinterpret_cast<unsigned long long *>(k0), v0,
                                               reinterpret_cast<unsigned long long *>(k1), v1, n, begin_bit, end_bit,
                                               st, in_alt);
}

int radix_sort_pairs32(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, int64_t n, int begin_bit, int end_bit,
                       cudaStream_t st, bool *in_alt) {
    return radix_sort_impl<uint32_t>(k0, v0, k1, v1, n, begin_bit, end_bit, st, in_alt);
}

int wait_selftest(int limit, cudaStream_t st) {
    DevBuf buf;
    RB3_TRY(buf.alloc(16, st));
    RB3_CUDA_TRY(cudaMemsetAsync(buf.p, 0, 16, st));
    unsigned int *err = reinterpret_cast<unsigned int *>(buf.as<uint8_t>() + 8);
    RB3_LAUNCH(k_wait_selftest, 1, 32, 0, st, buf.as<uint64_t>(), limit, err);
    unsigned int h = 0;
    RB3_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(h), cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    if (h) {
        set_error("bounded wait gave up after %d polls (self-test: nothing sets the flag)", limit);
        return RB3_E_TIMEOUT;
    }
    return RB3_OK;
}

}  // namespace rb3
