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

template <class T> static int scan_impl(const T *in, T *out, int64_t n, bool inclusive, int op, cudaStream_t st) {
    if (n <= 0) return RB3_OK;
    int64_t ntiles = (n + SC_TILE - 1) / SC_TILE;
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
// order = (warp, iteration, lane) = input order).  Per pass:
//   hist    -- per-tile digit counts, digit-major [256][ntiles]
//   scan    -- exclusive prefix over that array = global digit offsets
//   scatter -- stable in-tile ranks by warp multi-split (__match_any_sync),
//              pairs reordered in shared memory, then written out in runs.
// The scatter holds only the keys and their ranks in registers; a pair's value
// is loaded after the tile's ranks are known and goes straight to its place in
// shared memory.  That keeps the kernel at three CTAs per SM.
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITERS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITERS;
constexpr int RS_BINS = 256;

template <class K>
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const K *__restrict__ keys, int64_t n, int shift,
                                                        uint32_t mask, uint32_t *__restrict__ counts,
                                                        int64_t ntiles) {
    __shared__ uint32_t h[RS_WARPS][RS_BINS];
    for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&h[0][0])[i] = 0;
    __syncthreads();
    int w = threadIdx.x >> 5;
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
        int64_t g = base + i;
        if (g < n) atomicAdd(&h[w][(uint32_t)(keys[g] >> shift) & mask], 1u);
    }
    __syncthreads();
    uint32_t t = 0;
#pragma unroll
    for (int j = 0; j < RS_WARPS; ++j) t += h[j][threadIdx.x];
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = t;
}

template <class K> struct RsSmem {
    K k[RS_TILE];
    uint32_t v[RS_TILE];
    uint32_t wh[RS_WARPS][RS_BINS];
    uint32_t dstart[RS_BINS];
    uint32_t goff[RS_BINS];
    uint32_t wtot[32];
};

template <class K>
__global__ void __launch_bounds__(RS_THREADS, 3) k_rs_scatter(const K *__restrict__ kin,
                                                              const uint32_t *__restrict__ vin,
                                                              K *__restrict__ kout, uint32_t *__restrict__ vout,
                                                              int64_t n, int shift, uint32_t mask,
                                                              const uint32_t *__restrict__ offs, int64_t ntiles) {
    extern __shared__ __align__(16) unsigned char smraw[];
    RsSmem<K> &S = *reinterpret_cast<RsSmem<K> *>(smraw);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&S.wh[0][0])[i] = 0;
    S.goff[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE + w * (RS_ITERS * 32);
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
    uint32_t tot = 0;
#pragma unroll
    for (int j = 0; j < RS_WARPS; ++j) {
        uint32_t c = S.wh[j][threadIdx.x];
        S.wh[j][threadIdx.x] = tot;
        tot += c;
    }
    uint32_t ds = block_excl<uint32_t>(tot, 0, S.wtot);
    S.dstart[threadIdx.x] = ds;
    __syncthreads();
#pragma unroll
    for (int it = 0; it < RS_ITERS; ++it) {
        int64_t g = base + it * 32 + lane;
        if (g < n) {
            uint32_t d = (uint32_t)(kk[it] >> shift) & mask;
            lr[it] += S.dstart[d] + S.wh[w][d];
            S.k[lr[it]] = kk[it];
        }
    }
    // values: loaded now, stored at their pair's place
#pragma unroll
    for (int it = 0; it < RS_ITERS; ++it) {
        int64_t g = base + it * 32 + lane;
        if (g < n) S.v[lr[it]] = vin[g];
    }
    __syncthreads();
    int64_t tb = (int64_t)blockIdx.x * RS_TILE;
    int cnt = (int)((n - tb) < RS_TILE ? (n - tb) : RS_TILE);
    for (int i = threadIdx.x; i < cnt; i += RS_THREADS) {
        K k = S.k[i];
        uint32_t d = (uint32_t)(k >> shift) & mask;
        int64_t gp = (int64_t)S.goff[d] + (i - (int64_t)S.dstart[d]);
        kout[gp] = k;
        vout[gp] = S.v[i];
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
    static const cudaError_t attr = cudaFuncSetAttribute(k_rs_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)sizeof(RsSmem<K>));  // once, thread-safe
    RB3_CUDA_TRY(attr);
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    DevBuf counts;
    RB3_TRY(counts.alloc(sizeof(uint32_t) * RS_BINS * ntiles, st));
    K *ka = k0, *kb = k1;
    uint32_t *va = v0, *vb = v1;
    bool alt = false;
    const double kv = (double)sizeof(K) + 4.0;
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
        int nb = end_bit - shift < 8 ? end_bit - shift : 8;
        uint32_t mask = (1u << nb) - 1u;
        {
            Phase ph("k.rs_hist", st, (double)sizeof(K) * n);  // reads the keys
            RB3_LAUNCH(k_rs_hist<K>, (unsigned)ntiles, RS_THREADS, 0, st, ka, n, shift, mask, counts.as<uint32_t>(),
                       ntiles);
        }
        RB3_TRY(scan_u32(counts.as<uint32_t>(), counts.as<uint32_t>(), RS_BINS * ntiles, false, 0, st));
        {
            Phase ph("k.rs_scatter", st, 2.0 * kv * n);  // reads and writes (key, 4-byte value)
            RB3_LAUNCH(k_rs_scatter<K>, (unsigned)ntiles, RS_THREADS, sizeof(RsSmem<K>), st, ka, va, kb, vb, n, shift,
                       mask, counts.as<uint32_t>(), ntiles);
        }
        K *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
        alt = !alt;
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

}  // namespace rb3
