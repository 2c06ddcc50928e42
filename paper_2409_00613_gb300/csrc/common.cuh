// Shared internals of librb3: the index object, error / launch / profiling
// plumbing, stream-ordered scratch buffers and the device-side rank core.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/rb3.h"

#define RB3_EXPORT extern "C" __attribute__((visibility("default")))

// ---------------------------------------------------------------------------
// The index.  Blocks of D symbols, nblocks = n/D + 1 so that rank(a, n) reads a
// block that exists.
//  D = 64, 128, 256: 32-byte header (rank of each symbol at the block start:
//    uint32 low words at bytes 0..23, uint8 high bytes at 24..29), then D/2
//    payload bytes: one 32-byte sector per 64 symbols holding their codes as
//    four 64-bit bit-planes.
//  D = 32: one 32-byte sector per block, so that a rank is one memory request:
//    uint32 words 0..4 = rank of A, C, G, T, N at the block start minus that
//    symbol's rank at the start of the block's 2^32-symbol span (gbase; zero
//    below 2^32), words 5..7 = the three 32-bit bit-planes of the block's
//    symbols.  rank($, l) = l minus the other five ranks.
//  Run-length layout (rle = 1, made from a finished index by
//    rb3_index_compress, read-only): D = S symbols per span, `blocks` holds one
//    64-byte header per span (ranks at the span start, where its runs begin,
//    two decode marks) and `payload` the runs, cut at span boundaries (format
//    at NS_RLE below).
// ---------------------------------------------------------------------------
struct rb3_index {
    int64_t n = 0, m = 0;
    int64_t C[7] = {0, 0, 0, 0, 0, 0, 0};
    int32_t D = 64, log2D = 6, block_bytes = 64;
    int32_t single_strand = 0;
    int64_t nblocks = 0;
    uint8_t *blocks = nullptr;  // device
    // D = 32 and n >= 2^32 only: gbase[5 g + a - 1] = rank(a, g * 2^32), a = 1..5,
    // g = 0 .. n >> 32 (device; null otherwise)
    int64_t *gbase = nullptr;
    // sampled suffix array (optional): a row is sampled when its suffix starts at
    // an offset of its string that is a multiple of sa_s.  sdir holds, per 64
    // rows, {bit set of sampled rows, number of sampled rows before them}; svals
    // the sampled rows' (string << 40 | offset), in row order.
    int32_t sa_s = 0;
    int64_t n_samples = 0;
    uint64_t *sdir = nullptr;   // device, 2 * (n / 64 + 1) words
    uint64_t *svals = nullptr;  // device, n_samples
    // run-length layout: the runs of every span (device, payload_bytes + 16 bytes
    // of padding, so that the decoder's 8-byte reads stay inside)
    int32_t rle = 0;
    uint8_t *payload = nullptr;
    int64_t payload_bytes = 0, runs = 0;
    // build data of a batch (optional): its text and inverse suffix array
    uint8_t *text = nullptr;   // device, n codes (0 = sentinel)
    int32_t *isa = nullptr;    // device, n entries
    std::vector<int64_t> str_end;  // host: position of the sentinel ending DS string i
    int device = 0;
    // hot-level table of the SMEM search (device, built on first use by
    // rb3::hot_table and owned here): the bi-intervals of every A/C/G/T string
    // of length 1..hot_k, valid while n and the rank arrays are those it was
    // built from (hot_n, hot_src).  A table replaced by a deeper one stays in
    // hot_old until the index is freed (a search on another stream may still
    // read it).
    mutable void *hot = nullptr;
    mutable int32_t hot_k = 0;
    mutable int64_t hot_n = -1;
    mutable const void *hot_src = nullptr;
    mutable std::vector<void *> hot_old;
};

namespace rb3 {

constexpr int SIGMA = 6;
constexpr int HEADER_BYTES = 32;
constexpr int GSPAN_LOG2 = 32;  // D = 32 counts are relative to spans of 2^32 symbols

constexpr int kDefaultOccInterval = 32;  // one sector per rank
inline bool valid_occ_interval(int D) { return D == 32 || D == 64 || D == 128 || D == 256; }
// Run-length spans: a power of two from 512 (above every plain D, so that D alone
// tells the layouts apart) to 16384 (in-span offsets and ranks fit 16 bits).
inline bool valid_rle_span(int S) { return S >= 512 && S <= 16384 && (S & (S - 1)) == 0; }
constexpr int kDefaultRleSpan = 2048;
inline int block_bytes_for(int D) { return D == 32 ? 32 : HEADER_BYTES + D / 2; }
inline int64_t gbase_rows(int64_t n) { return (n >> GSPAN_LOG2) + 1; }

// ---- errors ---------------------------------------------------------------
void set_error(const char *fmt, ...);
std::string rb3_last_error_str();  // this thread's message
int cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define RB3_CUDA_TRY(expr)                                                       \
    do {                                                                         \
        cudaError_t e_ = (expr);                                                 \
        if (e_ != cudaSuccess) return rb3::cuda_fail(e_, #expr, __FILE__, __LINE__); \
    } while (0)

#define RB3_TRY(expr)                 \
    do {                              \
        int s_ = (expr);              \
        if (s_ != RB3_OK) return s_;  \
    } while (0)

#define RB3_CHECK_ARG(cond, msg)                          \
    do {                                                  \
        if (!(cond)) {                                    \
            rb3::set_error("invalid argument: %s", msg);  \
            return RB3_E_INVAL;                           \
        }                                                 \
    } while (0)

// ---- launches -------------------------------------------------------------
extern std::atomic<int64_t> g_launches;

#define RB3_LAUNCH(kern, grid, block, smem, stream, ...)                                  \
    do {                                                                                  \
        kern<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                         \
        rb3::g_launches.fetch_add(1, std::memory_order_relaxed);                          \
        cudaError_t e_ = cudaPeekAtLastError();                                           \
        if (e_ != cudaSuccess) return rb3::cuda_fail(e_, #kern, __FILE__, __LINE__);      \
    } while (0)

// ---- profiling: per-phase CUDA events on the caller's stream ---------------
// A phase may carry the algorithmic bytes its kernel moves (for the roofline).
bool profile_on();
void profile_push(const char *name, cudaEvent_t a, cudaEvent_t b, double bytes);

struct Phase {
    const char *name;
    cudaStream_t st;
    double bytes;
    cudaEvent_t a = nullptr, b = nullptr;
    Phase(const char *nm, cudaStream_t s, double algo_bytes = 0.0) : name(nm), st(s), bytes(algo_bytes) {
        if (profile_on() && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
            cudaEventRecord(a, st);
        else
            a = b = nullptr;
    }
    ~Phase() {
        if (a) {
            cudaEventRecord(b, st);
            profile_push(name, a, b, bytes);
        }
    }
};

// ---- stream-ordered device buffers ------------------------------------------
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFreeAsync(p, st);
        p = nullptr;
        bytes = 0;
    }
    int alloc(size_t nbytes, cudaStream_t s);
    template <class T> T *as() const { return static_cast<T *>(p); }
    void *detach() {
        void *q = p;
        p = nullptr;
        bytes = 0;
        return q;
    }
};

int dev_alloc(void **p, size_t bytes, cudaStream_t st);
void dev_free(void *p, cudaStream_t st);

// Pointer kind: true if the CUDA runtime knows it as device (or managed) memory.
bool is_device_ptr(const void *p);

// ---- device helpers -------------------------------------------------------
__host__ __device__ __forceinline__ int comp_sym(int a) {
    // Watson-Crick complement of $,A,C,G,T,N = $,T,G,C,A,N
    return (a >= 1 && a <= 4) ? 5 - a : a;
}

// Read-only view of an index for kernels (passed by value).
struct OccView {
    const uint8_t *__restrict__ blocks;
    const int64_t *__restrict__ gbase;  // D = 32 / run-length above 2^32 symbols, else null
    const uint8_t *__restrict__ payload;  // run-length layout only, else null
    int64_t n;
    int64_t C[7];
    int32_t log2D;
    int32_t bb;  // bytes per block
};

inline OccView occ_view(const rb3_index *x) {
    OccView v;
    v.blocks = x->blocks;
    v.gbase = x->gbase;
    v.payload = x->rle ? x->payload : nullptr;
    v.n = x->n;
    for (int i = 0; i < 7; ++i) v.C[i] = x->C[i];
    v.log2D = x->log2D;
    v.bb = x->block_bytes;
    return v;
}

__device__ __forceinline__ uint64_t ldg_u64(const uint8_t *p) {
    return __ldg(reinterpret_cast<const unsigned long long *>(p));
}

// One 32-byte sector in a single 256-bit load (read-only path).  Occ blocks are
// 32-byte aligned: block sizes are 32, 64, 96 or 160 bytes from a 256-aligned base.
struct Sec {
    uint32_t w[8];
};
__device__ __forceinline__ Sec ld_sec(const uint8_t *p) {
    Sec s;
    asm("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(s.w[0]), "=r"(s.w[1]), "=r"(s.w[2]), "=r"(s.w[3]), "=r"(s.w[4]), "=r"(s.w[5]), "=r"(s.w[6]),
          "=r"(s.w[7])
        : "l"(p));
    return s;
}

// The same load with a 64-byte L2 fetch-size hint: on a miss L2 asks DRAM for
// the 64-byte half-line holding the sector instead of the whole 128-byte line
// (measured: half the DRAM bytes per random sector read, same request rate).
// Every rank's block reads use it: they are random.
// RB3_RANK_HINT64 = 0 drops the hint (a measurement knob: with anchored merge
// segments the walk alone is ~5 % faster without it, the overlapped
// build-and-merge step ~1 % slower).
#ifndef RB3_RANK_HINT64
#define RB3_RANK_HINT64 1
#endif
__device__ __forceinline__ Sec ld_sec64(const uint8_t *p) {
#if !RB3_RANK_HINT64
    return ld_sec(p);
#endif
    Sec s;
    asm("ld.global.nc.L2::64B.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(s.w[0]), "=r"(s.w[1]), "=r"(s.w[2]), "=r"(s.w[3]), "=r"(s.w[4]), "=r"(s.w[5]), "=r"(s.w[6]),
          "=r"(s.w[7])
        : "l"(p));
    return s;
}

// Payload layout: every 64 symbols of a block form one 32-byte sector holding
// their 4-bit codes as four 64-bit bit-planes: plane b (bytes 8b..8b+7) has bit
// o set iff bit b of the code of symbol o is set.  Codes are 0..5, so plane 3
// is always zero.  A symbol's rank inside a sector is then a popcount of the
// AND of three (possibly complemented) planes under a prefix mask.
__device__ __forceinline__ uint64_t sec_plane(const Sec &s, int b) {
    return (uint64_t)s.w[2 * b] | ((uint64_t)s.w[2 * b + 1] << 32);
}

__device__ __forceinline__ uint64_t prefix_mask(int k) {  // bits [0, k), k may be <= 0 or >= 64
    return k >= 64 ? ~0ull : (k <= 0 ? 0ull : ((1ull << k) - 1ull));
}

// Number of symbols equal to c among the first k symbols (0..64) of a sector.
__device__ __forceinline__ int sec_count(const Sec &s, int c, int k) {
    const uint64_t p0 = sec_plane(s, 0), p1 = sec_plane(s, 1), p2 = sec_plane(s, 2);
    const uint64_t m = ((c & 1) ? p0 : ~p0) & ((c & 2) ? p1 : ~p1) & ((c & 4) ? p2 : ~p2);
    return __popcll(m & prefix_mask(k));
}

// Counts of every symbol among the first k symbols of a sector, added to r[].
__device__ __forceinline__ void sec_count_all(const Sec &s, int k, int64_t r[6]) {
    const uint64_t mk = prefix_mask(k);
    const uint64_t p0 = sec_plane(s, 0), p1 = sec_plane(s, 1), p2 = sec_plane(s, 2);
    const uint64_t b0 = p0 & mk, n0 = ~p0 & mk;
    const uint64_t t00 = ~p1 & ~p2, t10 = p1 & ~p2, t01 = ~p1 & p2;
    r[0] += __popcll(n0 & t00);
    r[1] += __popcll(b0 & t00);
    r[2] += __popcll(n0 & t10);
    r[3] += __popcll(b0 & t10);
    r[4] += __popcll(n0 & t01);
    r[5] += __popcll(b0 & t01);
}

// Header value of symbol c (registers only: the select is unrolled).
__device__ __forceinline__ int64_t hdr_get(const Sec &h, int c) {
    uint32_t lo = h.w[0], hib = h.w[6] & 0xFFu;
#pragma unroll
    for (int a = 1; a < 6; ++a)
        if (c == a) {
            lo = h.w[a];
            hib = (a < 4 ? (h.w[6] >> (8 * a)) : (h.w[7] >> (8 * (a - 4)))) & 0xFFu;
        }
    return (int64_t)lo | ((int64_t)hib << 32);
}

__device__ __forceinline__ void hdr_all(const Sec &h, int64_t r[6]) {
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        uint32_t hib = (a < 4 ? (h.w[6] >> (8 * a)) : (h.w[7] >> (8 * (a - 4)))) & 0xFFu;
        r[a] = (int64_t)h.w[a] | ((int64_t)hib << 32);
    }
}

// ---- run-length layout -------------------------------------------------------
// A run is one byte (symbol << 5 | f) and, for long runs, one or two length
// bytes: f < 30: length f + 1; f = 30: length 31 + the next byte; f = 31:
// length 287 + the next two bytes (little-endian).  Spans are at most 16384
// symbols, so every run fits and a span's runs take under 64 KiB.
//
// Span header, 64 bytes (two sectors, read as one 64-byte request):
//   uint32 w[0..4]  rank of A..N at the span start, minus the gbase of its
//                   2^32-symbol range (as for D = 32)
//   uint32 w[5..6]  byte offset of the span's runs in the payload (low, high)
//   uint32 w[7]     number of runs in the span
//   bytes 32..63    two decode marks, 16 bytes each: uint16 pos (offset in
//                   the span of the first symbol of a run), uint16 ranks of
//                   A..N from the span start to pos, uint32 byte offset of
//                   that run from the span's first run byte.  Mark j is the
//                   run holding offset (j + 1) * len / 3 of a span of len
//                   symbols (pos 0 for an empty span), so a rank decodes at
//                   most about a third of the span.
constexpr int NS_RLE = -1;  // compile-time layout tag next to NS = D / 64
constexpr int RLE_F1 = 30, RLE_F2 = 31;
constexpr int RLE_BASE1 = 31, RLE_BASE2 = 287;
constexpr int RLE_HDR_BYTES = 64;
constexpr int RLE_MARKS = 2;

__host__ __device__ __forceinline__ int rle_run_bytes(int64_t len) {
    return len < RLE_BASE1 ? 1 : (len < RLE_BASE2 ? 2 : 3);
}

// Sequential reader of a span's runs: aligned 8-byte loads, consumed a byte at
// a time (the payload is padded so that the last word read is inside it).
struct RunRd {
    const unsigned long long *w;
    uint64_t cur;
    int avail;
    __device__ __forceinline__ void init(const uint8_t *p) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(p);
        w = reinterpret_cast<const unsigned long long *>(a & ~(uintptr_t)7);
        const int sk = (int)(a & 7);
        cur = __ldg(w) >> (8 * sk);
        avail = 8 - sk;
    }
    __device__ __forceinline__ uint32_t byte() {
        if (avail == 0) {
            cur = __ldg(++w);
            avail = 8;
        }
        const uint32_t b = (uint32_t)(cur & 0xFFu);
        cur >>= 8;
        --avail;
        return b;
    }
    __device__ __forceinline__ void run(int *sym, int64_t *len) {
        const uint32_t b = byte(), f = b & 31u;
        *sym = (int)(b >> 5);
        if (f < (uint32_t)RLE_F1) {
            *len = (int64_t)f + 1;
        } else if (f == (uint32_t)RLE_F1) {
            *len = RLE_BASE1 + (int64_t)byte();
        } else {
            const uint32_t lo = byte();
            *len = RLE_BASE2 + (int64_t)(lo | (byte() << 8));
        }
    }
};

// Ranks inside a span (each below 2^16) packed three to a word, 21 bits each:
// acc[0] holds A, C, G; acc[1] T, N.  $ is never counted (rank($) = l minus
// the others).
__device__ __forceinline__ void rle_acc_add(uint64_t acc[2], int a, int64_t t) {
    const bool hi = a >= 4;
    const int sh = 21 * (hi ? a - 4 : a - 1);
    if (a != 0) {
        if (hi) acc[1] += (uint64_t)t << sh;
        else acc[0] += (uint64_t)t << sh;
    }
}

__device__ __forceinline__ void rle_acc_out(const uint64_t acc[2], const int64_t base[SIGMA], int64_t l,
                                            int64_t r[SIGMA]) {
    constexpr uint64_t M = (1ull << 21) - 1;
    r[1] = base[1] + (int64_t)(acc[0] & M);
    r[2] = base[2] + (int64_t)((acc[0] >> 21) & M);
    r[3] = base[3] + (int64_t)((acc[0] >> 42) & M);
    r[4] = base[4] + (int64_t)(acc[1] & M);
    r[5] = base[5] + (int64_t)((acc[1] >> 21) & M);
    r[0] = l - (r[1] + r[2] + r[3] + r[4] + r[5]);
}

// Span sp: the ranks at its start (gbase added), and the decode start for
// offset o: the last mark at or before o (or the span start), as its offset,
// packed ranks and first run byte.
__device__ __forceinline__ const uint8_t *rle_start(const OccView &v, int64_t sp, int64_t o, int64_t base[SIGMA],
                                                    int64_t *pos, uint64_t acc[2]) {
    const uint8_t *hp = v.blocks + sp * RLE_HDR_BYTES;
    const Sec h = ld_sec64(hp), mk = ld_sec64(hp + 32);
    base[0] = 0;
#pragma unroll
    for (int a = 1; a < SIGMA; ++a) base[a] = (int64_t)h.w[a - 1];
    if (v.gbase) {
        const int64_t *g = v.gbase + 5 * ((sp << v.log2D) >> GSPAN_LOG2);
#pragma unroll
        for (int a = 1; a < SIGMA; ++a) base[a] += g[a - 1];
    }
    const uint8_t *p = v.payload + ((uint64_t)h.w[5] | ((uint64_t)h.w[6] << 32));
    // mark j: words 8j..8j+3 of the second sector = pos | A << 16, C | G << 16, T | N << 16, byte offset
    const uint32_t p0 = mk.w[0] & 0xFFFFu, p1 = mk.w[4] & 0xFFFFu;
    const int j = (uint32_t)o >= p1 ? 1 : ((uint32_t)o >= p0 ? 0 : -1);
    acc[0] = acc[1] = 0;
    *pos = 0;
    if (j >= 0) {
        const uint32_t w0 = j ? mk.w[4] : mk.w[0], w1 = j ? mk.w[5] : mk.w[1], w2 = j ? mk.w[6] : mk.w[2],
                       w3 = j ? mk.w[7] : mk.w[3];
        *pos = w0 & 0xFFFFu;
        acc[0] = (uint64_t)(w0 >> 16) | ((uint64_t)(w1 & 0xFFFFu) << 21) | ((uint64_t)(w1 >> 16) << 42);
        acc[1] = (uint64_t)(w2 & 0xFFFFu) | ((uint64_t)(w2 >> 16) << 21);
        p += w3;
    }
    return p;
}

// rank(a, l) for every a, and (WANT_SYM, l < n) the symbol B[l]: the span of l
// is decoded from the last mark before l to the run holding l.
template <bool WANT_SYM>
__device__ __forceinline__ void rle_rank(const OccView &v, int64_t l, int64_t r[SIGMA], int *sym) {
    const int64_t sp = l >> v.log2D, s0 = sp << v.log2D, o = l - s0;
    int64_t base[SIGMA], pos;
    uint64_t acc[2];
    const uint8_t *p = rle_start(v, sp, o, base, &pos, acc);
    int64_t slen = v.n - s0;
    if (slen > ((int64_t)1 << v.log2D)) slen = (int64_t)1 << v.log2D;
    int64_t stop = WANT_SYM ? o + 1 : o;  // decode runs while they start before stop
    if (stop > slen) stop = slen;
    int sy = 0;
    if (pos < stop) {
        RunRd rd;
        rd.init(p);
        while (pos < stop) {
            int a;
            int64_t len;
            rd.run(&a, &len);
            const int64_t t = o - pos < len ? o - pos : len;  // below 0 only for WANT_SYM's last run
            rle_acc_add(acc, a, t > 0 ? t : 0);
            sy = a;
            pos += len;
        }
    }
    rle_acc_out(acc, base, l, r);
    if (WANT_SYM) *sym = sy;
}

// rank_all at l0 <= l1 of one span, decoded once (from the last mark before l0).
__device__ __forceinline__ void rle_rank2(const OccView &v, int64_t l0, int64_t l1, int64_t r0[SIGMA],
                                          int64_t r1[SIGMA]) {
    const int64_t sp = l1 >> v.log2D, s0 = sp << v.log2D, o0 = l0 - s0, o1 = l1 - s0;
    int64_t base[SIGMA], pos;
    uint64_t acc1[2];
    const uint8_t *p = rle_start(v, sp, o0, base, &pos, acc1);
    uint64_t acc0[2] = {acc1[0], acc1[1]};
    if (pos < o1) {
        RunRd rd;
        rd.init(p);
        while (pos < o1) {
            int a;
            int64_t len;
            rd.run(&a, &len);
            const int64_t t1 = o1 - pos < len ? o1 - pos : len;
            const int64_t t0 = o0 - pos < len ? o0 - pos : len;
            rle_acc_add(acc1, a, t1);
            rle_acc_add(acc0, a, t0 > 0 ? t0 : 0);
            pos += len;
        }
    }
    rle_acc_out(acc0, base, l0, r0);
    rle_acc_out(acc1, base, l1, r1);
}

// Loads of one rank: the header sector and the payload sectors that hold the
// nibbles before offset o, all issued before any is used.  NS = D/64 payload
// sectors per block (1, 2 or 4); sectors past o are not loaded.  NS = 0 is the
// D = 32 layout: the block is one sector, and the rank also needs the position
// (for $) and the span base.
template <int NS> struct BlockLd {
    Sec h, p[NS];
    int o;
};
template <> struct BlockLd<0> {
    Sec h;
    int o;
    int64_t l;
    const int64_t *gb;
};
// Run-length layout: the span is decoded at load time; the load keeps every
// rank at l and the symbol B[l].
template <> struct BlockLd<NS_RLE> {
    int64_t r[SIGMA];
    int sym;
};

template <int NS> __device__ __forceinline__ BlockLd<NS> block_load(const OccView &v, int64_t l) {
    BlockLd<NS> b;
    if constexpr (NS == NS_RLE) {
        rle_rank<true>(v, l, b.r, &b.sym);
    } else if constexpr (NS == 0) {
        b.h = ld_sec64(v.blocks + (l >> 5) * 32);
        b.o = (int)(l & 31);
        b.l = l;
        b.gb = v.gbase ? v.gbase + 5 * (l >> GSPAN_LOG2) : nullptr;
    } else {
        const uint8_t *blk = v.blocks + (l >> v.log2D) * (int64_t)v.bb;
        b.o = (int)(l & (64 * NS - 1));
        b.h = ld_sec64(blk);
#pragma unroll
        for (int j = 0; j < NS; ++j)
            if (NS == 1 || b.o > 64 * j) b.p[j] = ld_sec64(blk + HEADER_BYTES + 32 * j);
    }
    return b;
}

// D = 32: symbols equal to c among the block's symbols, as a bit mask.
__device__ __forceinline__ uint32_t s32_match(const Sec &s, int c) {
    const uint32_t p0 = s.w[5], p1 = s.w[6], p2 = s.w[7];
    return ((c & 1) ? p0 : ~p0) & ((c & 2) ? p1 : ~p1) & ((c & 4) ? p2 : ~p2);
}

template <int NS> __device__ __forceinline__ void block_rank_all(const BlockLd<NS> &b, int64_t r[6]) {
    if constexpr (NS == NS_RLE) {
#pragma unroll
        for (int a = 0; a < SIGMA; ++a) r[a] = b.r[a];
    } else if constexpr (NS == 0) {
        const uint32_t mk = (1u << b.o) - 1u;  // o <= 31
        const uint32_t p0 = b.h.w[5], p1 = b.h.w[6], p2 = b.h.w[7];
        const uint32_t b0 = p0 & mk, n0 = ~p0 & mk;
        const uint32_t t00 = ~p1 & ~p2, t10 = p1 & ~p2, t01 = ~p1 & p2;
        r[1] = (int64_t)b.h.w[0] + __popc(b0 & t00);
        r[2] = (int64_t)b.h.w[1] + __popc(n0 & t10);
        r[3] = (int64_t)b.h.w[2] + __popc(b0 & t10);
        r[4] = (int64_t)b.h.w[3] + __popc(n0 & t01);
        r[5] = (int64_t)b.h.w[4] + __popc(b0 & t01);
        if (b.gb) {
#pragma unroll
            for (int a = 1; a < SIGMA; ++a) r[a] += b.gb[a - 1];
        }
        r[0] = b.l - (r[1] + r[2] + r[3] + r[4] + r[5]);
    } else {
        hdr_all(b.h, r);
#pragma unroll
        for (int j = 0; j < NS; ++j)
            if (NS == 1 || b.o > 64 * j) sec_count_all(b.p[j], b.o - 64 * j, r);
    }
}

template <int NS> __device__ __forceinline__ int64_t block_rank(const BlockLd<NS> &b, int c) {
    if constexpr (NS == NS_RLE) {
        int64_t r = b.r[0];
#pragma unroll
        for (int a = 1; a < SIGMA; ++a)
            if (c == a) r = b.r[a];
        return r;
    } else if constexpr (NS == 0) {
        if (c == 0) {  // $: position minus the other five ranks
            int64_t r[SIGMA];
            block_rank_all<0>(b, r);
            return r[0];
        }
        uint32_t w = b.h.w[0];
#pragma unroll
        for (int a = 2; a < SIGMA; ++a)
            if (c == a) w = b.h.w[a - 1];
        int64_t r = (int64_t)w + __popc(s32_match(b.h, c) & ((1u << b.o) - 1u));
        if (b.gb) r += b.gb[c - 1];
        return r;
    } else {
        int64_t r = hdr_get(b.h, c);
#pragma unroll
        for (int j = 0; j < NS; ++j)
            if (NS == 1 || b.o > 64 * j) r += sec_count(b.p[j], c, b.o - 64 * j);
        return r;
    }
}

// rank_B(c, l) = |{i < l : B[i] = c}|  (Table 1).
template <int NS> __device__ __forceinline__ int64_t rank1(const OccView &v, int c, int64_t l) {
    BlockLd<NS> b = block_load<NS>(v, l);
    return block_rank<NS>(b, c);
}

// rank_B(a, l) for every symbol a.
template <int NS> __device__ __forceinline__ void rank_all(const OccView &v, int64_t l, int64_t r[SIGMA]) {
    if constexpr (NS == NS_RLE) {
        rle_rank<false>(v, l, r, nullptr);
    } else {
        BlockLd<NS> b = block_load<NS>(v, l);
        block_rank_all<NS>(b, r);
    }
}

// Any D (tile-level lookups outside the hot loops).
__device__ __forceinline__ void rank_all_any(const OccView &v, int64_t l, int64_t r[SIGMA]) {
    if (v.payload) {
        rank_all<NS_RLE>(v, l, r);
        return;
    }
    if (v.log2D == 5) {
        rank_all<0>(v, l, r);
        return;
    }
    const int ns = (1 << v.log2D) >> 6;
    if (ns == 1) rank_all<1>(v, l, r);
    else if (ns == 2) rank_all<2>(v, l, r);
    else rank_all<4>(v, l, r);
}

// Symbol B[i]: bit o of the three planes that hold it.
__device__ __forceinline__ int sym_at(const OccView &v, int64_t i) {
    if (v.payload) {
        int64_t r[SIGMA];
        int a;
        rle_rank<true>(v, i, r, &a);
        return a;
    }
    if (v.log2D == 5) {
        const uint32_t *w = reinterpret_cast<const uint32_t *>(v.blocks + (i >> 5) * 32);
        const int bit = (int)(i & 31);
        const uint32_t p0 = __ldg(w + 5), p1 = __ldg(w + 6), p2 = __ldg(w + 7);
        return (int)(((p0 >> bit) & 1u) | (((p1 >> bit) & 1u) << 1) | (((p2 >> bit) & 1u) << 2));
    }
    const uint8_t *blk = v.blocks + (i >> v.log2D) * (int64_t)v.bb;
    int o = (int)(i & ((1 << v.log2D) - 1));
    const uint8_t *sec = blk + HEADER_BYTES + 32 * (o >> 6);
    int bit = o & 63;
    uint64_t p0 = ldg_u64(sec), p1 = ldg_u64(sec + 8), p2 = ldg_u64(sec + 16);
    return (int)(((p0 >> bit) & 1u) | (((p1 >> bit) & 1u) << 1) | (((p2 >> bit) & 1u) << 2));
}

// Writer side: the 8 lanes 8g..8g+7 of a warp hold the plane bytes of the 8
// consecutive 8-symbol groups of one 64-symbol sector; an xor butterfly inside
// the 8 lanes builds each 64-bit plane and lanes 0..3 of the group store planes
// 0..3 (plane 3 zero).  mask: the active lanes (whole 8-lane groups).
__device__ __forceinline__ void store_planes(uint8_t *sec, uint32_t b0, uint32_t b1, uint32_t b2, unsigned mask,
                                             bool do_store) {
    const int j = threadIdx.x & 7;
    uint64_t v0 = (uint64_t)b0 << (8 * j), v1 = (uint64_t)b1 << (8 * j), v2 = (uint64_t)b2 << (8 * j);
#pragma unroll
    for (int d = 1; d < 8; d <<= 1) {
        v0 |= __shfl_xor_sync(mask, v0, d);
        v1 |= __shfl_xor_sync(mask, v1, d);
        v2 |= __shfl_xor_sync(mask, v2, d);
    }
    if (do_store && j < 4) *reinterpret_cast<uint64_t *>(sec + 8 * j) = j == 0 ? v0 : (j == 1 ? v1 : (j == 2 ? v2 : 0ull));
}

// The same for a D = 32 block: the 4 lanes 4g..4g+3 hold the plane bytes of its
// four 8-symbol groups; lanes 0..2 of the group store the 32-bit planes at
// words 5..7.  mask: the active lanes (whole 4-lane groups).
__device__ __forceinline__ void store_planes32(uint8_t *blk, uint32_t b0, uint32_t b1, uint32_t b2, unsigned mask,
                                               bool do_store) {
    const int j = threadIdx.x & 3;
    uint32_t v0 = b0 << (8 * j), v1 = b1 << (8 * j), v2 = b2 << (8 * j);
#pragma unroll
    for (int d = 1; d < 4; d <<= 1) {
        v0 |= __shfl_xor_sync(mask, v0, d);
        v1 |= __shfl_xor_sync(mask, v1, d);
        v2 |= __shfl_xor_sync(mask, v2, d);
    }
    if (do_store && j < 3) reinterpret_cast<uint32_t *>(blk)[5 + j] = j == 0 ? v0 : (j == 1 ? v1 : v2);
}

// Writer side: byte of plane b that holds symbols [8j, 8j+8) of a block.
__device__ __forceinline__ int plane_byte(int o_in_block, int b, int log2D) {
    if (log2D == 5) return 20 + 4 * b + (o_in_block >> 3);
    return HEADER_BYTES + 32 * (o_in_block >> 6) + 8 * b + ((o_in_block & 63) >> 3);
}

// Sampled suffix array: is row j sampled, and where is its value.
constexpr int SVAL_OFF_BITS = 40;
__device__ __forceinline__ bool sample_at(const uint64_t *__restrict__ sdir, int64_t j, int64_t *vidx) {
    const ulonglong2 w = __ldg(reinterpret_cast<const ulonglong2 *>(sdir) + (j >> 6));
    const uint64_t bit = 1ull << (j & 63);
    *vidx = (int64_t)w.y + __popcll(w.x & (bit - 1));
    return (w.x & bit) != 0;
}

// SA bi-interval (k, k', s) of Section "Double-strand BWT".
struct BiInt {
    int64_t k, kp, s;
};

// Algorithm 3, BackwardExt: for b < comp(a): k' += pi(comp b, k+s) - pi(comp b, k);
// s <- pi(a,k+s) - pi(a,k); k <- pi(a,k).  (C_B cancels in the differences.)
// Both blocks are loaded before either is counted.
template <int NS> __device__ __forceinline__ BiInt backward_ext(const OccView &v, BiInt x, int a) {
    int64_t r0[SIGMA], r1[SIGMA];
    if constexpr (NS == NS_RLE) {  // one decode when both ends share a span
        const int64_t e = x.k + x.s;
        if ((e >> v.log2D) == (x.k >> v.log2D)) {
            rle_rank2(v, x.k, e, r0, r1);
        } else {
            rle_rank<false>(v, x.k, r0, nullptr);
            rle_rank<false>(v, e, r1, nullptr);
        }
    } else {
        // both ends' blocks are requested before either is counted; when both
        // ends fall in one block it is read once
        const int64_t e = x.k + x.s;
        const int lg = NS == 0 ? 5 : v.log2D;
        const bool same = (e >> lg) == (x.k >> lg);
        BlockLd<NS> b0 = block_load<NS>(v, x.k);
        BlockLd<NS> b1;
        if (!same) {
            b1 = block_load<NS>(v, e);
        } else {
            b1 = b0;
            if constexpr (NS == 0) {
                b1.o = (int)(e & 31);
                b1.l = e;
            } else {
                b1.o = (int)(e & (64 * NS - 1));
                if (NS > 1)  // payload sectors the first offset did not need (block_load skips them)
#pragma unroll
                    for (int j = 0; j < NS; ++j)
                        if (b1.o > 64 * j && !(b0.o > 64 * j))
                            b1.p[j] = ld_sec64(v.blocks + (e >> v.log2D) * (int64_t)v.bb + HEADER_BYTES + 32 * j);
            }
        }
        block_rank_all<NS>(b0, r0);
        block_rank_all<NS>(b1, r1);
    }
    int64_t d[SIGMA];
#pragma unroll
    for (int i = 0; i < SIGMA; ++i) d[i] = r1[i] - r0[i];
    const int ac = comp_sym(a);
    int64_t add = 0;
#pragma unroll
    for (int b = 0; b < SIGMA; ++b)
        if (b < ac) add += d[(b >= 1 && b <= 4) ? 5 - b : b];
    int64_t s = d[0], k = v.C[0] + r0[0];
#pragma unroll
    for (int i = 1; i < SIGMA; ++i)
        if (a == i) {
            s = d[i];
            k = v.C[i] + r0[i];
        }
    BiInt y;
    y.kp = x.kp + add;
    y.s = s;
    y.k = k;
    return y;
}

// Algorithm 3, ForwardExt = swap(BackwardExt(swap(x), comp(a))).
template <int NS> __device__ __forceinline__ BiInt forward_ext(const OccView &v, BiInt x, int a) {
    BiInt y = {x.kp, x.k, x.s};
    y = backward_ext<NS>(v, y, comp_sym(a));
    BiInt z = {y.kp, y.k, y.s};
    return z;
}

// C_B(a) by register select.
__device__ __forceinline__ int64_t C_of(const OccView &v, int a) {
    int64_t c = v.C[0];
#pragma unroll
    for (int i = 1; i < SIGMA; ++i)
        if (a == i) c = v.C[i];
    return c;
}

// ---- block-level scans (256-thread blocks) -------------------------------
constexpr int SC_THREADS = 256;

template <class T> __device__ __forceinline__ T op2(T a, T b, int op) { return op == 0 ? a + b : (a > b ? a : b); }

template <class T> __device__ __forceinline__ T warp_incl(T v, int op) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v = op2(v, u, op);
    }
    return v;
}

// Exclusive scan of one value per thread across a 256-thread block.
template <class T> __device__ __forceinline__ T block_excl(T v, int op, T *wtot) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = warp_incl(v, op);
    if (lane == 31) wtot[w] = inc;
    __syncthreads();
    if (w == 0) {
        T t = lane < SC_THREADS / 32 ? wtot[lane] : T(0);
        T ti = warp_incl(t, op);
        if (lane < SC_THREADS / 32) wtot[lane] = ti;  // inclusive over warps
    }
    __syncthreads();
    T before = w ? wtot[w - 1] : T(0);
    T up = __shfl_up_sync(0xffffffffu, inc, 1);
    T excl = lane ? up : T(0);
    T r = op2(before, excl, op);
    __syncthreads();
    return r;
}

// ---- primitives (sort.cu) --------------------------------------------------
// Device-wide scans.  op: 0 = sum, 1 = max.
int scan_u32(const uint32_t *in, uint32_t *out, int64_t n, bool inclusive, int op, cudaStream_t st);
int scan_u64(const uint64_t *in, uint64_t *out, int64_t n, bool inclusive, cudaStream_t st);
int scan_u32_ws(const uint32_t *in, uint32_t *out, int64_t n, bool inclusive, uint32_t *part_ws, int64_t part_cap,
                cudaStream_t st);
// Stable LSD radix sort of (key, value) pairs on bits [begin_bit, end_bit).
// The result ends in (k0, v0) if *in_alt comes back false, else in (k1, v1).
int radix_sort_pairs(uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1, int64_t n, int begin_bit,
                     int end_bit, cudaStream_t st, bool *in_alt);
int radix_sort_pairs32(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, int64_t n, int begin_bit, int end_bit,
                       cudaStream_t st, bool *in_alt);

// ---- phases (build.cu / merge.cu / search.cu) -------------------------------
int build_batch_impl(const uint8_t *seq_dev, const int64_t *lens_host, int64_t n_seq, const rb3_opts &o,
                     cudaStream_t st, rb3_index *out);
int merge_impl(rb3_index *dst, const rb3_index *src, const rb3_opts &o, cudaStream_t st);
int wait_selftest(int limit, cudaStream_t st);
int walk_stats(int64_t out[4], bool reset);
int search_stats(int64_t out[2], bool reset);
int merge_positions(const rb3_index *dst, const rb3_index *src, const rb3_opts &o, cudaStream_t st, int64_t *pos,
                    unsigned int *err_dev = nullptr, const int32_t *owner = nullptr, int32_t part = 0);
// The scatter-merge of src into dst at the given merged rows pos (device,
// src->n entries, as merge_positions writes them for every part).
int merge_apply(rb3_index *dst, const rb3_index *src, const int64_t *pos, const unsigned int *walk_err,
                cudaStream_t st);
// Autotuner memory (tune.cu): 0 when nothing was tuned for this input shape.
int64_t tuned_seg_len(const rb3_index *dst, const rb3_index *src);
int64_t tuned_seed_cap(const rb3_index *dst, const rb3_index *src);
int64_t tuned_chunk_len(const rb3_index *idx, int64_t nq, int64_t total_q);
int append_batches(rb3_index *dst, const uint8_t *seq, const int64_t *lens, int64_t n_seq, const int64_t *batch_end,
                   int64_t n_batches, const rb3_opts &o, cudaStream_t caller);
int backward_search_impl(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, int64_t nq, int64_t total_q,
                         int64_t *lohi, cudaStream_t st);
// RB3_E_INVAL when a query symbol lies outside 1..5.
int check_codes(const uint8_t *q, int64_t n, cudaStream_t st);
// Haplotype diversity of every query (prm = a, b, q, e, W, redundancy);
// device pointers throughout.
int diversity_impl(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, int64_t nq, int64_t total_q,
                   const int32_t prm[6], int64_t *out, int64_t *n_out, cudaStream_t st);
int diversity_stats(int64_t out[2], bool reset);
// BWA-SW between the prefix DAWG of every query and the text's (prm = a, b, q,
// e, W); records of 7 int64 (qid, uk, us, k, k', s, H) sorted by (qid, uk, us,
// band rank); q, qoff device pointers, qo the offsets on the host.
int bwasw_impl(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, const std::vector<int64_t> &qo, int64_t nq,
               const int32_t prm[5], int64_t *out, int64_t cap, int64_t *n_out, cudaStream_t st);
// Hot-level table: entry hot_off(L) + w is the bi-interval of the string of
// length L whose base-4 digits (A..T = 0..3, first symbol most significant)
// spell w, as BackwardExt computes it from the whole index, last symbol first.
struct alignas(32) HotEnt {
    int64_t k, kp, s, pad;
};
__host__ __device__ __forceinline__ int64_t hot_off(int L) { return ((int64_t(1) << (2 * L)) - 4) / 3; }
constexpr int HOT_MAX = 12;
// The table of depth K for idx (built or rebuilt on stream st, which it then
// synchronizes, when the index has none of that depth or has changed since).
int hot_table(const rb3_index *idx, int K, cudaStream_t st, const HotEnt **out);
// The depth a search uses: o.hot_depth, else the tuned one, else log4(n) - 3
// clamped to 0..10 (0: no table).
int hot_depth_for(const rb3_index *idx, const rb3_opts &o, int64_t nq, int64_t total_q);
void free_hot(rb3_index *x);
int64_t tuned_hot_depth(const rb3_index *idx, int64_t nq, int64_t total_q);
int mem_search_impl(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, const int64_t *qoff_host,
                    int64_t nq, int64_t total_q, int32_t min_len, int64_t min_occ, const rb3_opts &o,
                    rb3_smem *out_dev, int64_t cap, int64_t *n_out, cudaStream_t st,
                    bool codes_checked = false);
int export_impl(const rb3_index *idx, uint8_t *codes_dev, int64_t *occ_dev, cudaStream_t st);
int rle_export_impl(const rb3_index *x, uint8_t *codes, int64_t *occ, cudaStream_t st);
// Merge of any two layouts: a run-length src is merged through a plain copy of
// it; a run-length dst is merged into directly (its spans rewritten).
int merge_any(rb3_index *dst, const rb3_index *src, const rb3_opts &o, cudaStream_t st);
int rle_check_impl(const rb3_index *x, cudaStream_t st);
// The run-length arrays of a run-length dst merged with a plain src at rows pos.
int rle_merge_arrays(const rb3_index *dst, const rb3_index *src, const int64_t *pos, cudaStream_t st,
                     rb3_index *out);
// Sampled suffix array of a batch from its SA (builder) and of a merge (from pos).
int sample_batch(rb3_index *x, const int32_t *SA, cudaStream_t st);
int sample_merge(const rb3_index *dst, const rb3_index *src, const int64_t *pos, const int64_t *kstart,
                 int64_t ntiles, int64_t nM, int tile_rows, rb3_index *out, cudaStream_t st);
void free_samples(rb3_index *x);
// Fills idx->C from its blocks (rank of every symbol at n).
int finalize_counts(rb3_index *idx, cudaStream_t st);

// Calls body with a compile-time NS = D/64 for D in {64, 128, 256}, NS = 0 for
// D = 32 and NS = NS_RLE for a run-length index (D = its span, 512 or more).
#define RB3_WITH_NS(D, ...)                      \
    do {                                         \
        if ((D) > 256) {                         \
            constexpr int NS = NS_RLE;           \
            __VA_ARGS__;                         \
        } else if ((D) == 32) {                  \
            constexpr int NS = 0;                \
            __VA_ARGS__;                         \
        } else if ((D) == 64) {                  \
            constexpr int NS = 1;                \
            __VA_ARGS__;                         \
        } else if ((D) == 128) {                 \
            constexpr int NS = 2;                \
            __VA_ARGS__;                         \
        } else {                                 \
            constexpr int NS = 4;                \
            __VA_ARGS__;                         \
        }                                        \
    } while (0)

inline int ilog2(int64_t x) {
    int r = 0;
    while ((int64_t(1) << (r + 1)) <= x) ++r;
    return r;
}

inline int num_sms() {
    static const int sms = [] {  // thread-safe one-time initialisation
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return n > 0 ? n : 1;
    }();
    return sms;
}

}  // namespace rb3
