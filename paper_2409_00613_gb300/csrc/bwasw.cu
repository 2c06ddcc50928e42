// BWA-SW between two prefix DAWGs (Section "Finding inexact matches with
// BWA-SW", Algorithm 5): the query's DAWG against the indexed text's.
//
// The query DAWG of P: a node is the SA interval (uk, us) of a substring of P
// in the BWT of the one-string, one-strand text P$ (substrings with one
// interval, x and xz, are one node), an edge x -> cx for every symbol c of
// A..N whose BackwardExt keeps the interval non-empty; the root is the whole
// interval (0, |P|+1).  An edge leads from a string to a one-symbol-longer one
// that starts earlier in P, so the graph is acyclic; nodes are visited in a
// topological order.  A text node is a bi-interval (k, k', s) of the indexed
// double-strand text; its children are its BackwardExt by A, C, G, T.
//
// The cells of a query node v gather, over the in-edges (u, c) of v, from u's
// kept cells: the four children of each (match +a if the text symbol is c,
// else -b; an N in P matches nothing) and the cell itself (insertion: E =
// max(H - q, E) - e, H = max(H, E)); then deletions to the closure (F of a
// child = max(H - q, F) - e, a cell re-extended whenever its H or F rises);
// the band keeps the W cells of largest H (ties: smaller k, k', s).  The
// root's one cell is the whole text (H = 0).  Only cells with H > 0 are kept
// (a cell that never rises above 0 extends nothing positive), and the result
// is every kept cell of every node but the root.
//
// Two kernels.  k_qdawg, one CTA per query: the suffix array of P$ by prefix
// doubling (bitonic sorts in shared memory), its BWT and rank table, the
// DAWG's nodes by level-synchronous BackwardExt from the root (a hash table
// in shared memory finds repeated intervals), a topological order by Kahn's
// waves, and every node's in-edges, written to global memory.  k_bwasw, one
// warp per query: the nodes in topological order, each node's cells in a
// table of the warp's own in shared memory (as the linear-query kernel), its
// kept cells (at most W) stored in global memory for its successors.  The
// records are then sorted by (query, query node, band rank).
#include <vector>

#include "align.cuh"

namespace rb3 {
namespace {

using namespace dv;

constexpr int BW_MAXP = 2047;         // longest query: P$ fits 2048 positions
constexpr int BW_NP = BW_MAXP + 1;    // 2048
constexpr int BW_MAXN = 2 * BW_NP;    // the SA intervals of P$'s substrings: below 2 |P$|
constexpr int BW_HASH = 8192;         // node hash slots (a power of two, twice the nodes)
constexpr int BW_THREADS = 256;
constexpr int BW_PER = BW_NP / BW_THREADS;
constexpr int BW_CAP_S = 256, BW_WARPS_S = 1;  // cell tables, as the linear-query kernel
constexpr int BW_CAP_L = 2048, BW_WARPS_L = 1;
static_assert(dv_warp_bytes(BW_CAP_S) % 16 == 0 && dv_warp_bytes(BW_CAP_L) % 16 == 0, "table alignment");

// edges of a query with np = |P| + 1: at most one per node and symbol
__host__ __device__ __forceinline__ int64_t bw_edges(int64_t np) { return 10 * np; }

// Per-query scratch, in a chunk of queries: nodes [nb, nb + 2 np), edges [eb,
// eb + 10 np); in_off has one more entry per query ([nb + j + i] for the i-th
// query of the chunk).
struct QDawg {
    int32_t *nn;       // [queries] nodes of the query's DAWG
    int32_t *uk, *us;  // [nodes] in topological order (position 0: the root)
    int32_t *in_off;   // [nodes + queries]
    int32_t *in_pred;  // [edges] predecessor's topological position
    uint8_t *in_c;     // [edges] edge symbol (1..5)
    int32_t *e_from, *e_to;  // [edges] staging in discovery order (node ids)
    uint8_t *e_c;
    int32_t *o_to;     // [edges] targets grouped by source
};

// ---- kernel A: the query DAWG ----------------------------------------------------

struct QSmem {
    uint64_t key[BW_NP];          // sort keys: (rank + 1, next rank + 1, position)
    uint16_t occ[6][BW_NP + 1];   // occ[c][i] = #{j < i : BP[j] = c}
    int32_t hkey[BW_HASH];        // node hash: interval key + 1 (0 = empty)
    int16_t hid[BW_HASH];         // node id of the slot
    int16_t rk[BW_NP];            // ranks of the prefix doubling
    int16_t nuk[BW_MAXN], nus[BW_MAXN];
    int32_t cnt[BW_MAXN];         // in-degrees (Kahn), then in-edge fill
    int32_t fill[BW_MAXN];        // out-edge counts, then fill
    int16_t ooff[BW_MAXN + 1];    // out-edges of node u: o_to[ooff[u] .. ooff[u+1])
    int16_t topo[BW_MAXN];        // node id at topological position
    int16_t tpos[BW_MAXN];        // topological position of a node id
    int32_t ioff[BW_MAXN + 1];    // in-edges by topological position
    uint8_t T[BW_NP], BP[BW_NP];
    int32_t C[7];
    int32_t nn, ne, tcount;
    int32_t tot;
    uint32_t wtot[32];
};

__device__ __forceinline__ uint32_t qd_hash(uint32_t key) {
    key ^= key >> 15;
    key *= 0x2c1b3c6du;
    key ^= key >> 12;
    return key & (BW_HASH - 1);
}

// Inserts the interval (lo, s) when absent (a new id), else nothing.
__device__ void qd_insert(QSmem &S, int lo, int s) {
    const int32_t tag = lo * 4096 + s + 1;
    for (uint32_t h = qd_hash((uint32_t)tag);; h = (h + 1) & (BW_HASH - 1)) {
        const int32_t cur = S.hkey[h];
        if (cur == tag) return;
        if (cur == 0) {
            const int32_t old = atomicCAS(&S.hkey[h], 0, tag);
            if (old == 0) {
                const int id = atomicAdd(&S.nn, 1);
                if (id < BW_MAXN) {  // below 2 |P$| for any P; the caller checks the count
                    S.nuk[id] = (int16_t)lo;
                    S.nus[id] = (int16_t)s;
                    S.hid[h] = (int16_t)id;
                }
                return;
            }
            if (old == tag) return;
        }
    }
}

// The id of an interval inserted before the last barrier.
__device__ int qd_lookup(const QSmem &S, int lo, int s) {
    const int32_t tag = lo * 4096 + s + 1;
    for (uint32_t h = qd_hash((uint32_t)tag);; h = (h + 1) & (BW_HASH - 1)) {
        const int32_t cur = S.hkey[h];
        if (cur == tag) return S.hid[h];
        if (cur == 0) return -1;
    }
}

__device__ __forceinline__ void bitonic_sort(uint64_t *key) {
    for (int k = 2; k <= BW_NP; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int idx = threadIdx.x; idx < BW_NP / 2; idx += BW_THREADS) {
                const int i = (idx / j) * 2 * j + (idx % j), p = i + j;
                const bool up = (i & k) == 0;
                const uint64_t a = key[i], b = key[p];
                if ((a > b) == up) {
                    key[i] = b;
                    key[p] = a;
                }
            }
            __syncthreads();
        }
}

// Exclusive scan of PER values per thread (thread t holds entries t*PER ..);
// returns the total.
template <int PER>
__device__ __forceinline__ int cta_scan(int v[PER], QSmem &S) {
    int s = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int t = v[i];
        v[i] = s;
        s += t;
    }
    const uint32_t before = block_excl<uint32_t>((uint32_t)s, 0, S.wtot);
#pragma unroll
    for (int i = 0; i < PER; ++i) v[i] += (int)before;
    if (threadIdx.x == BW_THREADS - 1) S.tot = (int)before + s;
    __syncthreads();
    const int r = S.tot;
    __syncthreads();
    return r;
}

// child of interval (k, s) of the query's BWT by symbol c: [lo, hi)
__device__ __forceinline__ void qd_child(const QSmem &S, int k, int s, int c, int *lo, int *hi) {
    *lo = S.C[c] + S.occ[c][k];
    *hi = S.C[c] + S.occ[c][k + s];
}

__global__ void __launch_bounds__(BW_THREADS) k_qdawg(const uint8_t *__restrict__ q, const int64_t *__restrict__ qoff,
                                                      int64_t q0, int64_t nq, const int64_t *__restrict__ nbase,
                                                      const int64_t *__restrict__ ebase, QDawg G,
                                                      unsigned int *__restrict__ err) {
    extern __shared__ __align__(16) uint8_t qd_smem[];
    QSmem &S = *reinterpret_cast<QSmem *>(qd_smem);
    const int64_t ci = blockIdx.x;  // query of the chunk
    if (ci >= nq) return;
    const int64_t qi = q0 + ci;
    const int tid = threadIdx.x;
    const int m = (int)(qoff[qi + 1] - qoff[qi]), np = m + 1;
    const uint8_t *P = q + qoff[qi];
    const int64_t nb = nbase[ci], eb = ebase[ci], emax = bw_edges(np);
    for (int i = tid; i < BW_NP; i += BW_THREADS) {
        S.T[i] = i < m ? P[i] : 0;
        S.rk[i] = i < np ? (int16_t)S.T[i] : 0;
    }
    for (int i = tid; i < BW_HASH; i += BW_THREADS) {
        S.hkey[i] = 0;
        S.hid[i] = -1;
    }
    for (int i = tid; i < BW_MAXN; i += BW_THREADS) {
        S.cnt[i] = 0;
        S.fill[i] = 0;
    }
    if (tid == 0) {
        S.nn = 0;
        S.ne = 0;
        S.tcount = 0;
    }
    __syncthreads();
    // ---- suffix array of P$ by prefix doubling: sort by (rank[i], rank[i+h]) ----
    for (int h = 1;; h <<= 1) {
        for (int i = tid; i < BW_NP; i += BW_THREADS)
            S.key[i] = i < np ? ((uint64_t)(S.rk[i] + 1) << 32) |
                                    ((uint64_t)(i + h < np ? S.rk[i + h] + 1 : 0) << 16) | (uint64_t)i
                              : ~0ull;
        __syncthreads();
        bitonic_sort(S.key);
        // new rank of the suffix at sorted place j = number of changes of the pair up to j
        int f[BW_PER];
#pragma unroll
        for (int t = 0; t < BW_PER; ++t) {
            const int j = tid * BW_PER + t;
            f[t] = (j > 0 && j < np && (S.key[j] >> 16) != (S.key[j - 1] >> 16)) ? 1 : 0;
        }
        int g[BW_PER];
#pragma unroll
        for (int t = 0; t < BW_PER; ++t) g[t] = f[t];
        const int changes = cta_scan<BW_PER>(g, S);
#pragma unroll
        for (int t = 0; t < BW_PER; ++t) {
            const int j = tid * BW_PER + t;
            if (j < np) S.rk[S.key[j] & 0xffff] = (int16_t)(g[t] + f[t]);
        }
        __syncthreads();
        if (changes + 1 >= np || h >= BW_NP) break;
    }
    // ---- BWT of P$ (the row of the whole text holds its last symbol, $) and its ranks ----
    for (int j = tid; j < np; j += BW_THREADS) {
        const int sa = (int)(S.key[j] & 0xffff);
        S.BP[j] = sa > 0 ? S.T[sa - 1] : S.T[np - 1];
    }
    __syncthreads();
    {
        int tot[6];
        for (int a = 0; a < 6; ++a) {
            int v[BW_PER];
#pragma unroll
            for (int t = 0; t < BW_PER; ++t) {
                const int j = tid * BW_PER + t;
                v[t] = (j < np && S.BP[j] == a) ? 1 : 0;
            }
            tot[a] = cta_scan<BW_PER>(v, S);
#pragma unroll
            for (int t = 0; t < BW_PER; ++t) S.occ[a][tid * BW_PER + t] = (uint16_t)v[t];
        }
        // occ at np (and past it): the totals
        for (int a = 0; a < 6; ++a)
            for (int j = np + tid; j <= BW_NP; j += BW_THREADS) S.occ[a][j] = (uint16_t)tot[a];
        if (tid == 0) {
            S.C[0] = 0;
            for (int a = 0; a < 6; ++a) S.C[a + 1] = S.C[a] + tot[a];
        }
    }
    __syncthreads();
    // ---- the DAWG's nodes, level by level from the root; ids are consecutive per level ----
    if (tid == 0) qd_insert(S, 0, np);
    __syncthreads();
    for (int lv0 = 0, lv1 = 1; lv1 > lv0;) {
        for (int pr = tid; pr < (lv1 - lv0) * 5; pr += BW_THREADS) {
            const int u = lv0 + pr / 5, c = pr % 5 + 1;
            int lo, hi;
            qd_child(S, S.nuk[u], S.nus[u], c, &lo, &hi);
            if (hi > lo) qd_insert(S, lo, hi - lo);
        }
        __syncthreads();
        for (int pr = tid; pr < (lv1 - lv0) * 5; pr += BW_THREADS) {
            const int u = lv0 + pr / 5, c = pr % 5 + 1;
            int lo, hi;
            qd_child(S, S.nuk[u], S.nus[u], c, &lo, &hi);
            if (hi > lo) {
                const int v = qd_lookup(S, lo, hi - lo);
                const int e = atomicAdd(&S.ne, 1);
                if (v >= 0 && v < BW_MAXN && e < emax) {
                    G.e_from[eb + e] = u;
                    G.e_to[eb + e] = v;
                    G.e_c[eb + e] = (uint8_t)c;
                    atomicAdd(&S.cnt[v], 1);
                    atomicAdd(&S.fill[u], 1);
                } else {
                    atomicOr(err, 1u);
                }
            }
        }
        __syncthreads();
        const int n_now = S.nn;
        __syncthreads();
        lv0 = lv1;
        lv1 = n_now;
        if (lv1 > BW_MAXN) {  // cannot happen (a suffix tree of |P$| leaves); reported, never indexed
            if (tid == 0) atomicOr(err, 1u);
            return;
        }
    }
    const int nn = S.nn, ne = S.ne < emax ? S.ne : (int)emax;
    // ---- out-edges grouped by source ----
    {
        int v[BW_MAXN / BW_THREADS];
        for (int t = 0; t < BW_MAXN / BW_THREADS; ++t) {
            const int u = tid * (BW_MAXN / BW_THREADS) + t;
            v[t] = u < nn ? S.fill[u] : 0;
        }
        cta_scan<BW_MAXN / BW_THREADS>(v, S);
        for (int t = 0; t < BW_MAXN / BW_THREADS; ++t) {
            const int u = tid * (BW_MAXN / BW_THREADS) + t;
            S.ooff[u] = (int16_t)v[t];
            S.fill[u] = 0;
        }
        if (tid == 0) S.ooff[BW_MAXN] = (int16_t)ne;
        __syncthreads();
        for (int e = tid; e < ne; e += BW_THREADS) {
            const int u = G.e_from[eb + e];
            const int at = S.ooff[u] + atomicAdd(&S.fill[u], 1);
            G.o_to[eb + at] = G.e_to[eb + e];
        }
        __syncthreads();
    }
    // ---- a topological order: Kahn's waves from the root ----
    if (tid == 0) {
        S.topo[0] = 0;
        S.tcount = 1;
    }
    __syncthreads();
    for (int w0 = 0, w1 = 1; w1 > w0;) {
        for (int i = w0 + tid; i < w1; i += BW_THREADS) {
            const int u = S.topo[i];
            const int e1 = u + 1 < nn ? S.ooff[u + 1] : ne;
            for (int e = S.ooff[u]; e < e1; ++e) {
                const int v = G.o_to[eb + e];
                if (atomicSub(&S.cnt[v], 1) == 1) S.topo[atomicAdd(&S.tcount, 1)] = (int16_t)v;
            }
        }
        __syncthreads();
        const int t_now = S.tcount;
        __syncthreads();
        w0 = w1;
        w1 = t_now;
    }
    if (S.tcount != nn) {  // every node is reached from the root and the graph is acyclic
        if (tid == 0) atomicOr(err, 2u);
        return;
    }
    for (int i = tid; i < nn; i += BW_THREADS) {
        const int u = S.topo[i];
        S.tpos[u] = (int16_t)i;
        G.uk[nb + i] = S.nuk[u];
        G.us[nb + i] = S.nus[u];
        S.cnt[i] = 0;
    }
    __syncthreads();
    // ---- in-edges by topological position of the target ----
    for (int e = tid; e < ne; e += BW_THREADS) atomicAdd(&S.cnt[S.tpos[G.e_to[eb + e]]], 1);
    __syncthreads();
    {
        int v[BW_MAXN / BW_THREADS];
        for (int t = 0; t < BW_MAXN / BW_THREADS; ++t) {
            const int i = tid * (BW_MAXN / BW_THREADS) + t;
            v[t] = i < nn ? S.cnt[i] : 0;
        }
        cta_scan<BW_MAXN / BW_THREADS>(v, S);
        for (int t = 0; t < BW_MAXN / BW_THREADS; ++t) {
            const int i = tid * (BW_MAXN / BW_THREADS) + t;
            S.ioff[i] = v[t];
            S.cnt[i] = 0;
        }
        if (tid == 0) S.ioff[BW_MAXN] = ne;
        __syncthreads();
    }
    int32_t *ioff_g = G.in_off + nb + ci;
    for (int i = tid; i <= nn; i += BW_THREADS) ioff_g[i] = i < nn ? S.ioff[i] : ne;
    for (int e = tid; e < ne; e += BW_THREADS) {
        const int v = S.tpos[G.e_to[eb + e]];
        const int at = S.ioff[v] + atomicAdd(&S.cnt[v], 1);
        G.in_pred[eb + at] = S.tpos[G.e_from[eb + e]];
        G.in_c[eb + at] = G.e_c[eb + e];
    }
    if (tid == 0) G.nn[ci] = nn;
}

// ---- kernel B: the cells of every query node -------------------------------------

struct Kept {
    int64_t *k, *kp, *s;
    int32_t *H, *E;
    int32_t *n;  // [nodes] kept cells of the node
};

// GM: the tables in global memory (gtab, one per warp of the launch).
template <int NS, int CAP, int WARPS, bool GM>
__global__ void __launch_bounds__(32 * WARPS)
    k_bwasw(OccView V, const int64_t *__restrict__ sel, int64_t nsel, const int64_t *__restrict__ nbase,
            const int64_t *__restrict__ ebase, QDawg G, DvParams p, Kept K, int32_t *__restrict__ overflow,
            uint8_t *__restrict__ gtab) {
    extern __shared__ __align__(16) uint8_t bw_smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t wi = (int64_t)blockIdx.x * WARPS + w;
    if (wi >= nsel) return;  // the whole warp leaves together
    const int64_t ci = sel ? sel[wi] : wi;
    const DvTab T = dv_tab<CAP>(GM ? gtab + (size_t)wi * dv_warp_bytes(CAP) : bw_smem + (size_t)w * dv_warp_bytes(CAP));
    DvSt st{0, 0, 0};
    dv_clear_all<CAP>(T, st, lane);
    const int64_t nb = nbase[ci], eb = ebase[ci];
    const int nn = G.nn[ci];
    const int32_t *ioff = G.in_off + nb + ci;
    const int W = p.W;
    if (lane == 0) {
        K.k[nb * W] = 0;
        K.kp[nb * W] = 0;
        K.s[nb * W] = V.n;
        K.H[nb * W] = 0;
        K.E[nb * W] = DV_NEG;
        K.n[nb] = 1;
        overflow[ci] = 0;
    }
    __syncwarp();
    bool over = false;
    unsigned long long n_ext = 0;
    for (int v = 1; v < nn && !over; ++v) {
        dv_clear<CAP>(T, st, lane);
        for (int e = ioff[v]; e < ioff[v + 1] && !over; ++e) {
            const int u = G.in_pred[eb + e], c = G.in_c[eb + e];
            const int cnt = K.n[nb + u];
            const int64_t at = (nb + u) * W + lane;
            int64_t ck = 0, ckp = 0, cs = 0;
            int32_t cH = 0, cE = DV_NEG;
            if (lane < cnt) {
                ck = K.k[at];
                ckp = K.kp[at];
                cs = K.s[at];
                cH = K.H[at];
                cE = K.E[at];
            }
            // match / mismatch: the children of every kept cell of u
            int64_t xk[4] = {0, 0, 0, 0}, xkp[4] = {0, 0, 0, 0}, xs[4] = {0, 0, 0, 0};
            if (lane < cnt) dv_children<NS>(V, ck, ckp, cs, xk, xkp, xs);
            n_ext += cnt;
#pragma unroll 1
            for (int a = 1; a <= 4 && !over; ++a) {
                const int32_t g = cH + (a == c ? p.a : -p.b);
                const int64_t k = dv_pick(xk, a - 1), kp = dv_pick(xkp, a - 1), s = dv_pick(xs, a - 1);
                dv_upsert_batch<CAP>(T, st, lane < cnt && s > 0 && g > 0, k, kp, s, g, DV_NEG, DV_NEG, lane, over);
            }
            // insertion: the query symbol against a gap, the text node unchanged
            const int32_t ev = max(cH - p.q, cE) - p.e;
            if (!over) dv_upsert_batch<CAP>(T, st, lane < cnt && ev > 0, ck, ckp, cs, ev, ev, DV_NEG, lane, over);
        }
        // deletion: a text symbol against a gap, until no cell is left to extend
        dv_close<NS, CAP>(V, T, st, p, lane, over, n_ext);
        const int tn = st.tn;
        if (over) break;
        // the band (a warp sort, or a score histogram and sorts of what it singles out)
        const int keep = min(tn, W);
        {
            const int j = dv_band<CAP>(T, tn, W, lane);
            if (lane < keep) {
                const int64_t at = (nb + v) * W + lane;
                K.k[at] = T.k[j];
                K.kp[at] = T.kp[j];
                K.s[at] = T.s[j];
                K.H[at] = T.H[j];
                K.E[at] = T.E[j];
            }
        }
        if (lane == 0) K.n[nb + v] = keep;
        __syncwarp();  // every lane is done with the table before the next node refills it
    }
    if (over && lane == 0) overflow[ci] = 1;
    (void)n_ext;
}

// Records: one key per kept cell of every node but the root, (query, uk, us,
// band rank) -> its flat cell index.
__global__ void k_bw_keys(const int64_t *__restrict__ nbase, const int64_t *__restrict__ node_q, int64_t nodes,
                          int64_t q0, QDawg G, Kept K, int W, const int64_t *__restrict__ rec_off,
                          uint64_t *__restrict__ key, uint32_t *__restrict__ val) {
    const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x >= nodes) return;
    const int64_t ci = node_q[x], j = x - nbase[ci];
    if (j == 0 || j >= G.nn[ci]) return;
    const int n = K.n[x];
    for (int r = 0; r < n; ++r) {
        const int64_t at = rec_off[x] + r;
        key[at] = ((uint64_t)(q0 + ci) << 28) | ((uint64_t)G.uk[x] << 17) | ((uint64_t)G.us[x] << 5) | (uint64_t)r;
        val[at] = (uint32_t)(x * W + r);
    }
}

__global__ void k_bw_counts(const int64_t *__restrict__ nbase, const int64_t *__restrict__ node_q, int64_t nodes,
                            QDawg G, Kept K, uint64_t *__restrict__ cnt) {
    const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x >= nodes) return;
    const int64_t ci = node_q[x], j = x - nbase[ci];
    cnt[x] = (j == 0 || j >= G.nn[ci]) ? 0 : (uint64_t)K.n[x];
}

__global__ void k_bw_out(const uint64_t *__restrict__ key, const uint32_t *__restrict__ val, int64_t n, Kept K,
                         int64_t *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t kk = key[i];
    const uint32_t c = val[i];
    int64_t *o = out + 7 * i;
    o[0] = (int64_t)(kk >> 28);
    o[1] = (int64_t)((kk >> 17) & 2047);
    o[2] = (int64_t)((kk >> 5) & 4095);
    o[3] = K.k[c];
    o[4] = K.kp[c];
    o[5] = K.s[c];
    o[6] = K.H[c];
}

static inline unsigned nb_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

template <int NS, int CAP, int WARPS>
int bw_launch(const rb3_index *idx, const int64_t *sel, int64_t nsel, const int64_t *nbase, const int64_t *ebase,
              const QDawg &G, const DvParams &p, const Kept &K, int32_t *overflow, cudaStream_t st) {
    const size_t smem = WARPS * dv_warp_bytes(CAP);
    auto kern = k_bwasw<NS, CAP, WARPS, false>;
    RB3_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RB3_LAUNCH(kern, nb_for(nsel, WARPS), 32 * WARPS, smem, st, occ_view(idx), sel, nsel, nbase, ebase, G, p, K,
               overflow, (uint8_t *)nullptr);
    return RB3_OK;
}

// The global-memory tier: one warp per CTA, at most BW_GM_WARPS tables at once.
constexpr int64_t BW_GM_WARPS = 1024;
template <int NS>
int bw_launch_gm(const rb3_index *idx, const int64_t *sel, int64_t nsel, const int64_t *nbase, const int64_t *ebase,
                 const QDawg &G, const DvParams &p, const Kept &K, int32_t *overflow, cudaStream_t st) {
    const int64_t nw = nsel < BW_GM_WARPS ? nsel : BW_GM_WARPS;
    DevBuf tab;
    RB3_TRY(tab.alloc(dv_warp_bytes(DV_CAP_G) * (size_t)nw, st));
    for (int64_t b = 0; b < nsel; b += nw) {
        const int64_t n = nsel - b < nw ? nsel - b : nw;
        RB3_LAUNCH((k_bwasw<NS, DV_CAP_G, 1, true>), (unsigned)n, 32, 0, st, occ_view(idx), sel + b, n, nbase, ebase,
                   G, p, K, overflow, tab.as<uint8_t>());
    }
    return RB3_OK;
}

}  // namespace

// The queries in chunks that fit a scratch budget; each chunk: the DAWGs, the
// cells (small tables, then large ones for the queries that outgrew them), the
// records sorted and appended to out.
int bwasw_impl(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, const std::vector<int64_t> &qo, int64_t nq,
               const int32_t prm[5], int64_t *out, int64_t cap, int64_t *n_out, cudaStream_t st) {
    *n_out = 0;
    RB3_TRY(check_codes(q, qo[nq], st));
    if (nq == 0) return RB3_OK;
    const DvParams p{prm[0], prm[1], prm[2], prm[3], prm[4], 0};
    const int W = p.W;
    static_assert(sizeof(QSmem) <= 227 * 1024, "query DAWG shared memory");
    RB3_CUDA_TRY(cudaFuncSetAttribute(k_qdawg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(QSmem)));
    // scratch bytes of one query: DAWG arrays and kept cells
    auto q_bytes = [&](int64_t np) {
        return (2 * np + 1) * (3 * 4) + 2 * np * (int64_t)W * 32 + 2 * np * 4 + bw_edges(np) * (4 * 4 + 2);
    };
    const int64_t budget = (int64_t)1 << 31;
    Phase ph("search.bwasw", st);
    DevBuf err;
    RB3_TRY(err.alloc(sizeof(unsigned int), st));
    RB3_CUDA_TRY(cudaMemsetAsync(err.p, 0, sizeof(unsigned int), st));
    int64_t written = 0, total = 0;
    for (int64_t q0 = 0; q0 < nq;) {
        int64_t q1 = q0, bytes = 0, nodes = 0, edges = 0;
        std::vector<int64_t> nbase, ebase, node_q;
        while (q1 < nq) {
            const int64_t np = qo[q1 + 1] - qo[q1] + 1;
            if (q1 > q0 && bytes + q_bytes(np) > budget) break;
            nbase.push_back(nodes);
            ebase.push_back(edges);
            for (int64_t j = 0; j < 2 * np; ++j) node_q.push_back(q1 - q0);
            nodes += 2 * np;
            edges += bw_edges(np);
            bytes += q_bytes(np);
            ++q1;
        }
        const int64_t cq = q1 - q0;
        DevBuf bq, bn, bi, be, bk, bkey, bval, bkey2, bval2, bcnt, boff;
        RB3_TRY(bq.alloc(sizeof(int64_t) * (2 * cq + nodes) + sizeof(int32_t) * cq, st));
        int64_t *d_nbase = bq.as<int64_t>(), *d_ebase = d_nbase + cq, *d_nodeq = d_ebase + cq;
        int32_t *d_over = reinterpret_cast<int32_t *>(d_nodeq + nodes);
        RB3_CUDA_TRY(cudaMemcpyAsync(d_nbase, nbase.data(), sizeof(int64_t) * cq, cudaMemcpyHostToDevice, st));
        RB3_CUDA_TRY(cudaMemcpyAsync(d_ebase, ebase.data(), sizeof(int64_t) * cq, cudaMemcpyHostToDevice, st));
        RB3_CUDA_TRY(cudaMemcpyAsync(d_nodeq, node_q.data(), sizeof(int64_t) * nodes, cudaMemcpyHostToDevice, st));
        QDawg G;
        RB3_TRY(bn.alloc(sizeof(int32_t) * (cq + 3 * nodes + cq), st));
        G.nn = bn.as<int32_t>();
        G.uk = G.nn + cq;
        G.us = G.uk + nodes;
        G.in_off = G.us + nodes;
        RB3_TRY(be.alloc((sizeof(int32_t) * 4 + 2) * (size_t)edges + 16, st));
        G.in_pred = be.as<int32_t>();
        G.e_from = G.in_pred + edges;
        G.e_to = G.e_from + edges;
        G.o_to = G.e_to + edges;
        G.in_c = reinterpret_cast<uint8_t *>(G.o_to + edges);
        G.e_c = G.in_c + edges;
        RB3_LAUNCH(k_qdawg, (unsigned)cq, BW_THREADS, sizeof(QSmem), st, q, qoff, q0, cq, d_nbase, d_ebase, G,
                   err.as<unsigned int>());
        Kept K;
        RB3_TRY(bk.alloc((size_t)nodes * W * 32 + sizeof(int32_t) * nodes, st));
        K.k = bk.as<int64_t>();
        K.kp = K.k + nodes * W;
        K.s = K.kp + nodes * W;
        K.H = reinterpret_cast<int32_t *>(K.s + nodes * W);
        K.E = K.H + nodes * W;
        K.n = K.E + nodes * W;
        RB3_CUDA_TRY(cudaMemsetAsync(K.n, 0, sizeof(int32_t) * nodes, st));
        // every query starts at the table size its best possible score suggests (a
        // deletion closure holds about a dozen cells per unit of score), and one that
        // outgrows its table runs again, from its start, with the next size
        std::vector<int64_t> tier[3];
        for (int64_t i = 0; i < cq; ++i) {
            const int64_t best = (qo[q0 + i + 1] - qo[q0 + i]) * (int64_t)p.a;
            tier[best <= 16 ? 0 : (best <= 160 ? 1 : 2)].push_back(i);
        }
        std::vector<int32_t> over(cq);
        DevBuf bs[3];
        for (int t = 0; t < 3; ++t) {
            if (tier[t].empty()) continue;
            RB3_TRY(bs[t].alloc(sizeof(int64_t) * tier[t].size(), st));
            RB3_CUDA_TRY(
                cudaMemcpyAsync(bs[t].p, tier[t].data(), sizeof(int64_t) * tier[t].size(), cudaMemcpyHostToDevice, st));
            const int64_t *ds = bs[t].as<int64_t>();
            const int64_t ns = (int64_t)tier[t].size();
            if (t == 0)
                RB3_WITH_NS(idx->D, RB3_TRY((bw_launch<NS, BW_CAP_S, BW_WARPS_S>(idx, ds, ns, d_nbase, d_ebase, G, p, K,
                                                                                 d_over, st))));
            else if (t == 1)
                RB3_WITH_NS(idx->D, RB3_TRY((bw_launch<NS, BW_CAP_L, BW_WARPS_L>(idx, ds, ns, d_nbase, d_ebase, G, p, K,
                                                                                 d_over, st))));
            else
                RB3_WITH_NS(idx->D, RB3_TRY((bw_launch_gm<NS>(idx, ds, ns, d_nbase, d_ebase, G, p, K, d_over, st))));
            RB3_CUDA_TRY(cudaMemcpyAsync(over.data(), d_over, sizeof(int32_t) * cq, cudaMemcpyDeviceToHost, st));
            RB3_CUDA_TRY(cudaStreamSynchronize(st));
            for (int64_t i : tier[t])
                if (over[i]) {
                    if (t == 2) {
                        set_error("bwasw: query %lld left more than %d candidate cells at a node", (long long)(q0 + i),
                                  DV_CAP_G);
                        return RB3_E_CAPACITY;
                    }
                    tier[t + 1].push_back(i);
                }
        }
        unsigned int herr = 0;
        RB3_CUDA_TRY(cudaMemcpyAsync(&herr, err.p, sizeof(herr), cudaMemcpyDeviceToHost, st));
        RB3_CUDA_TRY(cudaStreamSynchronize(st));
        if (herr) {
            set_error("bwasw: a query DAWG exceeded its bounds (flags %u)", herr);
            return RB3_E_CUDA;
        }
        // records of the chunk: counts per node, offsets, keys, sort, out
        RB3_TRY(bcnt.alloc(sizeof(uint64_t) * (nodes + 1), st));
        RB3_TRY(boff.alloc(sizeof(uint64_t) * (nodes + 1), st));
        RB3_LAUNCH(k_bw_counts, nb_for(nodes, 256), 256, 0, st, d_nbase, d_nodeq, nodes, G, K, bcnt.as<uint64_t>());
        RB3_CUDA_TRY(cudaMemsetAsync(bcnt.as<uint64_t>() + nodes, 0, sizeof(uint64_t), st));
        RB3_TRY(scan_u64(bcnt.as<uint64_t>(), boff.as<uint64_t>(), nodes + 1, false, st));
        uint64_t nrec = 0;
        RB3_CUDA_TRY(cudaMemcpyAsync(&nrec, boff.as<uint64_t>() + nodes, sizeof(nrec), cudaMemcpyDeviceToHost, st));
        RB3_CUDA_TRY(cudaStreamSynchronize(st));
        total += (int64_t)nrec;
        if (nrec > 0 && written + (int64_t)nrec <= cap) {
            RB3_TRY(bkey.alloc(sizeof(uint64_t) * nrec, st));
            RB3_TRY(bval.alloc(sizeof(uint32_t) * nrec, st));
            RB3_TRY(bkey2.alloc(sizeof(uint64_t) * nrec, st));
            RB3_TRY(bval2.alloc(sizeof(uint32_t) * nrec, st));
            RB3_LAUNCH(k_bw_keys, nb_for(nodes, 256), 256, 0, st, d_nbase, d_nodeq, nodes, q0, G, K, W,
                       reinterpret_cast<const int64_t *>(boff.as<uint64_t>()), bkey.as<uint64_t>(),
                       bval.as<uint32_t>());
            bool alt = false;
            RB3_TRY(radix_sort_pairs(bkey.as<uint64_t>(), bval.as<uint32_t>(), bkey2.as<uint64_t>(),
                                     bval2.as<uint32_t>(), (int64_t)nrec, 0, 28 + ilog2(q0 + cq) + 1, st, &alt));
            RB3_LAUNCH(k_bw_out, nb_for((int64_t)nrec, 256), 256, 0, st, alt ? bkey2.as<uint64_t>() : bkey.as<uint64_t>(),
                       alt ? bval2.as<uint32_t>() : bval.as<uint32_t>(), (int64_t)nrec, K, out + 7 * written);
            written += (int64_t)nrec;
        }
        RB3_CUDA_TRY(cudaStreamSynchronize(st));
        q0 = q1;
    }
    *n_out = total;
    if (total > cap) {
        set_error("bwasw: %lld records, output capacity %lld", (long long)total, (long long)cap);
        return RB3_E_CAPACITY;
    }
    return RB3_OK;
}

}  // namespace rb3
