// Local haplotype diversity (Section "Estimating local haplotype diversity"):
// Algorithm 5, the revised BWA-SW, applied to the graph of a linear query P,
// walked from its end to its start, against the prefix DAWG of the indexed
// text (a node is the bi-interval of a string, its children its BackwardExt by
// A, C, G and T, Algorithm 3).  The result is the set of bi-intervals whose
// end-to-end alignment with P scores H > 0, best first, redundant ones dropped.
//
// One warp per query.  The W <= 32 cells kept after a query symbol sit one per
// lane; a step's candidates go into a table of the warp's own in shared memory
// (found by a warp-wide compare, written by lane 0).  Only candidates with a
// positive score enter the table: a cell whose H never rises above 0 extends
// nothing (a match, an insertion or a deletion from it stays at or below 0),
// so the cells with H > 0 and their scores are those of the full recurrence.
//   match / mismatch  H(child) = H + a or H - b (N in P mismatches everything)
//   insertion         E = max(H - q, E) - e, same node, next query position
//   deletion          F(child) = max(H - q, F) - e, same query position, until
//                     no cell's H or F rises (a worklist of cells to re-extend)
// The band keeps the W cells of largest H, ties by smaller k, k', s.  The
// filter walks the band best first and drops a cell whose [k, k+s) or
// [k', k'+s) lies inside that of a cell kept before it.
#include "align.cuh"

namespace rb3 {
namespace {

using namespace dv;

// Three table sizes: every query first runs with small tables (six warps a
// CTA, three CTAs an SM); the queries whose step outgrew theirs run again
// with the large one (2,048 cells, two warps a CTA), and those that outgrew
// that with a table of 65,534 cells in global memory.
constexpr int DV_CAP_S = 256, DV_WARPS_S = 6;
constexpr int DV_CAP_L = 2048, DV_WARPS_L = 2;
static_assert(dv_warp_bytes(DV_CAP_S) % 16 == 0 && dv_warp_bytes(DV_CAP_L) % 16 == 0,
              "per-warp tables must keep 16-byte alignment");
// Rank-all reads (two per extended cell) and cells entered, summed over
// queries since the last reset.
__device__ unsigned long long g_dv_stats[2];

// Queries sel[0 .. nsel) (all nsel = nq of them when sel is null), one warp each.
// GM: the tables in global memory (gtab, one per warp of the launch), for the
// queries that outgrew the shared-memory ones.
template <int NS, int CAP, int WARPS, bool GM>
__global__ void __launch_bounds__(32 * WARPS)
    k_diversity(OccView V, const uint8_t *__restrict__ q, const int64_t *__restrict__ qoff,
                const int64_t *__restrict__ sel, int64_t nsel, DvParams p, int64_t *__restrict__ out,
                int64_t *__restrict__ n_out, uint8_t *__restrict__ gtab) {
    extern __shared__ __align__(16) uint8_t dv_smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t wi = (int64_t)blockIdx.x * WARPS + w;
    if (wi >= nsel) return;  // the whole warp leaves together
    const int64_t qi = sel ? sel[wi] : wi;
    const DvTab T = dv_tab<CAP>(GM ? gtab + (size_t)wi * dv_warp_bytes(CAP) : dv_smem + (size_t)w * dv_warp_bytes(CAP));
    DvSt st{0, 0, 0};
    dv_clear_all<CAP>(T, st, lane);
    const int64_t q0 = qoff[qi], m = qoff[qi + 1] - q0;

    // lane r holds the r-th kept cell; before any symbol only the root (H = 0)
    int64_t ck = 0, ckp = 0, cs = V.n;
    int32_t cH = 0, cE = DV_NEG;
    int ncur = m > 0 ? 1 : 0;
    bool overflow = false;
    unsigned long long n_ext = 0, n_cells = 0;  // warp-uniform counts

    for (int64_t i = m - 1; i >= 0 && ncur > 0 && !overflow; --i) {
        const int c = q[q0 + i];
        dv_clear<CAP>(T, st, lane);
        // match / mismatch: the children of every kept cell (lane t: cell t's child by a)
        {
            int64_t xk[4] = {0, 0, 0, 0}, xkp[4] = {0, 0, 0, 0}, xs[4] = {0, 0, 0, 0};
            if (lane < ncur) dv_children<NS>(V, ck, ckp, cs, xk, xkp, xs);
            n_ext += ncur;
#pragma unroll 1
            for (int a = 1; a <= 4 && !overflow; ++a) {
                const int32_t g = cH + (a == c ? p.a : -p.b);
                const int64_t k = dv_pick(xk, a - 1), kp = dv_pick(xkp, a - 1), s = dv_pick(xs, a - 1);
                dv_upsert_batch<CAP>(T, st, lane < ncur && s > 0 && g > 0, k, kp, s, g, DV_NEG, DV_NEG, lane, overflow);
            }
        }
        // insertion: the query symbol against a gap, the node unchanged
        {
            const int32_t ev = max(cH - p.q, cE) - p.e;
            if (!overflow) dv_upsert_batch<CAP>(T, st, lane < ncur && ev > 0, ck, ckp, cs, ev, ev, DV_NEG, lane, overflow);
        }
        // deletion: a text symbol against a gap, until no cell is left to extend
        dv_close<NS, CAP>(V, T, st, p, lane, overflow, n_ext);
        const int tn = st.tn;
        n_cells += tn;
        if (overflow) break;
        // the band (a warp sort, or a score histogram and sorts of what it singles out)
        const int keep = min(tn, p.W);
        int64_t nk = 0, nkp = 0, ns = 0;
        int32_t nH = 0, nE = DV_NEG;
        {
            const int j = dv_band<CAP>(T, tn, p.W, lane);
            if (lane < keep) {
                nk = T.k[j];
                nkp = T.kp[j];
                ns = T.s[j];
                nH = T.H[j];
                nE = T.E[j];
            }
        }
        ck = nk;
        ckp = nkp;
        cs = ns;
        cH = nH;
        cE = nE;
        ncur = keep;
        __syncwarp();  // every lane is done with the table before the next step refills it
    }

    if (lane == 0) {
        atomicAdd(&g_dv_stats[0], 2 * n_ext);
        atomicAdd(&g_dv_stats[1], n_cells);
    }
    if (overflow) {
        if (lane == 0) n_out[qi] = -1;
        return;
    }
    // redundancy filter over the band, best first
    unsigned kept_mask = ncur >= 32 ? DV_FULL : ((1u << ncur) - 1);
    if (p.redundancy) {
        kept_mask = 0;
        for (int r = 0; r < ncur; ++r) {
            const int64_t rk = __shfl_sync(DV_FULL, ck, r);
            const int64_t rkp = __shfl_sync(DV_FULL, ckp, r);
            const int64_t rs = __shfl_sync(DV_FULL, cs, r);
            const bool inside = ((kept_mask >> lane) & 1) &&
                                ((rk >= ck && rk + rs <= ck + cs) || (rkp >= ckp && rkp + rs <= ckp + cs));
            if (__ballot_sync(DV_FULL, inside) == 0) kept_mask |= 1u << r;
        }
    }
    int64_t *o = out + qi * (int64_t)p.W * 4;
    if ((kept_mask >> lane) & 1) {
        const int pos = __popc(kept_mask & ((1u << lane) - 1));
        o[4 * pos + 0] = ck;
        o[4 * pos + 1] = ckp;
        o[4 * pos + 2] = cs;
        o[4 * pos + 3] = cH;
    }
    if (lane == 0) n_out[qi] = __popc(kept_mask);
}

}  // namespace

int diversity_stats(int64_t out[2], bool reset) {
    unsigned long long h[2];
    RB3_CUDA_TRY(cudaMemcpyFromSymbol(h, g_dv_stats, sizeof(h)));
    out[0] = (int64_t)h[0];
    out[1] = (int64_t)h[1];
    if (reset) {
        const unsigned long long z[2] = {0, 0};
        RB3_CUDA_TRY(cudaMemcpyToSymbol(g_dv_stats, z, sizeof(z)));
    }
    return RB3_OK;
}

template <int NS, int CAP, int WARPS>
static int dv_launch(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, const int64_t *sel, int64_t nsel,
                     const DvParams &p, int64_t *out, int64_t *n_out, cudaStream_t st) {
    const size_t smem = WARPS * dv_warp_bytes(CAP);
    auto kern = k_diversity<NS, CAP, WARPS, false>;
    RB3_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned grid = (unsigned)((nsel + WARPS - 1) / WARPS);
    RB3_LAUNCH(kern, grid, 32 * WARPS, smem, st, occ_view(idx), q, qoff, sel, nsel, p, out, n_out,
               (uint8_t *)nullptr);
    return RB3_OK;
}

// The global-memory tier: one warp per CTA, at most DV_GM_WARPS tables at once.
constexpr int64_t DV_GM_WARPS = 1024;
template <int NS>
static int dv_launch_gm(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, const int64_t *sel, int64_t nsel,
                        const DvParams &p, int64_t *out, int64_t *n_out, cudaStream_t st) {
    const int64_t nw = nsel < DV_GM_WARPS ? nsel : DV_GM_WARPS;
    DevBuf tab;
    RB3_TRY(tab.alloc(dv_warp_bytes(DV_CAP_G) * (size_t)nw, st));
    for (int64_t b = 0; b < nsel; b += nw) {
        const int64_t n = nsel - b < nw ? nsel - b : nw;
        RB3_LAUNCH((k_diversity<NS, DV_CAP_G, 1, true>), (unsigned)n, 32, 0, st, occ_view(idx), q, qoff, sel + b, n, p,
                   out, n_out, tab.as<uint8_t>());
    }
    return RB3_OK;
}

int diversity_impl(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, int64_t nq, int64_t total_q,
                   const int32_t prm[6], int64_t *out, int64_t *n_out, cudaStream_t st) {
    RB3_TRY(check_codes(q, total_q, st));
    if (nq == 0) return RB3_OK;
    const DvParams p{prm[0], prm[1], prm[2], prm[3], prm[4], prm[5]};
    Phase ph("search.diversity", st);
    RB3_WITH_NS(idx->D, RB3_TRY((dv_launch<NS, DV_CAP_S, DV_WARPS_S>(idx, q, qoff, nullptr, nq, p, out, n_out, st))));
    // the queries that outgrew the small table, again with the large one
    std::vector<int64_t> n(nq), sel;
    RB3_CUDA_TRY(cudaMemcpyAsync(n.data(), n_out, sizeof(int64_t) * nq, cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < nq; ++i)
        if (n[i] < 0) sel.push_back(i);
    if (sel.empty()) return RB3_OK;
    DevBuf ds;
    RB3_TRY(ds.alloc(sizeof(int64_t) * sel.size(), st));
    RB3_CUDA_TRY(cudaMemcpyAsync(ds.p, sel.data(), sizeof(int64_t) * sel.size(), cudaMemcpyHostToDevice, st));
    RB3_WITH_NS(idx->D, RB3_TRY((dv_launch<NS, DV_CAP_L, DV_WARPS_L>(idx, q, qoff, ds.as<int64_t>(),
                                                                     (int64_t)sel.size(), p, out, n_out, st))));
    // those that outgrew the large table too, with the global-memory one
    RB3_CUDA_TRY(cudaMemcpyAsync(n.data(), n_out, sizeof(int64_t) * nq, cudaMemcpyDeviceToHost, st));
    RB3_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int64_t> sel2;
    for (int64_t i = 0; i < nq; ++i)
        if (n[i] < 0) sel2.push_back(i);
    if (sel2.empty()) return RB3_OK;
    DevBuf ds2;
    RB3_TRY(ds2.alloc(sizeof(int64_t) * sel2.size(), st));
    RB3_CUDA_TRY(cudaMemcpyAsync(ds2.p, sel2.data(), sizeof(int64_t) * sel2.size(), cudaMemcpyHostToDevice, st));
    RB3_WITH_NS(idx->D, RB3_TRY((dv_launch_gm<NS>(idx, q, qoff, ds2.as<int64_t>(), (int64_t)sel2.size(), p, out,
                                                  n_out, st))));
    return RB3_OK;  // ds and ds2 are freed in stream order after the launches
}

}  // namespace rb3
