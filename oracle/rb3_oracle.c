/*
 * rb3 oracle -- a plain, slow, CPU-only restatement of what the BWT build,
 * merge and search path computes, written from H. Li, "BWT construction and
 * search at the terabase scale" (arXiv 2409.00613).
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  The CUDA library never
 * links, includes or calls it; the two share no code, header, table or helper.
 *
 * Symbol codes: $=0 A=1 C=2 G=3 T=4 N=5.  Code order is the symbol order
 * $_0 < ... < $_{m-1} < A < C < G < T < N of Section "BWT construction".
 * Every sentinel is printed as 0 in a BWT (Section "Basic concepts"); in a
 * concatenated text T the i-th sentinel is the i-th 0 from the left, so
 * sentinel order is position order.
 *
 * Every function says which passage it follows.  Nothing here is blocked,
 * fused or reordered beyond what the cited definition or algorithm states.
 * All counts and positions are int64.
 */
#define _GNU_SOURCE
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_SIGMA 6 /* |Sigma'| = {$,A,C,G,T,N} */

/* Watson-Crick complement, Section "Double-strand BWT": the complements of
 * $,A,C,G,T,N are $,T,G,C,A,N. */
static const uint8_t orc_comp[ORC_SIGMA] = {0, 4, 3, 2, 1, 5};

int orc_version(void) { return 1; }

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Concatenation.  Section "Basic concepts": T = P_0 $_0 P_1 $_1 ... ;
 * Section "Double-strand BWT": T~ = P_0 $ rc(P_0) $ P_1 $ rc(P_1) $ ...
 * seq holds the strings back to back (codes 1..5), len their lengths.
 * Returns n = |T|; writes T when T != NULL.
 * ---------------------------------------------------------------------- */
int64_t orc_concat(const uint8_t *seq, const int64_t *len, int64_t nseq, int both, uint8_t *T)
{
    int64_t n = 0, off = 0;
    for (int64_t i = 0; i < nseq; ++i) {
        const uint8_t *P = seq + off;
        int64_t L = len[i];
        if (T) {
            for (int64_t j = 0; j < L; ++j) T[n + j] = P[j];
            T[n + L] = 0;
        }
        n += L + 1;
        if (both) {
            if (T) {
                /* reverse complement: rc(P)[j] = comp(P[L-1-j]) */
                for (int64_t j = 0; j < L; ++j) T[n + j] = orc_comp[P[L - 1 - j]];
                T[n + L] = 0;
            }
            n += L + 1;
        }
        off += L;
    }
    return n;
}

/* ------------------------------------------------------------------------
 * O1: suffix array by a comparison sort of all suffixes (Section "Basic
 * concepts": S(i) is the start of the i-th smallest suffix).  Two suffixes are
 * compared symbol by symbol; letters by code; a sentinel is below every
 * letter; two sentinels met at the same offset are ordered by their position
 * in T (sentinel $_i precedes $_j in T iff i < j).  Since the last symbol of
 * T is a sentinel, every comparison of two distinct suffixes ends.
 * ---------------------------------------------------------------------- */
static int cmp_suffix(const void *pa, const void *pb, void *ctx)
{
    const uint8_t *T = (const uint8_t *)ctx;
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    if (a == b) return 0;
    for (int64_t t = 0;; ++t) {
        uint8_t ca = T[a + t], cb = T[b + t];
        if (ca != cb) return ca < cb ? -1 : 1;
        if (ca == 0) return (a + t) < (b + t) ? -1 : 1; /* both sentinels */
    }
}

void orc_suffix_array(const uint8_t *T, int64_t n, int64_t *SA)
{
    for (int64_t i = 0; i < n; ++i) SA[i] = i;
    qsort_r(SA, (size_t)n, sizeof(int64_t), cmp_suffix, (void *)T);
}

/* B[i] = T[S(i)-1] with T[-1] = T[n-1] (Section "Basic concepts"). */
void orc_bwt_from_sa(const uint8_t *T, int64_t n, const int64_t *SA, uint8_t *B)
{
    for (int64_t i = 0; i < n; ++i) B[i] = SA[i] == 0 ? T[n - 1] : T[SA[i] - 1];
}

void orc_bwt(const uint8_t *T, int64_t n, uint8_t *B)
{
    int64_t *SA = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    orc_suffix_array(T, n, SA);
    orc_bwt_from_sa(T, n, SA, B);
    free(SA);
}

/* ------------------------------------------------------------------------
 * Plain rank table (Table 1): C_B(a) = |{i : B[i] < a}|,
 * rank_B(a,k) = |{i < k : B[i] = a}|, pi_B(a,k) = C_B(a) + rank_B(a,k).
 * Counts are stored for every 64th offset; the rest is counted by a loop.
 * ---------------------------------------------------------------------- */
typedef struct {
    const uint8_t *B;
    int64_t n;
    int64_t C[ORC_SIGMA + 1];
    int64_t *cp; /* cp[(k/64)*6 + a] = rank_B(a, 64*(k/64)) */
} orc_rank_t;

static orc_rank_t *rank_new(const uint8_t *B, int64_t n)
{
    orc_rank_t *r = (orc_rank_t *)calloc(1, sizeof(orc_rank_t));
    int64_t nb = n / 64 + 1, cnt[ORC_SIGMA] = {0};
    r->B = B;
    r->n = n;
    r->cp = (int64_t *)malloc(sizeof(int64_t) * ORC_SIGMA * (size_t)nb);
    for (int64_t i = 0; i <= n; ++i) {
        if ((i & 63) == 0)
            for (int a = 0; a < ORC_SIGMA; ++a) r->cp[(i >> 6) * ORC_SIGMA + a] = cnt[a];
        if (i < n) ++cnt[B[i]];
    }
    r->C[0] = 0;
    for (int a = 0; a < ORC_SIGMA; ++a) r->C[a + 1] = r->C[a] + cnt[a];
    return r;
}

static void rank_free(orc_rank_t *r)
{
    if (r) { free(r->cp); free(r); }
}

static inline int64_t rank_get(const orc_rank_t *r, int a, int64_t k)
{
    int64_t v = r->cp[(k >> 6) * ORC_SIGMA + a];
    for (int64_t i = k & ~(int64_t)63; i < k; ++i) v += r->B[i] == a;
    return v;
}

static inline int64_t pi_B(const orc_rank_t *r, int a, int64_t k) { return r->C[a] + rank_get(r, a, k); }

/* C_B(a) for a = 0..6 (C[6] = n) and the symbol counts. */
void orc_counts(const uint8_t *B, int64_t n, int64_t *C7)
{
    int64_t cnt[ORC_SIGMA] = {0};
    for (int64_t i = 0; i < n; ++i) ++cnt[B[i]];
    C7[0] = 0;
    for (int a = 0; a < ORC_SIGMA; ++a) C7[a + 1] = C7[a] + cnt[a];
}

/* Occ checkpoints: occ[j*6 + a] = rank_B(a, j*D) for j = 0 .. n/D. */
void orc_occ_table(const uint8_t *B, int64_t n, int64_t D, int64_t *occ)
{
    int64_t cnt[ORC_SIGMA] = {0};
    for (int64_t i = 0; i <= n; ++i) {
        if (i % D == 0)
            for (int a = 0; a < ORC_SIGMA; ++a) occ[(i / D) * ORC_SIGMA + a] = cnt[a];
        if (i < n) ++cnt[B[i]];
    }
}

/* ------------------------------------------------------------------------
 * Retrieve (the LF decoding in Section "Basic concepts": B[pi(i)] precedes
 * B[i] in T).  Decodes string i (0 <= i < m) into out (reversed twice so it
 * reads forward); returns its length, or -1 if more than cap symbols.
 * ---------------------------------------------------------------------- */
int64_t orc_retrieve(const uint8_t *B, int64_t n, int64_t i, uint8_t *out, int64_t cap)
{
    orc_rank_t *r = rank_new(B, n);
    int64_t L = 0, k = i;
    while (B[k] != 0) {
        if (L >= cap) { rank_free(r); return -1; }
        out[L++] = B[k];
        k = pi_B(r, B[k], k);
    }
    for (int64_t a = 0, b = L - 1; a < b; ++a, --b) { uint8_t t = out[a]; out[a] = out[b]; out[b] = t; }
    rank_free(r);
    return L;
}

/* ------------------------------------------------------------------------
 * O2: LF-decode certificate.  B is the BWT of the string list held in T
 * (T = P_0 $ P_1 $ ..., as made by orc_concat) iff
 *   (i)   |B| = |T| and B has the symbol counts of T,
 *   (ii)  for every i < m, LF-walking from row i spells P_i backwards and
 *         stops at a row holding $ (Retrieve),
 *   (iii) the walks visit every row of B exactly once.
 * Why: LF maps the rows holding a given symbol, in order, onto that symbol's
 * block of rows (Table 1: pi(k) = pi_B(B[k],k)); with (ii) and (iii) the row
 * walked to at step t of walk i stands for the suffix P_i[|P_i|-t..]$_i, and
 * induction on suffix length shows the rows are then in suffix order, which
 * is the definition B[i] = T[S(i)-1].
 * Returns 0 if certified, else a nonzero reason code.
 * ---------------------------------------------------------------------- */
int orc_certify(const uint8_t *B, int64_t n, const uint8_t *T, int64_t nT, int nthreads)
{
    if (n != nT) return 1;
    int64_t cB[ORC_SIGMA] = {0}, cT[ORC_SIGMA] = {0};
    for (int64_t i = 0; i < n; ++i) {
        if (B[i] >= ORC_SIGMA || T[i] >= ORC_SIGMA) return 2;
        ++cB[B[i]];
        ++cT[T[i]];
    }
    for (int a = 0; a < ORC_SIGMA; ++a)
        if (cB[a] != cT[a]) return 2;
    int64_t m = cT[0];
    if (n == 0) return 0;
    if (T[n - 1] != 0) return 2;
    /* end[i] = position of the i-th sentinel in T */
    int64_t *end = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    for (int64_t i = 0, j = 0; i < n; ++i)
        if (T[i] == 0) end[j++] = i;
    orc_rank_t *r = rank_new(B, n);
    uint8_t *seen = (uint8_t *)calloc((size_t)n, 1);
    int bad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
#endif
    for (int64_t i = 0; i < m; ++i) {
        int64_t start = i == 0 ? 0 : end[i - 1] + 1;
        int64_t k = i, t = end[i] - 1;
        for (;;) {
            if (__atomic_exchange_n(&seen[k], (uint8_t)1, __ATOMIC_RELAXED)) { bad |= 4; break; }
            uint8_t c = B[k];
            if (t < start) {
                if (c != 0) bad |= 8;
                break;
            }
            if (c != T[t]) { bad |= 16; break; }
            k = pi_B(r, c, k);
            --t;
        }
    }
    int64_t nseen = 0;
    for (int64_t i = 0; i < n; ++i) nseen += seen[i];
    if (!bad && nseen != n) bad = 32;
    free(seen);
    free(end);
    rank_free(r);
    return bad;
}

/* ------------------------------------------------------------------------
 * O3: Algorithm 1 (AppendBWT), taken step by step.  Inserts B2 into B1 and
 * writes the merged BWT (n1+n2 symbols) to M.
 *   m1, m2   <- number of $ in B1, B2
 *   R(k)     <- (B2[k], pi_{B2}(B2[k],k))            for every k
 *   for each i < m2 (the walks are independent; they run in parallel as in
 *   the paper): k <- i, l <- m1; repeat: (a,k') <- R(k); R(k) <- (a,k+l);
 *   k <- k'; l <- pi_{B1}(a,l) until a = $
 *   insert a after k symbols of B1 for every (a,k) in R, in increasing k.
 * The insertion is done by writing the merged string left to right: row q of
 * M takes the next B2 symbol when q is the next inserted position, else the
 * next B1 symbol.
 * pos_out (optional, n2 entries) receives the merged row of every B2 row.
 * ---------------------------------------------------------------------- */
void orc_merge(const uint8_t *B1, int64_t n1, const uint8_t *B2, int64_t n2, uint8_t *M,
               int64_t *pos_out, int nthreads)
{
    orc_rank_t *r1 = rank_new(B1, n1), *r2 = rank_new(B2, n2);
    int64_t m1 = r1->C[1] - r1->C[0], m2 = r2->C[1] - r2->C[0];
    int64_t *Rk = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n2 > 0 ? n2 : 1));
    int64_t *pos = pos_out ? pos_out : (int64_t *)malloc(sizeof(int64_t) * (size_t)(n2 > 0 ? n2 : 1));
    for (int64_t k = 0; k < n2; ++k) Rk[k] = pi_B(r2, B2[k], k);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = 0; i < m2; ++i) {
        int64_t k = i, l = m1;
        uint8_t a;
        do {
            a = B2[k];
            int64_t kn = Rk[k];
            pos[k] = k + l;
            k = kn;
            l = pi_B(r1, a, l);
        } while (a != 0);
    }
    int64_t j = 0, k = 0;
    for (int64_t q = 0; q < n1 + n2; ++q) {
        if (k < n2 && pos[k] == q) M[q] = B2[k++];
        else M[q] = B1[j++];
    }
    if (!pos_out) free(pos);
    free(Rk);
    rank_free(r1);
    rank_free(r2);
}

/* ------------------------------------------------------------------------
 * Incremental build: the string list is cut into consecutive groups of g
 * strings; the BWT of each group's concatenation is built with O1 and the
 * groups are appended one after another with Algorithm 1 (O3), which is the
 * driver loop of Section "Methods" (build a partial BWT, merge, repeat).
 * Writes the BWT of the whole list's concatenation to B and returns n.
 * ---------------------------------------------------------------------- */
int64_t orc_build_incremental(const uint8_t *seq, const int64_t *len, int64_t nseq, int both,
                              int64_t g, uint8_t *B, int nthreads)
{
    if (g < 1) g = 1;
    int64_t ngroups = (nseq + g - 1) / g;
    uint8_t **Bg = (uint8_t **)calloc((size_t)(ngroups > 0 ? ngroups : 1), sizeof(uint8_t *));
    int64_t *ng = (int64_t *)calloc((size_t)(ngroups > 0 ? ngroups : 1), sizeof(int64_t));
    int64_t *soff = (int64_t *)calloc((size_t)(nseq + 1), sizeof(int64_t));
    for (int64_t i = 0; i < nseq; ++i) soff[i + 1] = soff[i] + len[i];
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t G = 0; G < ngroups; ++G) {
        int64_t s0 = G * g, s1 = s0 + g < nseq ? s0 + g : nseq;
        int64_t n = orc_concat(seq + soff[s0], len + s0, s1 - s0, both, NULL);
        uint8_t *T = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
        orc_concat(seq + soff[s0], len + s0, s1 - s0, both, T);
        Bg[G] = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
        orc_bwt(T, n, Bg[G]);
        ng[G] = n;
        free(T);
    }
    int64_t ntot = 0;
    for (int64_t G = 0; G < ngroups; ++G) ntot += ng[G];
    uint8_t *cur = (uint8_t *)malloc((size_t)(ntot > 0 ? ntot : 1));
    uint8_t *tmp = (uint8_t *)malloc((size_t)(ntot > 0 ? ntot : 1));
    int64_t ncur = 0;
    for (int64_t G = 0; G < ngroups; ++G) {
        orc_merge(cur, ncur, Bg[G], ng[G], tmp, NULL, nthreads);
        uint8_t *t = cur; cur = tmp; tmp = t;
        ncur += ng[G];
        free(Bg[G]);
    }
    memcpy(B, cur, (size_t)ncur);
    free(cur); free(tmp); free(Bg); free(ng); free(soff);
    return ncur;
}

/* ------------------------------------------------------------------------
 * Backward search (Section "Suffix array interval and backward search"):
 * start from [0,n) and apply lo(aP) = pi_B(a,lo(P)), hi(aP) = pi_B(a,hi(P))
 * from the last symbol of P to the first.  Writes lo,hi for every query.
 * Queries are back to back in q; query i is q[qoff[i] .. qoff[i+1]).
 * ---------------------------------------------------------------------- */
void orc_backward_search(const uint8_t *B, int64_t n, const uint8_t *q, const int64_t *qoff, int64_t nq,
                         int64_t *lohi)
{
    orc_rank_t *r = rank_new(B, n);
    for (int64_t i = 0; i < nq; ++i) {
        int64_t lo = 0, hi = n;
        for (int64_t j = qoff[i + 1] - 1; j >= qoff[i]; --j) {
            lo = pi_B(r, q[j], lo);
            hi = pi_B(r, q[j], hi);
        }
        lohi[2 * i] = lo;
        lohi[2 * i + 1] = hi;
    }
    rank_free(r);
}

/* ------------------------------------------------------------------------
 * Algorithm 3.  BackwardExt: for all b < comp(a) (b may be $):
 *   k' += pi_B(comp(b), k+s) - pi_B(comp(b), k);
 *   s <- pi_B(a,k+s) - pi_B(a,k); k <- pi_B(a,k).
 * ForwardExt(B,(k,k',s),a) = swap(BackwardExt(B,(k',k,s),comp(a))).
 * ---------------------------------------------------------------------- */
typedef struct { int64_t k, kp, s; } biint_t;

static biint_t backward_ext(const orc_rank_t *r, biint_t x, int a)
{
    int ac = orc_comp[a];
    for (int b = 0; b < ac; ++b) {
        int bc = orc_comp[b];
        x.kp += pi_B(r, bc, x.k + x.s) - pi_B(r, bc, x.k);
    }
    int64_t lo = pi_B(r, a, x.k), hi = pi_B(r, a, x.k + x.s);
    x.s = hi - lo;
    x.k = lo;
    return x;
}

static biint_t forward_ext(const orc_rank_t *r, biint_t x, int a)
{
    biint_t y = {x.kp, x.k, x.s};
    y = backward_ext(r, y, orc_comp[a]);
    biint_t z = {y.kp, y.k, y.s};
    return z;
}

/* Exposed for pins: one BackwardExt / ForwardExt from (k,k',s). */
void orc_ext(const uint8_t *B, int64_t n, int64_t *kks, int a, int forward)
{
    orc_rank_t *r = rank_new(B, n);
    biint_t x = {kks[0], kks[1], kks[2]};
    x = forward ? forward_ext(r, x, a) : backward_ext(r, x, a);
    kks[0] = x.k; kks[1] = x.kp; kks[2] = x.s;
    rank_free(r);
}

/* ------------------------------------------------------------------------
 * Algorithm 4 (FindSMEM1 / FindSMEM), with these readings of the listing:
 *   - "e <- j" after the forward loop is C for-loop semantics: e = |P| when
 *     the loop runs out, e = j when it breaks at j; the SMEM's bi-interval is
 *     the one held before the failing ForwardExt;
 *   - when e = |P| the third loop would read P[|P|]: return |P| instead;
 *   - when the third loop runs out without returning, return i+1.
 * Records are (qid, start, end, k, k', s), queries in order, starts ascending.
 * Returns the number of SMEMs; writes at most cap records.
 * ---------------------------------------------------------------------- */
static int64_t find_smem1(const orc_rank_t *r, const uint8_t *P, int64_t len, int64_t i, int64_t ell,
                          int64_t smin, int64_t qid, int64_t *out, int64_t *nout, int64_t cap)
{
    if (i + ell > len) return len;
    biint_t x = {0, 0, r->n};
    for (int64_t j = i + ell - 1; j >= i; --j) {
        x = backward_ext(r, x, P[j]);
        if (x.s < smin) return j + 1;
    }
    int64_t j;
    for (j = i + ell; j < len; ++j) {
        biint_t y = forward_ext(r, x, P[j]);
        if (y.s < smin) break;
        x = y;
    }
    int64_t e = j;
    if (*nout < cap) {
        int64_t *o = out + 6 * (*nout);
        o[0] = qid; o[1] = i; o[2] = e; o[3] = x.k; o[4] = x.kp; o[5] = x.s;
    }
    ++*nout;
    if (e == len) return len;
    biint_t z = {0, 0, r->n};
    for (j = e; j >= i + 1; --j) {
        z = backward_ext(r, z, P[j]);
        if (z.s < smin) return j + 1;
    }
    return i + 1;
}

int64_t orc_smem(const uint8_t *B, int64_t n, const uint8_t *q, const int64_t *qoff, int64_t nq,
                 int64_t ell, int64_t smin, int64_t *out, int64_t cap)
{
    orc_rank_t *r = rank_new(B, n);
    int64_t nout = 0;
    for (int64_t t = 0; t < nq; ++t) {
        const uint8_t *P = q + qoff[t];
        int64_t len = qoff[t + 1] - qoff[t], i = 0;
        do {
            i = find_smem1(r, P, len, i, ell, smin, t, out, &nout, cap);
        } while (i < len);
    }
    rank_free(r);
    return nout;
}

/* Same as orc_smem, queries spread over threads; each thread appends into its
 * own list and the lists are concatenated in query order. */
/* ------------------------------------------------------------------------
 * Section "Estimating local haplotype diversity": Algorithm 5 (BWA-SW) on
 * the graph of a linear query P, traversed from its end to its start, against
 * the prefix DAWG of the text: a node is the bi-interval (k, k', s) of a
 * string occurring in T, its children its BackwardExt by A, C, G and T.
 * Readings of what the paper leaves open:
 *   - nodes are told apart by the whole bi-interval: strings with one SA
 *     interval but different k' (x and xz when every x is followed by z) are
 *     two nodes, so that the (k, k', s) reported is well defined;
 *   - scores: match +a, mismatch -b (N in P mismatches every symbol; no node
 *     has an N child), a gap of length L costs q + L*e, i.e. E and F become
 *     max(H - q, E or F) - e, as in the recurrences of Section "Finding
 *     inexact matches with BWA-SW";
 *   - the cells after P[i..m) are the nodes with H > 0; before any symbol
 *     the root (the empty string, H = 0) is the only cell;
 *   - the deletion loop of Algorithm 5 runs to its closure: a cell whose H
 *     rises by a deletion is extended again;
 *   - the band keeps the W cells of largest H, ties by smaller k, then k',
 *     then s (W = 0: no band);
 *   - the result, the cells after P[0], is ordered by H descending, then k,
 *     k', s; with redundancy set, a cell is dropped when its [k, k+s) or its
 *     [k', k'+s) lies inside that of a cell kept before it.
 * Writes (k, k', s, H) records (at most cap) and returns their number.
 * Test infrastructure: small inputs, lists searched linearly.
 * ---------------------------------------------------------------------- */
typedef struct { int64_t k, kp, s, H, E, F; } dcell_t;
#define DNEG (INT64_MIN / 4)

typedef struct { dcell_t *c; int64_t n, cap; } dlist_t;

static int64_t dlist_get(dlist_t *L, biint_t v)
{
    for (int64_t i = 0; i < L->n; ++i)
        if (L->c[i].k == v.k && L->c[i].kp == v.kp && L->c[i].s == v.s) return i;
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 64;
        L->c = (dcell_t *)realloc(L->c, sizeof(dcell_t) * L->cap);
    }
    dcell_t z = {v.k, v.kp, v.s, DNEG, DNEG, DNEG};
    L->c[L->n] = z;
    return L->n++;
}

static int dcell_cmp(const void *pa, const void *pb)
{
    const dcell_t *x = (const dcell_t *)pa, *y = (const dcell_t *)pb;
    if (x->H != y->H) return x->H > y->H ? -1 : 1;
    if (x->k != y->k) return x->k < y->k ? -1 : 1;
    if (x->kp != y->kp) return x->kp < y->kp ? -1 : 1;
    if (x->s != y->s) return x->s < y->s ? -1 : 1;
    return 0;
}

static int64_t dmax(int64_t x, int64_t y) { return x > y ? x : y; }

static int64_t diversity_one(const orc_rank_t *r, int64_t n, const uint8_t *P, int64_t m, int64_t a, int64_t b,
                             int64_t q, int64_t e, int64_t W, int redundancy, int64_t *out, int64_t cap)
{
    dlist_t cur = {0, 0, 0}, nxt = {0, 0, 0};
    biint_t root = {0, 0, n};
    int64_t ri = dlist_get(&cur, root);
    cur.c[ri].H = 0;
    for (int64_t i = m - 1; i >= 0; --i) {
        nxt.n = 0;
        for (int64_t t = 0; t < cur.n; ++t) { /* match or mismatch: a child per symbol */
            const dcell_t c = cur.c[t];
            for (int x = 1; x <= 4; ++x) {
                biint_t v = backward_ext(r, (biint_t){c.k, c.kp, c.s}, x);
                if (v.s == 0) continue;
                int64_t j = dlist_get(&nxt, v);
                nxt.c[j].H = dmax(nxt.c[j].H, c.H + (x == P[i] ? a : -b));
            }
        }
        for (int64_t t = 0; t < cur.n; ++t) { /* insertion: P[i] against a gap, same node */
            const dcell_t c = cur.c[t];
            const int64_t ev = dmax(c.H - q, c.E) - e;
            int64_t j = dlist_get(&nxt, (biint_t){c.k, c.kp, c.s});
            nxt.c[j].E = dmax(nxt.c[j].E, ev);
            nxt.c[j].H = dmax(nxt.c[j].H, nxt.c[j].E);
        }
        for (int changed = 1; changed;) { /* deletion: a text symbol against a gap, to the closure */
            changed = 0;
            for (int64_t t = 0; t < nxt.n; ++t) {
                if (nxt.c[t].H <= 0) continue;
                for (int x = 1; x <= 4; ++x) {
                    const dcell_t c = nxt.c[t];
                    biint_t v = backward_ext(r, (biint_t){c.k, c.kp, c.s}, x);
                    if (v.s == 0) continue;
                    const int64_t fv = dmax(c.H - q, c.F) - e;
                    int64_t j = dlist_get(&nxt, v);
                    if (fv > nxt.c[j].F) {
                        nxt.c[j].F = fv;
                        nxt.c[j].H = dmax(nxt.c[j].H, fv);
                        changed = 1;
                    }
                }
            }
        }
        cur.n = 0;
        for (int64_t t = 0; t < nxt.n; ++t) /* the cells: H > 0 */
            if (nxt.c[t].H > 0) {
                int64_t j = dlist_get(&cur, (biint_t){nxt.c[t].k, nxt.c[t].kp, nxt.c[t].s});
                cur.c[j] = nxt.c[t];
            }
        if (W > 0 && cur.n > W) { /* the band */
            qsort(cur.c, (size_t)cur.n, sizeof(dcell_t), dcell_cmp);
            cur.n = W;
        }
        if (cur.n == 0) break;
    }
    if (m == 0) cur.n = 0; /* no symbol consumed: only the root, H = 0 */
    qsort(cur.c, (size_t)cur.n, sizeof(dcell_t), dcell_cmp);
    int64_t nout = 0;
    dcell_t *kept = (dcell_t *)malloc(sizeof(dcell_t) * (cur.n ? cur.n : 1));
    for (int64_t t = 0; t < cur.n; ++t) {
        const dcell_t c = cur.c[t];
        int drop = 0;
        for (int64_t u = 0; redundancy && u < nout && !drop; ++u)
            drop = (c.k >= kept[u].k && c.k + c.s <= kept[u].k + kept[u].s) ||
                   (c.kp >= kept[u].kp && c.kp + c.s <= kept[u].kp + kept[u].s);
        if (drop) continue;
        kept[nout] = c;
        if (nout < cap) {
            int64_t *o = out + 4 * nout;
            o[0] = c.k; o[1] = c.kp; o[2] = c.s; o[3] = c.H;
        }
        ++nout;
    }
    free(kept);
    free(cur.c);
    free(nxt.c);
    return nout;
}

int64_t orc_diversity(const uint8_t *B, int64_t n, const uint8_t *P, int64_t m, int64_t a, int64_t b, int64_t q,
                      int64_t e, int64_t W, int redundancy, int64_t *out, int64_t cap)
{
    orc_rank_t *r = rank_new(B, n);
    const int64_t nout = diversity_one(r, n, P, m, a, b, q, e, W, redundancy, out, cap);
    rank_free(r);
    return nout;
}

/* orc_diversity for the queries q[qoff[i] .. qoff[i+1]), one rank table for
 * all of them: query i's records (at most W, W >= 1) at out + 4*W*i, their
 * number in n_out[i]. */
void orc_diversity_many(const uint8_t *B, int64_t n, const uint8_t *qs, const int64_t *qoff, int64_t nq, int64_t a,
                        int64_t b, int64_t q, int64_t e, int64_t W, int redundancy, int64_t *out, int64_t *n_out)
{
    orc_rank_t *r = rank_new(B, n);
    for (int64_t i = 0; i < nq; ++i)
        n_out[i] = diversity_one(r, n, qs + qoff[i], qoff[i + 1] - qoff[i], a, b, q, e, W, redundancy,
                                 out + 4 * W * i, W);
    rank_free(r);
}

/* ------------------------------------------------------------------------
 * Section "Finding inexact matches with BWA-SW": Algorithm 5 between the prefix
 * DAWG of a query P, stored explicitly (nodes are the SA intervals (k, s) of
 * P's substrings in the BWT BP of the one-string text P$, an edge x -> cx for
 * every symbol c A..N with cx in P), and the prefix DAWG of the indexed text,
 * walked implicitly by BackwardExt (nodes are bi-intervals, children by A..T).
 * Query nodes are taken in a topological order (Kahn's algorithm over the
 * edges); the pair of roots starts with H = 0 and is extended although H is
 * not positive; every other cell is kept while H > 0.  Scores, gaps, node
 * identity, the deletion closure and the band (W, 0 = none, after the
 * deletions of each query node) are those of orc_diversity.
 * Writes (uk, us, k, k', s, H) for every kept cell of every query node but
 * the root (at most cap records) and returns their number.
 * Test infrastructure: small inputs, lists searched linearly.
 * ---------------------------------------------------------------------- */
typedef struct { int64_t k, s; } pnode_t;

int64_t orc_bwasw(const uint8_t *B, int64_t n, const uint8_t *BP, int64_t np, int64_t a, int64_t b, int64_t q,
                  int64_t e, int64_t W, int64_t *out, int64_t cap)
{
    orc_rank_t *r = rank_new(B, n), *rp = rank_new(BP, np);
    /* the query DAWG: nodes by breadth-first BackwardExt from the root */
    int64_t nn = 1, ncap = 64, ne = 0, ecap = 64;
    pnode_t *nodes = (pnode_t *)malloc(sizeof(pnode_t) * ncap);
    int64_t(*edge)[3] = (int64_t(*)[3])malloc(sizeof(int64_t[3]) * ecap); /* from, to, symbol */
    nodes[0].k = 0;
    nodes[0].s = np;
    for (int64_t u = 0; u < nn; ++u)
        for (int c = 1; c <= 5; ++c) {
            const int64_t lo = pi_B(rp, c, nodes[u].k), hi = pi_B(rp, c, nodes[u].k + nodes[u].s);
            if (hi == lo) continue;
            int64_t v = 0;
            while (v < nn && !(nodes[v].k == lo && nodes[v].s == hi - lo)) ++v;
            if (v == nn) {
                if (nn == ncap) nodes = (pnode_t *)realloc(nodes, sizeof(pnode_t) * (ncap *= 2));
                nodes[nn].k = lo;
                nodes[nn].s = hi - lo;
                ++nn;
            }
            if (ne == ecap) edge = (int64_t(*)[3])realloc(edge, sizeof(int64_t[3]) * (ecap *= 2));
            edge[ne][0] = u;
            edge[ne][1] = v;
            edge[ne][2] = c;
            ++ne;
        }
    /* a topological order (Kahn) */
    int64_t *indeg = (int64_t *)calloc((size_t)nn, sizeof(int64_t)), *order = (int64_t *)malloc(sizeof(int64_t) * nn);
    for (int64_t i = 0; i < ne; ++i) ++indeg[edge[i][1]];
    int64_t no = 0;
    order[no++] = 0;
    for (int64_t h = 0; h < no; ++h)
        for (int64_t i = 0; i < ne; ++i)
            if (edge[i][0] == order[h] && --indeg[edge[i][1]] == 0) order[no++] = edge[i][1];
    /* cells of every query node */
    dlist_t *cells = (dlist_t *)calloc((size_t)nn, sizeof(dlist_t));
    int64_t ri = dlist_get(&cells[0], (biint_t){0, 0, n});
    cells[0].c[ri].H = 0;
    int64_t nout = 0;
    for (int64_t h = 1; h < no; ++h) {
        const int64_t u = order[h];
        dlist_t *nxt = &cells[u];
        for (int64_t i = 0; i < ne; ++i) {
            if (edge[i][1] != u) continue;
            const dlist_t *pre = &cells[edge[i][0]];
            const int c = (int)edge[i][2];
            for (int64_t t = 0; t < pre->n; ++t) { /* match or mismatch */
                const dcell_t cc = pre->c[t];
                for (int x = 1; x <= 4; ++x) {
                    biint_t v = backward_ext(r, (biint_t){cc.k, cc.kp, cc.s}, x);
                    if (v.s == 0) continue;
                    int64_t j = dlist_get(nxt, v);
                    nxt->c[j].H = dmax(nxt->c[j].H, cc.H + (x == c ? a : -b));
                }
            }
            for (int64_t t = 0; t < pre->n; ++t) { /* insertion: the query symbol against a gap */
                const dcell_t cc = pre->c[t];
                const int64_t ev = dmax(cc.H - q, cc.E) - e;
                int64_t j = dlist_get(nxt, (biint_t){cc.k, cc.kp, cc.s});
                nxt->c[j].E = dmax(nxt->c[j].E, ev);
                nxt->c[j].H = dmax(nxt->c[j].H, nxt->c[j].E);
            }
        }
        for (int changed = 1; changed;) { /* deletion, to the closure */
            changed = 0;
            for (int64_t t = 0; t < nxt->n; ++t) {
                if (nxt->c[t].H <= 0) continue;
                for (int x = 1; x <= 4; ++x) {
                    const dcell_t cc = nxt->c[t];
                    biint_t v = backward_ext(r, (biint_t){cc.k, cc.kp, cc.s}, x);
                    if (v.s == 0) continue;
                    const int64_t fv = dmax(cc.H - q, cc.F) - e;
                    int64_t j = dlist_get(nxt, v);
                    if (fv > nxt->c[j].F) {
                        nxt->c[j].F = fv;
                        nxt->c[j].H = dmax(nxt->c[j].H, fv);
                        changed = 1;
                    }
                }
            }
        }
        int64_t kept = 0; /* the cells: H > 0 */
        for (int64_t t = 0; t < nxt->n; ++t)
            if (nxt->c[t].H > 0) nxt->c[kept++] = nxt->c[t];
        nxt->n = kept;
        qsort(nxt->c, (size_t)nxt->n, sizeof(dcell_t), dcell_cmp);
        if (W > 0 && nxt->n > W) nxt->n = W; /* the band */
        for (int64_t t = 0; t < nxt->n; ++t, ++nout)
            if (nout < cap) {
                int64_t *o = out + 6 * nout;
                o[0] = nodes[u].k; o[1] = nodes[u].s;
                o[2] = nxt->c[t].k; o[3] = nxt->c[t].kp; o[4] = nxt->c[t].s; o[5] = nxt->c[t].H;
            }
    }
    for (int64_t u = 0; u < nn; ++u) free(cells[u].c);
    free(cells);
    free(indeg);
    free(order);
    free(edge);
    free(nodes);
    rank_free(rp);
    rank_free(r);
    return nout;
}

int64_t orc_smem_mt(const uint8_t *B, int64_t n, const uint8_t *q, const int64_t *qoff, int64_t nq,
                    int64_t ell, int64_t smin, int64_t *out, int64_t cap, int nthreads)
{
    orc_rank_t *r = rank_new(B, n);
    int64_t *cnt = (int64_t *)calloc((size_t)(nq + 1), sizeof(int64_t));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t t = 0; t < nq; ++t) {
        const uint8_t *P = q + qoff[t];
        int64_t len = qoff[t + 1] - qoff[t], i = 0, c = 0;
        do {
            i = find_smem1(r, P, len, i, ell, smin, t, NULL, &c, 0);
        } while (i < len);
        cnt[t + 1] = c;
    }
    for (int64_t t = 0; t < nq; ++t) cnt[t + 1] += cnt[t];
    int64_t total = cnt[nq];
    if (total <= cap) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64)
#endif
        for (int64_t t = 0; t < nq; ++t) {
            const uint8_t *P = q + qoff[t];
            int64_t len = qoff[t + 1] - qoff[t], i = 0, c = 0;
            int64_t *o = out + 6 * cnt[t];
            do {
                i = find_smem1(r, P, len, i, ell, smin, t, o, &c, cnt[t + 1] - cnt[t]);
            } while (i < len);
        }
    }
    free(cnt);
    rank_free(r);
    return total;
}

/* ------------------------------------------------------------------------
 * O5: brute force on the text itself (tiny inputs only).
 * occ(P) = number of offsets t with T[t, t+|P|) = P (Section "Suffix array
 * interval and backward search"); lo(P) = number of suffixes of T that are
 * lexicographically smaller than P, under the symbol order above.
 * ---------------------------------------------------------------------- */
int64_t orc_occ_brute(const uint8_t *T, int64_t n, const uint8_t *P, int64_t len)
{
    int64_t c = 0;
    for (int64_t t = 0; t + len <= n; ++t) {
        int64_t j = 0;
        while (j < len && T[t + j] == P[j]) ++j;
        c += j == len;
    }
    return c;
}

int64_t orc_lo_brute(const uint8_t *T, int64_t n, const uint8_t *P, int64_t len)
{
    int64_t c = 0;
    for (int64_t t = 0; t < n; ++t) {
        /* compare suffix T[t..] with P; P holds letters only */
        int64_t j = 0;
        while (j < len && t + j < n && T[t + j] == P[j]) ++j;
        if (j == len) continue;                 /* P is a prefix: not smaller */
        if (t + j >= n || T[t + j] < P[j]) ++c; /* mismatch decides */
    }
    return c;
}

/* SMEMs by their definition (Section "Finding supermaximal exact matches",
 * with occurrence threshold s_min): f(i) = max{e : occ(P[i,e)) >= s_min};
 * [i, f(i)) is reported iff f(i) - i >= ell and (i = 0 or f(i) > f(i-1)).
 * The record carries (lo(X), lo(rc(X)), occ(X)) for X = P[i, f(i)), each
 * counted on T directly.  Same record layout as orc_smem. */
int64_t orc_smem_brute(const uint8_t *T, int64_t n, const uint8_t *q, const int64_t *qoff, int64_t nq,
                       int64_t ell, int64_t smin, int64_t *out, int64_t cap)
{
    int64_t nout = 0;
    for (int64_t t = 0; t < nq; ++t) {
        const uint8_t *P = q + qoff[t];
        int64_t len = qoff[t + 1] - qoff[t], fprev = -1;
        uint8_t *rc = (uint8_t *)malloc((size_t)(len > 0 ? len : 1));
        for (int64_t i = 0; i < len; ++i) {
            int64_t e = i;
            while (e < len && orc_occ_brute(T, n, P + i, e + 1 - i) >= smin) ++e;
            if (e - i >= ell && (i == 0 || e > fprev)) {
                if (nout < cap) {
                    int64_t L = e - i;
                    for (int64_t j = 0; j < L; ++j) rc[j] = orc_comp[P[i + L - 1 - j]];
                    int64_t *o = out + 6 * nout;
                    o[0] = t; o[1] = i; o[2] = e;
                    o[3] = orc_lo_brute(T, n, P + i, L);
                    o[4] = orc_lo_brute(T, n, rc, L);
                    o[5] = orc_occ_brute(T, n, P + i, L);
                }
                ++nout;
            }
            fprev = e;
        }
        free(rc);
    }
    return nout;
}
