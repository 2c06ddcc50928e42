/*
 * rb3.h -- C ABI of librb3.so: GB300 (sm_103a) multi-string double-strand BWT
 * construction by batch build + merge, and backward / SMEM search and local
 * haplotype diversity on the result.  The method is H. Li, "BWT construction and search at the terabase
 * scale" (arXiv 2409.00613); each call cites the passage that defines what it
 * computes.  All arithmetic is integer and exact.
 *
 * Conventions shared by every call
 * --------------------------------
 *  Symbols.  uint8 codes $=0 A=1 C=2 G=3 T=4 N=5, ordered
 *    $_0 < ... < $_{m-1} < A < C < G < T < N   (Section "BWT construction").
 *    Input strings and queries hold letters 1..5 only.  N is an ordinary
 *    symbol: it matches N and is its own complement (Section "Double-strand
 *    BWT": the complements of $,A,C,G,T,N are $,T,G,C,A,N).
 *  Integers.  Every count, rank and position is int64 (a BWT may exceed 2^32
 *    symbols; one index holds at most 2^40).
 *  Pointers.  Any array argument may be a device pointer or a host pointer;
 *    the library tells them apart with cudaPointerGetAttributes.  Host inputs
 *    are copied to the device inside the call; host outputs are filled before
 *    the call returns.
 *  Streams.  `stream` is a cudaStream_t (NULL = the legacy default stream).
 *    Every device operation is enqueued on it.  Calls whose result size is
 *    data dependent (build, merge, mem_search, haplotype_diversity)
 *    synchronize that stream before they return; the others return once the work is enqueued when all their
 *    outputs are device memory.
 *  Ownership.  The library owns every rb3_index and its scratch memory
 *    (stream-ordered cudaMallocAsync); callers own every output buffer.
 *  Errors.  Every int-returning call returns RB3_OK or an RB3_E_* code and
 *    sets a per-thread message readable with rb3_last_error().  There is no
 *    CPU fallback: without a usable CUDA device every compute call returns
 *    RB3_E_CUDA.
 */
#ifndef RB3_H
#define RB3_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RB3_OK 0
#define RB3_E_INVAL 1    /* bad argument: NULL, negative size, symbol out of range, wrong index kind */
#define RB3_E_NOMEM 2    /* a device or host allocation failed */
#define RB3_E_CUDA 3     /* a CUDA call failed (no device, launch error, ...) */
#define RB3_E_TIMEOUT 4  /* a bounded device-side wait gave up; the context is still usable */
#define RB3_E_CAPACITY 5 /* caller's output buffer too small; the needed size is returned */
#define RB3_E_IO 6       /* file read / write / format error */

#define RB3_SYM_SENTINEL 0
#define RB3_SYM_A 1
#define RB3_SYM_C 2
#define RB3_SYM_G 3
#define RB3_SYM_T 4
#define RB3_SYM_N 5

/* Opaque, device-resident index: a 4-bit packed BWT B with interleaved Occ
 * checkpoints, C_B(a) for every symbol, n = |B|, m = number of sentinels.
 * Layout in HBM: blocks of D symbols; block b is 32 header bytes (for each
 * symbol a, rank_B(a, b*D) as uint32 low words at bytes 0..23 and uint8 high
 * bytes at 24..29) followed by D/2 payload bytes: every 64 symbols form one
 * 32-byte sector holding their 4-bit codes bit-sliced, as four 64-bit planes
 * (plane j, bytes 8j..8j+7, has bit o set iff bit j of the code of symbol o is
 * set; plane 3 is zero since codes are 0..5).  D = 32 packs a whole block into
 * one 32-byte sector, so that a rank is a single memory request: uint32 words
 * 0..4 hold rank_B(a, b*32) for a = A..N minus rank_B(a, s*2^32) for the span
 * s = (b*32) >> 32 the block lies in (the index keeps those span bases, one row
 * per 2^32 symbols), and words 5..7 are the three 32-bit planes of its 32 codes;
 * rank_B($, l) = l minus the other five.  An index returned by rb3_build_batch also keeps
 * the batch's text and inverse suffix array, which rb3_merge uses to walk the
 * new strings in segments; rb3_drop_build_data frees them. */
typedef struct rb3_index rb3_index;

/* Tuning knobs.  Zero in any field means "default / autotuned". */
typedef struct {
    int32_t occ_interval;  /* D, symbols per Occ block: 32, 64, 128 or 256 (default 32) */
    int32_t single_strand; /* 0: index both strands (the paper's default, Section "Methods"); 1: forward only */
    int64_t seg_len;       /* merge: walk segment length L (default: autotuned) */
    int64_t seed_cap;      /* merge: ForwardExt steps after which a segment seed stops and leaves its
                              candidates (at most 63 suffixes) to the resolve pass; merge_form 3: most
                              steps of a seed, then the walk from above takes the segment (default 2*L;
                              single strand: the seed's backward-search window, default 4*L) */
    int32_t merge_form;    /* 0: segmented batched walk with bounded seeds, segment tops moved to content
                              anchors (within +-L/4 of every L-th position, so the batch's homologous
                              segments start at the same locus and walk side by side); 1: plain
                              Algorithm 1, one walk per string; 2: as 0 with tops every L symbols from
                              the string end; 3: as 0 with uncapped seeds and the takeover chain */
    int32_t search_form;   /* 0: chunked work-stealing SMEM search, one extension per lane per step;
                              1: plain, one query per thread; 2: chunked, each lane looping on its own */
    int64_t chunk_len;     /* SMEM: query chunk length (default 256) */
    int32_t walk_ctas_per_sm; /* merge: 256-thread CTAs per SM in the persistent walk's grid, 1..8
                                 (default 8, of which 4 are resident at once) */
    int32_t sa_sample;     /* build: keep a sampled suffix array for rb3_locate: every suffix starting at
                              an offset of its string that is a multiple of sa_sample (a power of two,
                              2..1024; 0 = none).  A merge keeps it when both inputs have the same rate. */
    int32_t batch_mb;      /* append: device-memory budget of one batch build, MiB (0 = none).  Each caller
                              batch is cut into runs of whole strings whose build footprint (estimated at
                              RB3_BUILD_BYTES_PER_SYMBOL per indexed symbol) fits it; a string that alone
                              exceeds it is built by itself.  Results do not depend on the cut. */
    int32_t hot_depth;     /* SMEM search (search_form 0): depth K of the hot-level table, the SA
                              bi-intervals of every A/C/G/T string of length 1..K (32 bytes each, 4^K
                              strings at depth K), built once per index on the device and kept with it.
                              A backward extension that starts from the whole index looks its first
                              symbols up there (as many as the FindSMEM loop will take, at most K, when
                              they hold no N and the looked-up interval still occurs >= min_occ times)
                              instead of extending symbol by symbol; the records are the same.
                              0: autotuned, else log4(n) - 3 clamped to 0..10; -1: no table; 1..12. */
    int32_t reserved[4];
} rb3_opts;

/* Device bytes a batch build holds at its peak per indexed symbol (both strands
 * count), as measured with rb3_device_peak on the pangenome workload, rounded up. */
#define RB3_BUILD_BYTES_PER_SYMBOL 64

/* One SMEM: query qid, query interval [start, end), and the SA bi-interval
 * (k, k', s) = (lo(X), lo(rc X), occ(X)) of X = query[start, end)
 * (Section "Double-strand BWT", SA bi-interval). 40 bytes. */
typedef struct {
    int64_t qid;
    int32_t start, end;
    int64_t k, kp, s;
} rb3_smem;

/* Fills *o with defaults (all zero). */
void rb3_opts_default(rb3_opts *o);

/* Partial BWT of one batch (Section "BWT construction": the BWT of a batch is
 * computed on its own and then merged; Section "Basic concepts" and Table 1
 * define T, S and B[i] = T[S(i)-1]).
 * seq: the n_seq strings back to back, codes 1..5 (device or host), of total
 *   length sum(len); len: n_seq lengths >= 0 (host or device).
 * The indexed text is T = P0 $ rc(P0) $ P1 $ rc(P1) $ ... (Section
 * "Double-strand BWT"), or P0 $ P1 $ ... with single_strand; sentinels are
 * ordered by position.  The batch's text must hold fewer than 2^31 symbols.
 * *out receives a new index owned by the caller (free with rb3_index_free).
 * RB3_E_INVAL on a symbol outside 1..5 or a negative length. */
int rb3_build_batch(const uint8_t *seq, const int64_t *len, int64_t n_seq, const rb3_opts *o,
                    void *stream, rb3_index **out);

/* An index of zero strings (n = m = 0); merging a batch into it yields the batch. */
int rb3_index_empty(const rb3_opts *o, rb3_index **out);

/* Algorithm 1 (AppendBWT): dst := BWT(strings of dst, then strings of src).
 * The sentinels of src rank after those of dst (the walk starts at l = m1).
 * src is unchanged.  With src's build data the new strings are walked in
 * segments seeded by ForwardExt (Algorithm 3): a seed that has not resolved
 * after seed_cap steps leaves the few suffixes it still ties with as
 * candidates, the segment walks them all at once, and a pass down each string
 * picks the true one, so the walk's depth does not grow with the length of a
 * match with the index; without the build data, or with merge_form = 1, one
 * walk per string as in the paper.  The result is the same bit for bit.
 * rb3_merge uses default options.  RB3_E_CUDA (dst unchanged) if the walk's
 * own consistency check fails. */
int rb3_merge(rb3_index *dst, const rb3_index *src, void *stream);
int rb3_merge_opts(rb3_index *dst, const rb3_index *src, const rb3_opts *o, void *stream);

/* The merge in parts, for merging on several GPUs (each holding a copy of dst
 * and src).  Algorithm 1's walks are independent given B1 (Section "BWT
 * construction": the merge is parallel over the strings of B2), so the input
 * strings of src can be split among parts; every part computes the merged
 * rows of its strings' suffixes, the parts' arrays are added up (all-reduce),
 * and every part applies the whole array to its own copy of dst.
 *
 * rb3_merge_partition (host only; no GPU): owner[i] in [0, parts) for each of
 * the n_seq input strings (lengths len), longest first to the part with the
 * fewest symbols so far; deterministic, so every part computes the same.
 * rb3_merge_positions: pos[k] (device, src->n entries, caller-owned) = the row
 * of the merged index that B2 row k goes to (k + l of Algorithm 1), written for
 * the rows of the input strings with owner[i] == part (both strands) and 0 for
 * every other row, so that the parts' arrays sum to the whole; owner = NULL
 * writes every row.  With an empty dst the part owning string 0 writes every
 * row.  Options as rb3_merge_opts.  dst and src are not modified.
 * rb3_merge_apply: dst := the merge of src into dst at the rows pos (host or
 * device, src->n entries); pos must increase and lie in [0, n(dst) + n(src)),
 * else RB3_E_INVAL and dst is unchanged.  rb3_merge equals
 * rb3_merge_positions (owner NULL) then rb3_merge_apply.  dst may be
 * run-length encoded (the walk ranks its spans; rb3_merge_apply rewrites them);
 * src must be plain (RB3_E_INVAL otherwise). */
int rb3_merge_partition(const int64_t *len, int64_t n_seq, int32_t parts, int32_t *owner);
int rb3_merge_positions(const rb3_index *dst, const rb3_index *src, const rb3_opts *o, const int32_t *owner,
                        int32_t part, int64_t *pos, void *stream);
int rb3_merge_apply(rb3_index *dst, const rb3_index *src, const int64_t *pos, void *stream);

/* The build loop of Section "Methods": for each batch of strings, build its
 * BWT (as rb3_build_batch) and merge it into dst (as rb3_merge), in order.
 * The build of batch b+1 runs on the device while batch b is merged, as the
 * paper runs partial BWT construction and BWT merge together (Table 2, note
 * 7); this uses two internal streams (ordered after the work already on
 * `stream`) and one host thread, and keeps at most two built batches beyond
 * the one being merged.  seq / len: all strings back to back (host or device);
 * batch_end[b] = number of strings in batches 0..b (non-decreasing, the last
 * equal to n_seq).  The result is the same as building and merging the
 * batches one by one.  Synchronizes `stream`. */
int rb3_append_batches(rb3_index *dst, const uint8_t *seq, const int64_t *len, int64_t n_seq,
                       const int64_t *batch_end, int64_t n_batches, const rb3_opts *o, void *stream);

/* Backward search (Section "Suffix array interval and backward search"):
 * for query i = q[qoff[i] .. qoff[i+1]) writes lo_hi[2i] = lo(P) (the number of
 * suffixes smaller than P) and lo_hi[2i+1] = hi(P) = lo(P) + occ(P).
 * qoff: nq+1 non-decreasing offsets; lo_hi: 2*nq int64, caller-owned. */
int rb3_backward_search(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, int64_t nq,
                        int64_t *lo_hi, void *stream);

/* BWA-SW between two prefix DAWGs (Section "Finding inexact matches with
 * BWA-SW", Algorithm 5): for every query P = q[qoff[i] .. qoff[i+1]), its
 * prefix DAWG -- a node is the SA interval (uk, us) of a substring of P in the
 * BWT of the one-string, one-strand text P$ (strings with one interval are one
 * node), an edge x -> cx for every symbol c of A..N that keeps the interval
 * non-empty -- against the indexed text's (a node is a bi-interval (k, k', s);
 * its children its BackwardExt by A, C, G, T), the query's nodes in a
 * topological order.  The cells of a query node gather, over its in-edges
 * (u, c), the four children of each kept cell of u (match +a when the text
 * symbol is c, else -b; N matches nothing) and the cell itself (insertion,
 * E = max(H - gap_open, E) - gap_ext), then deletions to the closure (F of a
 * child = max(H - gap_open, F) - gap_ext); the W cells of largest H are kept
 * (ties: smaller k, k', s).  The root's cell is the whole text with H = 0.
 * out: 7 int64 per record (qid, uk, us, k, k', s, H), every kept cell with
 * H > 0 of every query node but the root, sorted by (qid, uk, us, then H
 * descending, k, k', s); host or device memory, caller-owned.  If more than
 * cap records exist, *n_out holds the number and RB3_E_CAPACITY is returned.
 * Queries of at most 2047 bases; W in 1..32; scores as
 * rb3_haplotype_diversity; a double-strand index of any layout.
 * RB3_E_CAPACITY also when a query node left more than 65,534 candidate cells
 * (the deletion closure of a long exact match holds about a dozen cells per
 * unit of score on a pangenome). */
int rb3_bwasw(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, int64_t nq, int32_t a, int32_t b,
              int32_t gap_open, int32_t gap_ext, int32_t W, int64_t *out, int64_t cap, int64_t *n_out, void *stream);

/* Local haplotype diversity (Section "Estimating local haplotype diversity"):
 * Algorithm 5 (the revised BWA-SW of Section "Finding inexact matches with
 * BWA-SW") on the graph of each linear query q[qoff[i] .. qoff[i+1]), walked
 * from its end to its start, against the prefix DAWG of the indexed text; a
 * node is the bi-interval (k, k', s) of a string, its children its
 * BackwardExt by A, C, G, T.  Scores: match +a, mismatch -b (N in a query
 * mismatches every symbol), a gap of length L costs gap_open + L * gap_ext.
 * After each query symbol the W cells of largest H (ties: smaller k, k', s)
 * are kept; deletions are applied until no cell's score rises.  The result of
 * query i is the set of nodes aligned end to end with H > 0, best first; with
 * redundancy = 1 a node is dropped when its [k, k+s) or [k', k'+s) lies
 * inside that of a node kept before it.
 * out: nq * W records of 4 int64 (k, k', s, H), query i's from out + 4*W*i;
 * n_out[i]: the number of query i's records.  Both caller-owned, host or
 * device memory; q and qoff too.  Needs a double-strand index (any layout).
 * RB3_E_INVAL: a symbol outside 1..5, W outside 1..32, a < 1, b < 0,
 * gap_open < 0, gap_ext < 1, a score above 65536, a query longer than
 * 2^29 / a, or a single-strand index.  RB3_E_CAPACITY when a query symbol
 * left more than 65,534 candidate cells: that query's n_out is -1, every
 * other query's result is written. */
int rb3_haplotype_diversity(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, int64_t nq, int32_t a,
                            int32_t b, int32_t gap_open, int32_t gap_ext, int32_t W, int32_t redundancy,
                            int64_t *out, int64_t *n_out, void *stream);

/* Counters of rb3_haplotype_diversity since the last reset, summed over
 * queries: out[0] = rank-all reads (two per extended cell: the ranks of every
 * symbol at k and at k + s), out[1] = cells entered into the per-step tables.
 * Synchronises the device; reset != 0 zeroes them after reading. */
int rb3_diversity_stats(int64_t *out, int32_t reset);

/* Locate (Section "Locating with FM-index", Algorithm 2): for each row i of
 * the BWT (0 <= rows[j] < n), out[2j] = the index of the string its suffix
 * starts in (strings numbered as concatenated: P0, rc(P0), P1, ... for a
 * double-strand index, in the order they were built and merged) and
 * out[2j+1] = the offset of the suffix on that string.  Needs an index built
 * with opts.sa_sample = s (merges keep the sample when both inputs have the
 * same rate); the sample holds every suffix starting at an offset that is a
 * multiple of s, so a row takes at most s - 1 LF steps.  rows and out may be
 * host or device memory.  RB3_E_INVAL on a row outside [0, n) or an index
 * without a sample. */
int rb3_locate(const rb3_index *idx, const int64_t *rows, int64_t n_rows, int64_t *out, void *stream);

/* SMEMs of length >= min_len occurring >= min_occ times (Section "Finding
 * supermaximal exact matches", Algorithm 4 with Algorithm 3), for every query.
 * Needs a double-strand index.  Records are sorted by (qid, start).  If more
 * than cap records exist, nothing is written, *n_out holds the number needed
 * and RB3_E_CAPACITY is returned; call again with a larger buffer. */
int rb3_mem_search(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, int64_t nq, int32_t min_len,
                   int64_t min_occ, rb3_smem *out, int64_t cap, int64_t *n_out, void *stream);
int rb3_mem_search_opts(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, int64_t nq,
                        int32_t min_len, int64_t min_occ, const rb3_opts *o, rb3_smem *out, int64_t cap,
                        int64_t *n_out, void *stream);

/* No counterpart in the paper: an allocation-free form of rb3_mem_search for
 * callers that cannot allocate device memory while they search -- their device
 * memory belongs to their own allocator or a fixed memory plan, or their
 * request loop must not call cudaMalloc / cudaFree, which can block and
 * synchronize the device.  Same records in the same order as rb3_mem_search.
 * q, qoff and out must be device pointers (out may be NULL when cap = 0).
 * Limits: at most 131,072 queries per call, and at most 524,288 query chunks
 * (a query of L bases counts max(1, ceil(L/256)) chunks); larger calls return
 * RB3_E_INVAL without doing any work.  qoff must not decrease and no query may
 * reach 2^31 bases: such a qoff is refused with RB3_E_INVAL before any search
 * kernel runs.  The scratch is a file-scope device
 * array of 4,726,868 bytes that every GPU which loads the library holds until
 * the process exits; the library allocates nothing else for this call.  The
 * first call on a device looks up that array's device address
 * (cudaGetSymbolAddress), so make it before any stream capture.  All calls
 * share the array, and it keeps the last call's contents (the call clears what
 * must start at zero): calls that overlap on the GPU race, so do not run two
 * at once.  Synchronizes the stream; RB3_E_CAPACITY as for rb3_mem_search. */
int rb3_mem_search_noalloc(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, int64_t nq, int32_t min_len,
                           int64_t min_occ, rb3_smem *out, int64_t cap, int64_t *n_out, void *stream);

/* ---- Served SMEM search (continuous batching) ----------------------------
 * A server keeps an index resident and answers SMEM requests (one query each)
 * as they arrive.  `slots` worker threads, each with its own stream and fixed
 * buffers, take every waiting request that fits a budget of query bases (a
 * longer request alone) as soon as they are free, and run them as one chunked
 * micro-batch (as rb3_mem_search); requests arriving while others run are
 * admitted by the next free slot, so micro-batches overlap on the device.
 * Each request gets exactly the SMEMs rb3_mem_search gives for its query
 * alone (qid field 0).  The index must outlive the server and must not be
 * merged into while it serves. */
typedef struct rb3_server rb3_server;

typedef struct {
    int32_t min_len;            /* SMEM length threshold (default 31) */
    int32_t slots;              /* micro-batches in flight (default 4) */
    int64_t min_occ;            /* occurrence threshold (default 1) */
    int64_t max_batch_bases;    /* query bases per micro-batch (default 32 Mi) */
    int64_t max_batch_requests; /* requests per micro-batch (default 4096; 1 = no batching) */
    int64_t search_form;        /* rb3_opts.search_form of the micro-batches' search (default 0) */
    int64_t hot_depth;          /* rb3_opts.hot_depth of the micro-batches' search (default 0); the
                                   table is built when the server is created */
    int64_t reserved[2];
} rb3_server_opts;

typedef struct {
    int64_t req_id, tag, n_smem;
    int32_t status;         /* RB3_OK or the error of its micro-batch */
    int32_t batch_requests; /* size of the micro-batch it ran in */
    int64_t t_submit_ns;    /* CLOCK_MONOTONIC at rb3_server_submit */
    int64_t t_done_ns;      /* CLOCK_MONOTONIC when its results reached the host */
} rb3_completion;

void rb3_server_opts_default(rb3_server_opts *o);
int rb3_server_create(const rb3_index *idx, const rb3_server_opts *o, rb3_server **out);
/* Queues one query (host memory, copied; codes 1..5); returns at once. */
int rb3_server_submit(rb3_server *s, const uint8_t *q, int64_t len, int64_t tag, int64_t *req_id);
/* Up to cap completions, oldest first; waits up to wait_us for the first. */
int rb3_server_poll(rb3_server *s, rb3_completion *out, int64_t cap, int64_t *n, int32_t wait_us);
/* Copies a completed request's SMEMs (start-ordered) and releases them. */
int rb3_server_take(rb3_server *s, int64_t req_id, rb3_smem *out, int64_t cap, int64_t *n);
int64_t rb3_server_batches(rb3_server *s);
/* Where the slots' time went since the server was created (tracing; summed over
 * slots): out[0] micro-batches, out[1] requests, out[2] query bases, out[3] ns
 * gathering the requests' queries into a slot's pinned buffer, out[4] ns from
 * there to the records on the host (query and offset copies, the search, the
 * records' copy back, the stream synchronized), out[5] ns splitting the
 * records by request and publishing the completions. */
int rb3_server_stats(rb3_server *s, int64_t out[6]);
/* Open-loop load generator on native threads (four submitting, as several
 * clients would, and the caller's collecting): submits query i (q[qoff[i] ..
 * qoff[i+1]), host memory) at t0 + arrival_ns[i] (non-decreasing, relative to
 * a start t0 a few ms after the call), collects every completion and drops its
 * records; done_ns[i] = its completion time - t0 (latency = done_ns[i] -
 * arrival_ns[i]) and, if batch is not NULL, batch[i] = the size of the
 * micro-batch it ran in.  Returns when all n have completed, or at the first
 * error.  Do not submit or poll from other threads meanwhile. */
int rb3_server_replay(rb3_server *s, const uint8_t *q, const int64_t *qoff, int64_t n, const int64_t *arrival_ns,
                      int64_t *done_ns, int32_t *batch);
void rb3_server_destroy(rb3_server *s);

/* ---- Autotuner (no counterpart in the paper; tunes this build's knobs) ----
 * rb3_tune_merge times the merge's walk phase (into scratch: dst and src are
 * not modified) for several segment lengths around the default, each with seed
 * caps of 1, 2 and 4 segment lengths (unless base->seed_cap is set), and
 * writes the fastest into best->seg_len and best->seed_cap; rb3_tune_search times the chunked SMEM search
 * (q, qoff: device) for several chunk lengths and writes best->chunk_len, then (unless
 * base->hot_depth is set) for hot-level depths -1, 6, 8 and 10 and writes best->hot_depth.  The
 * choice is remembered per input shape (device, D, strand mode, log2 size
 * classes) and used by rb3_merge / rb3_mem_search when their knob is 0; with
 * RB3_TUNE_FILE set it is also persisted there.  best_ms (optional) receives
 * the winner's time.  Both synchronize the stream. */
int rb3_tune_merge(const rb3_index *dst, const rb3_index *src, const rb3_opts *base, rb3_opts *best, double *best_ms,
                   void *stream);
int rb3_tune_search(const rb3_index *idx, const uint8_t *q, const int64_t *qoff, int64_t nq, int32_t min_len,
                    int64_t min_occ, const rb3_opts *base, rb3_opts *best, double *best_ms, void *stream);

/* Layout autotuner for a whole incremental build (the input of
 * rb3_append_batches: seq host or device, len, batch_end): builds batch 1 and
 * merges it into batch 0 at the Occ intervals D = 32, 64 and 128, each with
 * rb3_tune_merge's segment length and seed cap, and writes into *best the
 * fastest D whose projected index (every batch's symbols at D's bytes per
 * symbol: 1, 1 and 0.75) fits index_mb MiB (0 = no limit; if none fits, the
 * smallest), with its seg_len and seed_cap.  cand_ms[3] / cand_mb[3]
 * (optional) receive each D's build + merge time and projected index MiB.
 * Needs two batches; allocates and frees its own indexes; synchronizes the
 * stream. */
int rb3_tune_build(const uint8_t *seq, const int64_t *len, int64_t n_seq, const int64_t *batch_end, int64_t n_batches,
                   const rb3_opts *base, int64_t index_mb, rb3_opts *best, double *cand_ms, double *cand_mb,
                   void *stream);

/* Unpacks B into codes (n bytes, one symbol per byte) and, when occ != NULL,
 * writes occ[j*6 + a] = rank_B(a, j*D) for j = 0 .. n/D (Table 1). */
int rb3_export(const rb3_index *idx, uint8_t *codes, int64_t *occ, void *stream);

/* n, m, C[0..6] (C[a] = C_B(a), C[6] = n), D (the span S of a run-length
 * index) and flags (bit0: single strand, bit1: holds build data, bit2:
 * run-length layout, bits 8..: the sampled suffix array's rate, 0 if none).
 * Any output pointer may be NULL. */
int rb3_index_info(const rb3_index *idx, int64_t *n, int64_t *m, int64_t *C, int32_t *occ_interval,
                   int32_t *flags);

/* Run-length copy of a finished index for queries (Section "BWT construction",
 * Fig. 2b: the static, run-length encoded BWT with marginal counts per block).
 * The BWT is cut into spans of `span` symbols (a power of two, 512..16384;
 * 0 = 2048).  Device layout: one 64-byte header per span (uint32 rank of A..N
 * at the span start, relative to its 2^32-symbol range, as for D = 32; the
 * uint64 byte offset of the span's runs; their number; two decode marks: the
 * span offset, in-span ranks of A..N and byte offset of the runs holding
 * offsets len/3 and 2 len/3), then the runs, cut at span boundaries, one byte
 * each (symbol << 5 | f: f < 30 gives length f + 1, f = 30 length 31 + the
 * next byte, f = 31 length 287 + the next two bytes, little-endian).  A rank
 * reads the span's header and decodes its runs from the last mark before the
 * position.  The copy keeps src's sampled suffix array; src is unchanged.
 * rb3_backward_search, rb3_mem_search (all forms), rb3_mem_search_noalloc,
 * the server, rb3_locate, rb3_export (occ rows = the span headers),
 * rb3_index_save / rb3_index_load take it.  It can be merged into directly:
 * rb3_merge / rb3_merge_opts / rb3_append_batches / rb3_merge_positions /
 * rb3_tune_merge take it as dst, the walk ranking its spans, and the merge
 * rewrites every span from its old runs and the batch's symbols at their merged
 * rows (no plain copy of dst; the result is run-length at the same span, dst
 * unchanged on failure).  As src of rb3_merge a run-length index is expanded to
 * a transient plain D = 32 copy (one byte per symbol); rb3_merge_positions and
 * rb3_tune_merge refuse it as src (RB3_E_INVAL).
 * RB3_E_INVAL for a bad span or a src that is already run-length encoded. */
int rb3_index_compress(const rb3_index *src, int32_t span, void *stream, rb3_index **out);

/* Device bytes the index holds (blocks or span headers, runs, span bases,
 * sampled suffix array; build data not counted) and its number of runs (-1
 * for a plain index).  Either pointer may be NULL. */
int rb3_index_bytes(const rb3_index *idx, int64_t *device_bytes, int64_t *runs);

/* Counts of the segmented merge walks (Algorithm 1 with ForwardExt seeds)
 * since the last reset, added up by the walks as they finish: out[0] seeds
 * run, out[1] Occ block reads of the seeds (one per ForwardExt whose two ends
 * share a block, else two), out[2] block reads of the walk steps (one per new
 * symbol, plus one per position walked a second time), out[3] positions walked
 * a second time from their segment's resolved top (merge_form 0 and 2), or
 * segments taken over from above (merge_form 3).  At D = 32 a block read is
 * one 32-byte memory request.  reset != 0 zeroes them after the read.
 * Synchronizes the device. */
int rb3_walk_stats(int64_t *out, int32_t reset);

/* Counts of the step-machine SMEM search (rb3_mem_search's default form,
 * Algorithm 4 over the extensions of Algorithm 3) since the last reset, added
 * up by its warps as they finish: out[0] extensions (BackwardExt or
 * ForwardExt), out[1] Occ block reads (one per extension whose two interval
 * ends share a block, else two; at D = 32 a block read is one 32-byte memory
 * request).  reset != 0 zeroes them after the read.  Synchronizes the device. */
int rb3_search_stats(int64_t *out, int32_t reset);

/* Self-test of the bounded device-side waits (the radix sort's look-back wait,
 * the same device function): one thread waits on a flag that nothing sets,
 * for `limit` polls (1..2^20, about 0.1 us each), then records the time-out
 * and returns.  Returns RB3_E_TIMEOUT, the status a real wait that gave up
 * reports; the context stays usable.  Synchronizes the stream. */
int rb3_selftest_wait(int32_t limit, void *stream);

/* The high-water mark of device memory in use by this library's stream-ordered
 * allocations (the device's default memory pool) since the last reset, in
 * bytes; reset != 0 sets the mark back to the memory in use now and returns
 * that (so a later call minus it is what a call in between added at its
 * peak).  Host-side query. */
int rb3_device_peak(int64_t *used_high, int32_t reset);

/* Frees the batch text and inverse suffix array kept by rb3_build_batch. */
int rb3_drop_build_data(rb3_index *idx);

/* Static on-disk image (header + the packed blocks, which already hold the
 * Occ checkpoints, + the span bases of a D = 32 or run-length index past 2^32,
 * + a run-length index's runs, + the sampled suffix array when there is one),
 * in the spirit of the paper's static, memory-mappable BWT (Section "BWT
 * construction").  Appending after a load continues the build.  A run-length
 * image is checked on load (offsets, run lengths and counts span by span);
 * an inconsistent one gives RB3_E_IO. */
int rb3_index_save(const rb3_index *idx, const char *path);
int rb3_index_load(const char *path, void *stream, rb3_index **out);

void rb3_index_free(rb3_index *idx);

/* Message of the last failed call on this thread ("" if none). */
const char *rb3_last_error(void);

/* Host helper: ACGT/acgt -> 1..4, every other byte -> N (5). */
int rb3_encode_ascii(const char *ascii, int64_t n, uint8_t *codes);

/* Per-phase device timing.  When enabled, every phase of build / merge /
 * search, and each hot kernel on its own, is bracketed by CUDA events on the
 * caller's stream; durations, call counts and the algorithmic bytes the
 * kernels moved are accumulated per name.  Launches of the library's kernels
 * are counted always.  Fills names[i] (valid until the next read), ms[i],
 * calls[i], bytes[i] for i < min(*n, cap); any output array may be NULL. */
int rb3_profile_enable(int on);
int rb3_profile_reset(void);
int rb3_profile_read(const char **names, double *ms, int64_t *calls, double *bytes, int32_t cap, int32_t *n);
/* Every phase recorded since rb3_profile_reset, in the order they were drained
 * (per stream, the order they ran), with its start relative to the reset (an
 * event recorded on the legacy stream then) and its duration, in ms: shows
 * which phases of different streams ran at the same time.  names[i] are static
 * strings.  *n receives the number of phases (up to cap are written). */
int rb3_profile_timeline(const char **names, double *start_ms, double *dur_ms, int64_t cap, int64_t *n);
int64_t rb3_launch_count(void);

/* Random-access roofline probe (measurement only; touches no index).  Times
 * random reads of bytes_per_access (32, 64 or 128) bytes at 32-byte-aligned
 * random addresses of a device buffer of buffer_bytes (>= 64 MiB; use one much
 * larger than L2), with threads_per_sm threads on every SM.  dependent = 0:
 * each thread keeps 4 independent reads in flight; dependent = 1: each thread
 * follows a chain whose next address depends on the data read (the pattern of
 * an LF walk); 2 and 3: the same with bytes_per_access/32 lanes reading the
 * sectors of one access in a single instruction (one request per access);
 * 4 and 5: 0 and 1 with a 64-byte L2 fetch-size hint on every read.
 * Writes the delivered GB/s and millions of reads per second. */
int rb3_probe_random_gather(int32_t bytes_per_access, int32_t dependent, int32_t threads_per_sm, int64_t buffer_bytes,
                            double *gbs, double *maccess_per_s, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RB3_H */
