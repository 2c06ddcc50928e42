"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element
by element (bit-exact: every output is integer)."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2409_00613_gb300 as rb

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
FIELDS = ("qid", "start", "end", "k", "kp", "s")


def build(S, s0=0, s1=None, host=False, **opts):
    s1 = len(S.lens) if s1 is None else s1
    off = S.offsets
    seq = S.seq[off[s0]:off[s1]].copy()
    lens = S.lens[s0:s1].copy()
    if not host:
        seq = torch.from_numpy(seq).to(DEV)
    return rb.rb3_build_batch(seq, lens, opts=opts or None)


def ref_bwt(S, s0=0, s1=None, both=True):
    s1 = len(S.lens) if s1 is None else s1
    sub = S.subset(s0, s1)
    return oracle.bwt(oracle.concat(sub.seq, sub.lens, both))


def smem_rows(recs, n):
    if n == 0:
        return np.zeros((0, 6), dtype=np.int64)
    return np.stack([recs[f].astype(np.int64) for f in FIELDS], axis=1)


def check_index(idx, B, D=None):
    info = rb.rb3_index_info(idx)
    if D is not None:
        assert info["occ_interval"] == D
    codes, occ = rb.rb3_export(idx, want_occ=True)
    assert np.array_equal(codes, B)
    assert np.array_equal(occ, oracle.occ_table(B, info["occ_interval"]))
    assert info["n"] == len(B)
    assert info["C"] == list(oracle.counts(B))


def test_config0_tiny_build_merge_search():
    S, Q = synth.tiny()
    B_all = ref_bwt(S)
    A = build(S, 0, 32)
    B = build(S, 32, 64)
    check_index(A, ref_bwt(S, 0, 32))
    check_index(B, ref_bwt(S, 32, 64))
    rb.rb3_merge(A, B)
    check_index(A, B_all)
    assert rb.rb3_index_info(A)["m"] == 128
    direct = build(S, 0, 64)
    check_index(direct, B_all)
    # plain Algorithm 1 form gives the same bits
    A2 = build(S, 0, 32)
    rb.rb3_merge_opts(A2, B, {"merge_form": 1})
    check_index(A2, B_all)
    # backward search: 1,000 queries of 20 bp, device and host buffers
    want = oracle.backward_search(B_all, Q.q, Q.qoff)
    got = rb.rb3_backward_search(A, torch.from_numpy(Q.q).to(DEV), torch.from_numpy(Q.qoff).to(DEV))
    assert np.array_equal(got, want)
    assert np.array_equal(rb.rb3_backward_search(A, Q.q, Q.qoff), want)
    assert np.all(want[:, 1] > want[:, 0])  # every query was sampled from the text


@pytest.mark.parametrize("D", [32, 64, 128, 256])
@pytest.mark.parametrize("both", [True, False])
def test_random_lists_batches(D, both):
    g = synth.rng(1000 + D + both)
    for trial in range(5):
        n_str = int(g.integers(3, 40))
        S = synth.random_strings(g, n_str, int(g.integers(5, 700)), n_frac=0.03, allow_empty=True)
        cuts = sorted(set([0, n_str] + list(g.integers(0, n_str, size=2))))
        opts = {"occ_interval": D, "single_strand": int(not both)}
        idx = None
        for a, b in zip(cuts[:-1], cuts[1:]):
            part = build(S, a, b, host=bool(trial & 1), **opts)
            check_index(part, ref_bwt(S, a, b, both), D)
            if idx is None:
                idx = part
            else:
                mopts = dict(opts, seg_len=int(g.integers(3, 64)), seed_cap=int(g.integers(1, 20)),
                             merge_form=(0, 2, 3)[trial % 3])
                rb.rb3_merge_opts(idx, part, mopts)
        check_index(idx, ref_bwt(S, 0, n_str, both), D)


def test_merge_into_empty_and_empty_batches():
    g = synth.rng(77)
    S = synth.random_strings(g, 9, 300, n_frac=0.02)
    idx = rb.rb3_index_empty()
    assert rb.rb3_index_info(idx)["n"] == 0
    for a, b in [(0, 0), (0, 4), (4, 4), (4, 9)]:
        part = build(S, a, b)
        rb.rb3_merge(idx, part)
    check_index(idx, ref_bwt(S))
    # merging an empty batch leaves the index unchanged
    rb.rb3_merge(idx, build(S, 0, 0))
    check_index(idx, ref_bwt(S))


def test_all_empty_strings_and_single_symbols():
    S = synth.Strings(np.array([1, 5], dtype=np.uint8), np.array([0, 1, 0, 0, 1, 0], dtype=np.int64))
    check_index(build(S), ref_bwt(S))


def test_large_groups_low_complexity():
    """Long single-symbol runs make suffix groups far larger than the shared-memory
    path handles (the radix path of the builder)."""
    g = synth.rng(5)
    parts = [np.full(3000, 5, np.uint8), synth.random_bases(g, 500), np.full(2500, 1, np.uint8),
             np.tile(np.array([1, 2], np.uint8), 1500), synth.random_bases(g, 100)]
    seq = np.concatenate(parts)
    S = synth.Strings(seq, np.array([3000, 500, 2500, 3000, 100], dtype=np.int64))
    check_index(build(S), ref_bwt(S))
    A = build(S, 0, 2)
    rb.rb3_merge_opts(A, build(S, 2, 5), {"seg_len": 100})
    check_index(A, ref_bwt(S))


@pytest.mark.parametrize("both", [True, False])
def test_n_free_batches_sentinel_windows(both):
    """Batches without N take the 2-bit round-0 key: strings that end a few
    symbols after a shared prefix (U$ against U A..A, the ties the count field
    breaks), all-A strings of every length up to past the key width, empty
    strings, long A and C runs (groups larger than shared memory), and random
    N-free lists; against the oracle, built whole and by merges."""
    g = synth.rng(4242 + both)
    seqs = [np.zeros(0, np.uint8)]
    for k in range(0, 24):
        seqs.append(np.full(k, 1, np.uint8))                                  # A^k
        seqs.append(np.concatenate([[2], np.full(k, 1, np.uint8)]).astype(np.uint8))  # C A^k
        seqs.append(np.concatenate([[3, 2], np.full(k, 1, np.uint8), [4]]).astype(np.uint8))  # G C A^k T
    seqs += [np.full(2500, 1, np.uint8), np.full(1800, 2, np.uint8), synth.random_bases(g, 400)]
    for _ in range(30):
        seqs.append(synth.random_bases(g, int(g.integers(0, 60))))
    order = g.permutation(len(seqs))
    seqs = [seqs[i] for i in order]
    S = synth.Strings(np.concatenate(seqs).astype(np.uint8), np.array([len(x) for x in seqs], np.int64))
    assert not np.any(S.seq == 5)
    opts = {"single_strand": int(not both)}
    check_index(build(S, **opts), ref_bwt(S, both=both))
    half = len(seqs) // 2
    A = build(S, 0, half, **opts)
    rb.rb3_merge_opts(A, build(S, half, len(seqs), **opts), dict(opts, seg_len=50))
    check_index(A, ref_bwt(S, both=both))
    for trial in range(4):
        R = synth.random_strings(g, int(g.integers(3, 40)), int(g.integers(5, 300)), n_frac=0.0, allow_empty=True)
        check_index(build(R, **opts), ref_bwt(R, both=both))


def test_mixed_occ_intervals():
    """Merges between indexes of different Occ intervals (the result takes the
    destination's), segmented and plain walks."""
    g = synth.rng(606)
    S = synth.random_strings(g, 24, 900, n_frac=0.03)
    for D1, D2 in [(32, 64), (64, 32), (32, 256), (128, 32)]:
        for form in (0, 1, 2):
            idx = build(S, 0, 10, occ_interval=D1)
            rb.rb3_merge_opts(idx, build(S, 10, 24, occ_interval=D2), {"merge_form": form, "seg_len": 50})
            assert rb.rb3_index_info(idx)["occ_interval"] == D1
            check_index(idx, ref_bwt(S), D1)


@pytest.mark.parametrize("D", [32, 64])
def test_backward_search_edges(D):
    g = synth.rng(9)
    S = synth.random_strings(g, 12, 200, n_frac=0.05)
    B = ref_bwt(S)
    idx = build(S, occ_interval=D)
    pats = [np.zeros(0, np.uint8), np.array([5], np.uint8), np.array([5, 5, 5], np.uint8)]
    for _ in range(200):
        L = int(g.integers(1, 15))
        s = int(g.integers(0, len(S.seq) - L))
        pats.append(S.seq[s:s + L].copy() if g.random() < 0.7 else synth.random_bases(g, L))
    q = np.concatenate(pats)
    qoff = np.concatenate([[0], np.cumsum([len(p) for p in pats])]).astype(np.int64)
    assert np.array_equal(rb.rb3_backward_search(idx, q, qoff), oracle.backward_search(B, q, qoff))


@pytest.mark.parametrize("D", [32, 64])
@pytest.mark.parametrize("chunk", [0, 5, 17, 64])
@pytest.mark.parametrize("ell,smin", [(1, 1), (4, 1), (12, 2), (19, 1)])
def test_smem_vs_oracle(chunk, ell, smin, D):
    S = synth.pangenome(seed=31, founder_len=3000, n_hap=6, batch=3)
    B = ref_bwt(S)
    idx = build(S, 0, 3, occ_interval=D)
    rb.rb3_merge(idx, build(S, 3, 6, occ_interval=D))
    Q = synth.mem_queries(S, seed=32, nq=300, median=80, lo=1, hi=600, sub=0.02)
    want = oracle.smem(B, Q.q, Q.qoff, ell, smin)
    for form in (0, 1, 2):
        recs, n = rb.rb3_mem_search_opts(idx, torch.from_numpy(Q.q).to(DEV), torch.from_numpy(Q.qoff).to(DEV),
                                         ell, smin, {"chunk_len": chunk, "search_form": form})
        assert np.array_equal(smem_rows(recs, n), want), (form, chunk, ell, smin)


@pytest.mark.parametrize("layout", [32, 128, "rle512"])
def test_smem_hot_levels_vs_oracle(layout):
    """The hot-level table (depth -1 = none, 2, 3, 7, 12): a backward loop that
    starts from the whole index takes its first symbols from the table; the
    records equal the oracle's, the algorithmic extension count is the same at
    every depth and the rank-block reads fall."""
    S = synth.pangenome(seed=36, founder_len=4000, n_hap=6, batch=3)
    B = ref_bwt(S)
    D = 32 if layout == "rle512" else layout
    idx = build(S, 0, 3, occ_interval=D)
    rb.rb3_merge(idx, build(S, 3, 6, occ_interval=D))
    if layout == "rle512":
        idx = rb.rb3_index_compress(idx, 512)
    Q = synth.mem_queries(S, seed=37, nq=400, median=90, lo=1, hi=700, sub=0.02)
    g = synth.rng(38)
    q = Q.q.copy()
    nmask = g.random(len(q)) < 0.01  # N inside the looked-up windows
    q[nmask] = 5
    dq, doff = torch.from_numpy(q).to(DEV), torch.from_numpy(Q.qoff).to(DEV)
    for ell, smin in ((1, 1), (4, 1), (12, 2), (31, 1)):
        want = oracle.smem(B, q, Q.qoff, ell, smin)
        stats = {}
        for K in (-1, 2, 3, 7, 12):
            rb.rb3_search_stats(reset=True)
            recs, n = rb.rb3_mem_search_opts(idx, dq, doff, ell, smin, {"hot_depth": K, "chunk_len": 64})
            stats[K] = rb.rb3_search_stats()
            assert np.array_equal(smem_rows(recs, n), want), (layout, ell, smin, K)
        assert len({v["extensions"] for v in stats.values()}) == 1, stats
        if ell >= 12:
            assert stats[7]["block_reads"] < stats[-1]["block_reads"], stats
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_mem_search_opts(idx, dq, doff, 31, 1, {"hot_depth": 13})
    assert e.value.code == rb.RB3_E_INVAL


def test_hot_table_follows_merges():
    """A table built for an index is rebuilt after a merge changes it."""
    S = synth.pangenome(seed=39, founder_len=3000, n_hap=6, batch=3)
    idx = build(S, 0, 3)
    Q = synth.mem_queries(S, seed=40, nq=200, median=90, lo=31, hi=400, sub=0.01)
    dq, doff = torch.from_numpy(Q.q).to(DEV), torch.from_numpy(Q.qoff).to(DEV)
    recs, n = rb.rb3_mem_search_opts(idx, dq, doff, 31, 1, {"hot_depth": 8})
    assert np.array_equal(smem_rows(recs, n), oracle.smem(ref_bwt(S, 0, 3), Q.q, Q.qoff, 31, 1))
    rb.rb3_merge(idx, build(S, 3, 6))
    for K in (8, 5, 9):  # same depth after the merge, a shallower one, a deeper one
        recs, n = rb.rb3_mem_search_opts(idx, dq, doff, 31, 1, {"hot_depth": K})
        assert np.array_equal(smem_rows(recs, n), oracle.smem(ref_bwt(S), Q.q, Q.qoff, 31, 1)), K


def test_smem_capacity_and_single_strand_rejected():
    S = synth.pangenome(seed=33, founder_len=2000, n_hap=3, batch=3)
    idx = build(S)
    Q = synth.mem_queries(S, seed=34, nq=50, median=100, lo=40, hi=200, sub=0.0)
    want = oracle.smem(ref_bwt(S), Q.q, Q.qoff, 10, 1)
    assert len(want) > 3
    out = np.empty(2, dtype=rb.SMEM_DTYPE)
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_mem_search(idx, Q.q, Q.qoff, 10, 1, out=out, cap=2)
    assert e.value.code == rb.RB3_E_CAPACITY
    ss = build(S, single_strand=1)
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_mem_search(ss, Q.q, Q.qoff, 10, 1)
    assert e.value.code == rb.RB3_E_INVAL


def test_invalid_symbols_rejected():
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_build_batch(np.array([1, 2, 7], np.uint8), np.array([3], np.int64))
    assert e.value.code == rb.RB3_E_INVAL
    S = synth.pangenome(seed=35, founder_len=500, n_hap=2, batch=2)
    idx = build(S)
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_backward_search(idx, np.array([1, 0, 2], np.uint8), np.array([0, 3], np.int64))
    assert e.value.code == rb.RB3_E_INVAL


def test_pangenome_medium_incremental():
    """Near-identical haplotypes (long exact matches, both strands): batch builds
    and segmented merges against the oracle's own incremental build."""
    S = synth.pangenome(seed=41, founder_len=60_000, n_hap=12, batch=4)
    T = oracle.concat(S.seq, S.lens, True)
    want = oracle.build_incremental(S.seq, S.lens, True, 1, nthreads=4)
    assert oracle.certify(want, T) == 0
    idx = build(S, 0, 4)
    for b0, b1 in [(4, 8), (8, 12)]:
        rb.rb3_merge_opts(idx, build(S, b0, b1), {"seg_len": 997})
    check_index(idx, want)
    # plain Algorithm 1 form of the same merges
    idx2 = build(S, 0, 4)
    for b0, b1 in [(4, 8), (8, 12)]:
        rb.rb3_merge_opts(idx2, build(S, b0, b1), {"merge_form": 1})
    check_index(idx2, want)


@pytest.mark.parametrize("D", [32, 64])
def test_save_load_resume(tmp_path, D):
    S = synth.pangenome(seed=51, founder_len=5000, n_hap=6, batch=2)
    idx = build(S, 0, 2, occ_interval=D)
    rb.rb3_merge(idx, build(S, 2, 4, occ_interval=D))
    p = str(tmp_path / "x.rb3")
    rb.rb3_index_save(idx, p)
    back = rb.rb3_index_load(p)
    assert rb.rb3_index_info(back)["has_build_data"] is False
    rb.rb3_merge(back, build(S, 4, 6, occ_interval=D))  # resume: load + further merge
    rb.rb3_merge(idx, build(S, 4, 6, occ_interval=D))
    check_index(back, ref_bwt(S), D)
    check_index(idx, ref_bwt(S), D)


def test_append_batches_pipeline():
    """Build-and-merge of several batches with builds overlapping merges equals
    building and merging them one by one (and the oracle)."""
    S = synth.pangenome(seed=71, founder_len=40_000, n_hap=15, batch=3)
    want = oracle.build_incremental(S.seq, S.lens, True, 1, nthreads=4)
    ends = np.array([b for (_, b) in S.batches[1:]], dtype=np.int64) - S.batches[0][1]
    off = S.offsets
    rest = S.seq[off[S.batches[0][1]]:]
    lens = S.lens[S.batches[0][1]:].copy()
    for host in (False, True):
        idx = build(S, 0, S.batches[0][1])
        seq = rest.copy() if host else torch.from_numpy(rest.copy()).to(DEV)
        rb.rb3_append_batches(idx, seq, lens, ends)
        check_index(idx, want)
    # an empty index as the start, batches of different sizes, empty batches,
    # strings on the device and on the host (copies staged a batch ahead)
    for host in (False, True):
        idx = rb.rb3_index_empty()
        seq = S.seq.copy() if host else torch.from_numpy(S.seq.copy()).to(DEV)
        rb.rb3_append_batches(idx, seq, S.lens.copy(), np.array([0, 2, 2, 7, 15], dtype=np.int64))
        check_index(idx, want)


def test_bounded_wait_times_out_and_context_survives():
    """The look-back wait of the radix passes, run by the self-test on a flag
    that nothing sets, gives up after its limit and reports RB3_E_TIMEOUT; the
    context stays usable (a build afterwards matches the oracle)."""
    import time
    t0 = time.time()
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_selftest_wait(1 << 16)
    assert e.value.code == rb.RB3_E_TIMEOUT
    assert time.time() - t0 < 30
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_selftest_wait(0)
    assert e.value.code == rb.RB3_E_INVAL
    g = synth.rng(55)
    S = synth.random_strings(g, 20, 400, n_frac=0.0)
    check_index(build(S), ref_bwt(S))


def test_walk_stats_count_every_new_symbol_once():
    """The walk's counters: one rank read per new symbol except the strings'
    sentinels (n2 - m2), plus one per position walked a second time from a
    resolved segment top, whatever the segment length and seed cap; seeds at
    most one per segment below a sentinel."""
    S = synth.pangenome(seed=93, founder_len=30_000, n_hap=6, batch=3)
    for L, cap in ((50, 0), (700, 0), (50, 8), (700, 100000)):
        idx = build(S, 0, 3)
        src = build(S, 3, 6)
        info = rb.rb3_index_info(src)
        rb.rb3_walk_stats(reset=True)
        rb.rb3_merge_opts(idx, src, {"seg_len": L, "seed_cap": cap})
        st = rb.rb3_walk_stats(reset=True)
        assert st["walk_block_reads"] - st["walked_again"] == info["n"] - info["m"], st
        if cap == 100000:
            assert st["walked_again"] == 0, st  # every seed resolved: nothing to walk again
        # both strands of each haplotype are strings of len + 1 symbols, cut every L from their end
        seeds_max = 2 * sum(-(-(int(l) + 1) // L) - 1 for l in S.lens[3:6])
        assert 0 < st["seeds"] <= seeds_max, (st, seeds_max)
        assert st["seed_block_reads"] >= st["seeds"]
        check_index(idx, ref_bwt(S))


def test_append_batch_memory_budget():
    """batch_mb cuts each caller batch into runs of whole strings that fit the
    budget: the same BWT (against the oracle), a lower device-memory peak."""
    S = synth.pangenome(seed=91, founder_len=20_000, n_hap=8, batch=4)
    B = ref_bwt(S)
    ends = np.array([b for (_, b) in S.batches], dtype=np.int64)
    seq = torch.from_numpy(S.seq.copy()).to(DEV)
    peaks = []
    for mb in (0, 1):
        idx = rb.rb3_index_empty()
        torch.cuda.synchronize()
        rb.rb3_device_peak(reset=True)
        rb.rb3_append_batches(idx, seq, S.lens.copy(), ends, {"batch_mb": mb})
        torch.cuda.synchronize()
        peaks.append(rb.rb3_device_peak())
        check_index(idx, B)
        idx.free()
    assert peaks[1] < peaks[0], peaks
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_append_batches(rb.rb3_index_empty(), seq, S.lens.copy(), ends, {"batch_mb": -1})
    assert e.value.code == rb.RB3_E_INVAL


def test_append_batches_error_propagates():
    S = synth.pangenome(seed=72, founder_len=5_000, n_hap=6, batch=2)
    seq = S.seq.copy()
    seq[S.offsets[4] + 10] = 9  # invalid symbol in the third batch
    idx = rb.rb3_index_empty()
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_append_batches(idx, seq, S.lens.copy(), np.array([2, 4, 6], dtype=np.int64))
    assert e.value.code == rb.RB3_E_INVAL


def test_autotuner_choices_keep_results():
    S = synth.pangenome(seed=91, founder_len=50_000, n_hap=8, batch=4)
    want = oracle.build_incremental(S.seq, S.lens, True, 1, nthreads=4)
    idx = build(S, 0, 4)
    src = build(S, 4, 8)
    best, ms = rb.rb3_tune_merge(idx, src)
    assert best.seg_len >= 256 and ms > 0
    check_index(idx, oracle.bwt(oracle.concat(S.subset(0, 4).seq, S.subset(0, 4).lens, True)))  # untouched
    rb.rb3_merge(idx, src)  # uses the remembered segment length
    check_index(idx, want)
    Q = synth.mem_queries(S, seed=92, nq=2000, median=150, lo=31, hi=3000)
    q, qoff = torch.from_numpy(Q.q).to(DEV), torch.from_numpy(Q.qoff).to(DEV)
    best, ms = rb.rb3_tune_search(idx, q, qoff, 31, 1)
    assert best.chunk_len in (64, 128, 256, 512, 1024, 4096)
    assert best.hot_depth in (-1, 6, 8, 10)
    recs, n = rb.rb3_mem_search(idx, q, qoff, 31, 1)  # the remembered chunk length and depth
    assert np.array_equal(smem_rows(recs, n), oracle.smem(want, Q.q, Q.qoff, 31, 1))


# ---- locate (sampled suffix array) ------------------------------------------

@pytest.mark.parametrize("D", [32, 64])
@pytest.mark.parametrize("both", [True, False])
def test_locate_every_row_vs_oracle(D, both):
    """Every row of indexes built from several batches (merged into an empty
    index, segmented and plain merges) located against the oracle's S(i)."""
    g = synth.rng(800 + D + both)
    for trial, s in enumerate((2, 8, 32)):
        n_str = int(g.integers(3, 30))
        S = synth.random_strings(g, n_str, int(g.integers(5, 500)), n_frac=0.03, allow_empty=True)
        cuts = sorted(set([0, n_str] + [int(c) for c in g.integers(0, n_str, size=2)]))
        opts = {"occ_interval": D, "single_strand": int(not both), "sa_sample": s}
        idx = rb.rb3_index_empty(opts)
        for a, b in zip(cuts[:-1], cuts[1:]):
            part = build(S, a, b, host=bool(trial & 1), **opts)
            assert rb.rb3_index_info(part)["sa_sample"] == s
            rb.rb3_merge_opts(idx, part, dict(opts, merge_form=trial % 3, seg_len=int(g.integers(3, 64))))
        assert rb.rb3_index_info(idx)["sa_sample"] == s
        T = oracle.concat(S.seq, S.lens, both)
        rows = np.arange(len(T), dtype=np.int64)
        want = oracle.locate(T, oracle.suffix_array(T), rows)
        assert np.array_equal(rb.rb3_locate(idx, rows), want)
        assert np.array_equal(rb.rb3_locate(idx, torch.from_numpy(rows).to(DEV)), want)  # device rows


def test_locate_smem_hits_spell_the_queries():
    """SMEM intervals of a pangenome index located: each hit's string, from its
    offset, spells the query's SMEM; and it equals the oracle's S(i)."""
    S = synth.pangenome(seed=61, founder_len=30_000, n_hap=9, batch=3)
    opts = {"sa_sample": 16}
    idx = rb.rb3_index_empty(opts)
    ends = np.array([b for (_, b) in S.batches], dtype=np.int64)
    rb.rb3_append_batches(idx, torch.from_numpy(S.seq.copy()).to(DEV), S.lens.copy(), ends, opts)
    Q = synth.mem_queries(S, seed=62, nq=400, median=120, lo=31, hi=800, sub=0.01)
    recs, n = rb.rb3_mem_search(idx, torch.from_numpy(Q.q).to(DEV), torch.from_numpy(Q.qoff).to(DEV), 31, 1)
    assert n > 100
    rows = recs["k"].astype(np.int64)
    loc = rb.rb3_locate(idx, rows)
    T = oracle.concat(S.seq, S.lens, True)
    assert np.array_equal(loc, oracle.locate(T, oracle.suffix_array(T), rows))
    comp = np.array([0, 4, 3, 2, 1, 5], dtype=np.uint8)
    ds = []
    for o, l in zip(S.offsets[:-1], S.lens):
        s_ = S.seq[o:o + l]
        ds += [s_, comp[s_[::-1]]]
    for r, (t, off) in zip(recs, loc):
        q = Q.q[Q.qoff[r["qid"]] + r["start"]:Q.qoff[r["qid"]] + r["end"]]
        assert np.array_equal(ds[t][off:off + len(q)], q)


def test_locate_errors_and_save_load(tmp_path):
    S = synth.pangenome(seed=63, founder_len=4_000, n_hap=4, batch=2)
    plain = build(S)
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_locate(plain, np.array([0], np.int64))
    assert e.value.code == rb.RB3_E_INVAL
    idx = build(S, 0, 2, sa_sample=8)
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_locate(idx, np.array([rb.rb3_index_info(idx)["n"]], np.int64))
    assert e.value.code == rb.RB3_E_INVAL
    other = build(S, 0, 2, sa_sample=8)
    rb.rb3_merge(other, build(S, 2, 4, sa_sample=4))  # different rates: the merge keeps no sample
    assert rb.rb3_index_info(other)["sa_sample"] == 0
    rb.rb3_merge(idx, build(S, 2, 4, sa_sample=8))
    p = str(tmp_path / "s.rb3")
    rb.rb3_index_save(idx, p)
    back = rb.rb3_index_load(p)
    rows = np.arange(rb.rb3_index_info(idx)["n"], dtype=np.int64)
    assert rb.rb3_index_info(back)["sa_sample"] == 8
    assert np.array_equal(rb.rb3_locate(back, rows), rb.rb3_locate(idx, rows))
    T = oracle.concat(S.seq, S.lens, True)
    assert np.array_equal(rb.rb3_locate(back, rows), oracle.locate(T, oracle.suffix_array(T), rows))


@pytest.mark.parametrize("form", [0, 1, 2, 3])
def test_merge_in_parts_equals_the_oracle(form):
    """The merge split into parts (as over several GPUs, here one after the
    other on one): each part's rows are Algorithm 1's positions of its own
    strings' suffixes and 0 elsewhere, the parts add up to the oracle's whole
    position array, and applying it gives the oracle's merged BWT."""
    g = synth.rng(4300 + form)
    S = synth.random_strings(g, 17, 900, n_frac=0.02, allow_empty=True)
    a, b = 6, 17
    B1 = ref_bwt(S, 0, a)
    sub = S.subset(a, b)
    T2 = oracle.concat(sub.seq, sub.lens, True)
    SA2 = oracle.suffix_array(T2)
    _, want = oracle.merge(B1, oracle.bwt_from_sa(T2, SA2), want_pos=True)
    string_of_row = np.searchsorted(np.flatnonzero(T2 == 0), SA2) // 2
    opts = {"merge_form": form, "seg_len": 40, "seed_cap": 8}
    for parts in (1, 2, 3):
        dst, src = build(S, 0, a), build(S, a, b)
        owner = rb.rb3_merge_partition(S.lens[a:b], parts)
        total = torch.zeros(len(T2), dtype=torch.int64, device=DEV)
        for p in range(parts):
            pos = torch.full((len(T2),), -7, dtype=torch.int64, device=DEV)
            rb.rb3_merge_positions(dst, src, pos, owner, p, opts)
            got = pos.cpu().numpy()
            mine = owner[string_of_row] == p
            assert np.array_equal(got[mine], want[mine]) and not got[~mine].any(), (parts, p)
            total += pos
        assert np.array_equal(total.cpu().numpy(), want)
        rb.rb3_merge_apply(dst, src, total)
        check_index(dst, ref_bwt(S, 0, b))
    # into an empty index: the part owning string 0 writes every row
    empty, src = rb.rb3_index_empty(), build(S, a, b)
    owner = rb.rb3_merge_partition(S.lens[a:b], 2)
    total = torch.zeros(len(T2), dtype=torch.int64, device=DEV)
    for p in range(2):
        pos = torch.empty(len(T2), dtype=torch.int64, device=DEV)
        rb.rb3_merge_positions(empty, src, pos, owner, p, opts)
        total += pos
    rb.rb3_merge_apply(empty, src, total.cpu().numpy())  # host pos
    check_index(empty, ref_bwt(S, a, b))


def test_merge_apply_refuses_bad_positions():
    g = synth.rng(4400)
    S = synth.random_strings(g, 8, 300, allow_empty=False)
    dst, src = build(S, 0, 4), build(S, 4, 8)
    before = rb.rb3_export(dst)
    n2 = rb.rb3_index_info(src)["n"]
    pos = torch.zeros(n2, dtype=torch.int64, device=DEV)
    rb.rb3_merge_positions(dst, src, pos)
    for bad in ("dup", "neg", "past"):
        p = pos.clone()
        if bad == "dup":
            p[5] = p[4]
        elif bad == "neg":
            p[0] = -1
        else:
            p[-1] = rb.rb3_index_info(dst)["n"] + n2
        with pytest.raises(rb.RB3Error) as e:
            rb.rb3_merge_apply(dst, src, p)
        assert e.value.code == rb.RB3_E_INVAL
        assert np.array_equal(rb.rb3_export(dst), before)
    rb.rb3_merge_apply(dst, src, pos)
    check_index(dst, ref_bwt(S))


def test_tune_build_picks_a_layout_and_the_result_is_exact():
    """rb3_tune_build on the first two batches of an uneven-genome input: the
    fastest D among 32/64/128 with its segment length and seed cap; appending
    every batch with those options gives the oracle's BWT; a budget that only
    the D = 128 layout fits (1 MiB for ~1.2 Msym: 1.14 MiB at D = 32 or 64,
    0.86 at 128) gives D = 128."""
    S = synth.uneven(n_founders=3, founder_len=60_000, n_genomes=12, per_cluster=4, median=50_000, sigma=0.0,
                     lo=50_000, hi=50_000, batch=4)
    ends = np.array([b for (_, b) in S.batches], dtype=np.int64)
    best, table = rb.rb3_tune_build(S.seq, S.lens, ends)
    assert [d for d, _, _ in table] == [32, 64, 128] and all(ms > 0 for _, ms, _ in table)
    assert best.occ_interval == min(table, key=lambda t: t[1])[0]
    assert best.seg_len > 0 and best.seed_cap > 0
    idx = rb.rb3_index_empty(best)
    rb.rb3_append_batches(idx, torch.from_numpy(S.seq.copy()).to(DEV), S.lens, ends, best)
    check_index(idx, ref_bwt(S), best.occ_interval)
    small, table = rb.rb3_tune_build(torch.from_numpy(S.seq.copy()).to(DEV), S.lens, ends, index_mb=1)
    assert table[2][2] <= 1 < table[0][2] and table[0][2] == table[1][2]
    assert small.occ_interval == 128
    idx = rb.rb3_index_empty(small)
    rb.rb3_append_batches(idx, torch.from_numpy(S.seq.copy()).to(DEV), S.lens, ends, small)
    check_index(idx, ref_bwt(S), 128)
