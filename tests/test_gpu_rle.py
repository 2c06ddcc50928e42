"""GPU parity of the run-length index (Section "BWT construction", Fig. 2b):
compressed copies of plain indexes against the CPU oracle, bit-exact — the
BWT and its runs, the span-start ranks, backward search, SMEM search in every
form, locate, save / load — and the calls that must refuse one."""
import time

import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2409_00613_gb300 as rb

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
FIELDS = ("qid", "start", "end", "k", "kp", "s")


def build(S, s0=0, s1=None, **opts):
    s1 = len(S.lens) if s1 is None else s1
    off = S.offsets
    seq = torch.from_numpy(S.seq[off[s0]:off[s1]].copy()).to(DEV)
    return rb.rb3_build_batch(seq, S.lens[s0:s1].copy(), opts=opts or None)


def ref(S, a, b):
    sub = S.subset(a, b)
    return oracle.bwt(oracle.concat(sub.seq, sub.lens, True))


def smem_rows(recs, n):
    if n == 0:
        return np.zeros((0, 6), dtype=np.int64)
    return np.stack([recs[f].astype(np.int64) for f in FIELDS], axis=1)


def check_rle(R, B, span):
    info = rb.rb3_index_info(R)
    assert info["run_length"] and info["occ_interval"] == span
    assert info["n"] == len(B) and info["C"] == list(oracle.counts(B))
    codes, occ = rb.rb3_export(R, want_occ=True)
    assert np.array_equal(codes, B)
    assert np.array_equal(occ, oracle.occ_table(B, span))
    sym, ln = oracle.runs(B, span)
    assert rb.rb3_index_bytes(R)["runs"] == len(sym)


@pytest.mark.parametrize("span", [512, 1024, 16384])
@pytest.mark.parametrize("both", [True, False])
def test_rle_export_and_backward_search(span, both):
    """Random string lists (N symbols, empty strings) and a pangenome, several
    tiles of spans and a ragged last span: exported BWT, span-start ranks and
    run count against the oracle; backward search against the oracle."""
    g = synth.rng(900 + span % 1000 + both)
    cases = [synth.random_strings(g, 40, 300, n_frac=0.05, allow_empty=True),
             synth.pangenome(seed=901, founder_len=20_000, n_hap=6, batch=6)]
    for S in cases:
        B = oracle.bwt(oracle.concat(S.seq, S.lens, both))
        for D in (32, 64):
            idx = build(S, occ_interval=D, single_strand=int(not both))
            R = rb.rb3_index_compress(idx, span)
            check_rle(R, B, span)
            pats = [np.zeros(0, np.uint8), np.array([5], np.uint8)]
            for _ in range(300):
                L = int(g.integers(1, 40))
                s = int(g.integers(0, len(S.seq) - L))
                pats.append(S.seq[s:s + L].copy() if g.random() < 0.8 else synth.random_bases(g, L))
            q = np.concatenate(pats)
            qoff = np.concatenate([[0], np.cumsum([len(p) for p in pats])]).astype(np.int64)
            want = oracle.backward_search(B, q, qoff)
            assert np.array_equal(rb.rb3_backward_search(R, q, qoff), want)
            assert np.array_equal(rb.rb3_backward_search(idx, q, qoff), want)


def test_rle_empty_and_tiny_indexes():
    """Empty index, one string, all-empty strings: spans with no runs."""
    E = rb.rb3_index_empty()
    R = rb.rb3_index_compress(E)
    assert rb.rb3_index_info(R)["n"] == 0
    assert rb.rb3_index_bytes(R)["runs"] == 0
    for seqs in ([np.array([1, 1, 1, 2], np.uint8)], [np.zeros(0, np.uint8)] * 5):
        S = synth.Strings(np.concatenate(seqs), np.array([len(s) for s in seqs], np.int64))
        B = oracle.bwt(oracle.concat(S.seq, S.lens, True))
        R = rb.rb3_index_compress(build(S), 512)
        check_rle(R, B, 512)


@pytest.mark.parametrize("span", [512, 4096])
@pytest.mark.parametrize("ell,smin", [(1, 1), (12, 2), (19, 1)])
def test_rle_smem_all_forms_vs_oracle(span, ell, smin):
    S = synth.pangenome(seed=31, founder_len=3000, n_hap=6, batch=3)
    B = oracle.bwt(oracle.concat(S.seq, S.lens, True))
    idx = build(S, 0, 3)
    rb.rb3_merge(idx, build(S, 3, 6))
    R = rb.rb3_index_compress(idx, span)
    Q = synth.mem_queries(S, seed=32, nq=300, median=80, lo=1, hi=600, sub=0.02)
    want = oracle.smem(B, Q.q, Q.qoff, ell, smin)
    q, qoff = torch.from_numpy(Q.q).to(DEV), torch.from_numpy(Q.qoff).to(DEV)
    for form in (0, 1, 2):
        for chunk in (0, 17):
            recs, n = rb.rb3_mem_search_opts(R, q, qoff, ell, smin, {"chunk_len": chunk, "search_form": form})
            assert np.array_equal(smem_rows(recs, n), want), (form, chunk)
    cap = max(len(want), 1)
    out = torch.empty(40 * cap, dtype=torch.uint8, device=DEV)
    n = rb.rb3_mem_search_noalloc(R, q, qoff, ell, smin, out, cap)
    assert np.array_equal(smem_rows(out[:n * 40].cpu().numpy().view(rb.SMEM_DTYPE), n), want)


def test_rle_locate_save_load_and_refusals(tmp_path):
    """Locate every row of a compressed index with a sampled suffix array;
    save / load keeps every byte; a damaged image is refused on load; bad
    spans, double compression and merge tuning are refused."""
    S = synth.pangenome(seed=63, founder_len=6_000, n_hap=6, batch=3)
    idx = build(S, 0, 3, sa_sample=8)
    rb.rb3_merge(idx, build(S, 3, 6, sa_sample=8))
    R = rb.rb3_index_compress(idx, 1024)
    assert rb.rb3_index_info(R)["sa_sample"] == 8
    T = oracle.concat(S.seq, S.lens, True)
    B = oracle.bwt(T)
    rows = np.arange(len(T), dtype=np.int64)
    want = oracle.locate(T, oracle.suffix_array(T), rows)
    assert np.array_equal(rb.rb3_locate(R, rows), want)
    p = str(tmp_path / "r.rb3")
    rb.rb3_index_save(R, p)
    back = rb.rb3_index_load(p)
    check_rle(back, B, 1024)
    assert np.array_equal(rb.rb3_locate(back, rows), want)
    assert rb.rb3_index_bytes(back) == rb.rb3_index_bytes(R)
    plain_bytes = rb.rb3_index_bytes(idx)["device_bytes"]
    assert rb.rb3_index_bytes(R)["device_bytes"] < plain_bytes
    # damage: one run's symbol changed to another (the span's counts then
    # disagree with the next header), and the payload size field enlarged
    raw = bytearray(open(p, "rb").read())
    n_spans = len(T) // 1024 + 1
    base = 8 + 12 * 8 + 64 * n_spans  # magic, header words, span headers (no span bases below 2^32)
    pb = int.from_bytes(raw[base:base + 8], "little")
    assert 0 < pb < len(raw)
    bad1 = bytearray(raw)
    first = base + 16
    bad1[first] = ((((bad1[first] >> 5) % 5) + 1) << 5) | (bad1[first] & 31)  # another symbol, same length
    bad2 = bytearray(raw)
    bad2[base:base + 8] = (pb + 1).to_bytes(8, "little")
    for k, bad in enumerate((bad1, bad2)):
        q = str(tmp_path / f"bad{k}.rb3")
        open(q, "wb").write(bytes(bad))
        with pytest.raises(rb.RB3Error) as e:
            rb.rb3_index_load(q)
        assert e.value.code == rb.RB3_E_IO
    for bad_span in (256, 1000, 32768):
        with pytest.raises(rb.RB3Error) as e:
            rb.rb3_index_compress(idx, bad_span)
        assert e.value.code == rb.RB3_E_INVAL
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_index_compress(R)
    assert e.value.code == rb.RB3_E_INVAL
    # merge tuning takes a run-length dst (the walk ranks its spans), not a run-length src
    best, ms = rb.rb3_tune_merge(R, build(S, 0, 1))
    assert best.seg_len >= 256 and ms > 0
    check_rle(R, B, 1024)  # not modified
    for call in (lambda: rb.rb3_tune_merge(idx, R),
                 lambda: rb.rb3_merge_positions(idx, R, pos=torch.zeros(len(B), dtype=torch.int64, device=DEV))):
        with pytest.raises(rb.RB3Error) as e:
            call()
        assert e.value.code == rb.RB3_E_INVAL
    # the plain index is untouched by all of it
    codes = rb.rb3_export(idx)
    assert np.array_equal(codes, B)


@pytest.mark.parametrize("span", [512, 2048])
def test_rle_merges_and_appends(span):
    """Merges with a run-length input on either side, and appends to a
    run-length index (merged into directly, its spans rewritten): the result
    against the oracle's BWT of the concatenation, the sampled suffix array
    carried along, the inputs unchanged."""
    S = synth.pangenome(seed=77, founder_len=5_000, n_hap=8, batch=2)
    T_all = oracle.concat(S.seq, S.lens, True)
    B_all = oracle.bwt(T_all)
    parts = [(0, 2), (2, 4), (4, 6), (6, 8)]
    opts = {"sa_sample": 4}
    # run-length dst, plain src (segmented and plain walk forms)
    R = rb.rb3_index_compress(build(S, 0, 2, **opts), span)
    for k, (a, b) in enumerate(parts[1:3]):
        src = build(S, a, b, **opts)
        rb.rb3_merge_opts(R, src, {"merge_form": k % 2})
        check_rle(R, ref(S, 0, b), span)
        assert np.array_equal(rb.rb3_export(src), ref(S, a, b))
    # plain dst, run-length src
    P = build(S, 0, 6, **opts)
    Rs = rb.rb3_index_compress(build(S, 6, 8, **opts), span)
    rb.rb3_merge(P, Rs)
    assert not rb.rb3_index_info(P)["run_length"]
    assert np.array_equal(rb.rb3_export(P), B_all)
    check_rle(Rs, ref(S, 6, 8), span)
    # both run-length
    rb.rb3_merge(R, Rs)
    check_rle(R, B_all, span)
    # append the last batches to a run-length index, in two batches
    A = rb.rb3_index_compress(build(S, 0, 4, **opts), span)
    off = S.offsets
    seq = torch.from_numpy(S.seq[off[4]:off[8]].copy()).to(DEV)
    rb.rb3_append_batches(A, seq, S.lens[4:8].copy(), np.array([2, 4], np.int64), opts)
    check_rle(A, B_all, span)
    rows = np.arange(len(T_all), dtype=np.int64)
    assert rb.rb3_index_info(A)["sa_sample"] == 4
    assert np.array_equal(rb.rb3_locate(A, rows), oracle.locate(T_all, oracle.suffix_array(T_all), rows))


def _image(idx, path):
    rb.rb3_index_save(idx, path)
    return open(path, "rb").read()


@pytest.mark.parametrize("span", [512, 2048, 16384])
@pytest.mark.parametrize("form", [0, 1, 3])
def test_rle_merge_image_equals_compressed_plain_merge(tmp_path, span, form):
    """A merge into a run-length index writes, byte for byte, the image that
    compressing the plain merge gives (span headers, marks, runs, sampled
    suffix array), and its BWT is the oracle's; single strand too."""
    S = synth.pangenome(seed=78, founder_len=7_000, n_hap=6, batch=2)
    for both in (True, False):
        opts = {"sa_sample": 8, "single_strand": 0 if both else 1}
        P = build(S, 0, 2, **opts)
        R = rb.rb3_index_compress(build(S, 0, 2, **opts), span)
        for a, b in ((2, 3), (3, 6)):
            o = {"merge_form": form, "seg_len": 512, "seed_cap": 256 if form != 3 else 0}
            rb.rb3_merge_opts(P, build(S, a, b, **opts), o)
            rb.rb3_merge_opts(R, build(S, a, b, **opts), o)
            sub = S.subset(0, b)
            B = oracle.bwt(oracle.concat(sub.seq, sub.lens, both))
            assert np.array_equal(rb.rb3_export(R), B), (span, form, both, b)
            want = _image(rb.rb3_index_compress(P, span), str(tmp_path / "c.rb3"))
            assert _image(R, str(tmp_path / "m.rb3")) == want, (span, form, both, b)


def test_rle_merge_edges_and_parts():
    """Merges into an empty run-length index, of an empty batch, of content the
    index already holds (an exact duplicate), and the merge in parts (two
    position arrays summed, then applied) into a run-length dst; the merge
    holds no plain copy of dst (device peak below one byte per indexed symbol)."""
    S = synth.pangenome(seed=79, founder_len=20_000, n_hap=6, batch=2)
    span = 1024
    E = rb.rb3_index_compress(rb.rb3_index_empty(), span)
    rb.rb3_merge(E, build(S, 0, 2))
    check_rle(E, ref(S, 0, 2), span)
    rb.rb3_merge(E, rb.rb3_build_batch(np.zeros(0, np.uint8), np.zeros(0, np.int64)))
    check_rle(E, ref(S, 0, 2), span)
    dup = build(S, 1, 2)  # haplotype 1 again
    rb.rb3_merge(E, dup)
    seq = np.concatenate([S.seq[:S.offsets[2]], S.seq[S.offsets[1]:S.offsets[2]]])
    lens = np.concatenate([S.lens[:2], S.lens[1:2]])
    check_rle(E, oracle.bwt(oracle.concat(seq, lens, True)), span)
    # in parts: each part's positions, summed, then applied to a run-length dst
    R = rb.rb3_index_compress(build(S, 0, 4), span)
    src = build(S, 4, 6)
    owner = rb.rb3_merge_partition(S.lens[4:6], 2)
    n2 = rb.rb3_index_info(src)["n"]
    total = torch.zeros(n2, dtype=torch.int64, device=DEV)
    for part in range(2):
        pos = torch.empty(n2, dtype=torch.int64, device=DEV)
        rb.rb3_merge_positions(R, src, owner=owner, part=part, pos=pos)
        total += pos
    n1 = rb.rb3_index_info(R)["n"]
    torch.cuda.synchronize()
    base = rb.rb3_device_peak(reset=True)  # in use now: dst, src and its build data
    rb.rb3_merge_apply(R, src, total)
    torch.cuda.synchronize()
    peak = rb.rb3_device_peak() - base
    check_rle(R, ref(S, 0, 6), span)
    # what the merge added at its peak: the merged runs and headers, the batch's
    # symbols (1 B each), span counts and offsets -- never a copy of dst's n1
    # symbols (a plain copy, the merged plain index and its codes: 3 n1 + 2 n2)
    assert peak < n1 + 2 * n2, (peak, n1, n2)


def test_rle_server_round_trip():
    """The continuous-batching server over a run-length index gives the
    oracle's SMEMs per request."""
    S = synth.pangenome(seed=71, founder_len=8_000, n_hap=4, batch=4)
    B = oracle.bwt(oracle.concat(S.seq, S.lens, True))
    R = rb.rb3_index_compress(build(S), 2048)
    Q = synth.mem_queries(S, seed=72, nq=64, median=150, lo=31, hi=800, sub=0.01)
    srv = rb.rb3_server_create(R, min_len=31)
    ids = []
    for i in range(64):
        ids.append(rb.rb3_server_submit(srv, Q.q[Q.qoff[i]:Q.qoff[i + 1]].copy(), tag=i))
    done, t0 = {}, time.time()
    while len(done) < 64:
        for c in rb.rb3_server_poll(srv, 64, 100000):
            done[int(c["req_id"])] = c
        assert time.time() - t0 < 120, "server did not complete the requests"
    for i, rid in enumerate(ids):
        c = done[rid]
        assert c["status"] == 0
        got = rb.rb3_server_take(srv, rid, int(c["n_smem"]))
        one = Q.q[Q.qoff[i]:Q.qoff[i + 1]]
        want = oracle.smem(B, one, np.array([0, len(one)], np.int64), 31, 1)
        rows = smem_rows(got, len(got))
        rows[:, 0] = 0
        assert np.array_equal(rows, want)
    rb.rb3_server_destroy(srv)
