"""Full-size GPU parity on the benchmark workload (pangenome merge: 5 Mb founder,
50 haplotypes, batches of 10, both strands, ~500 Msym), in the configuration
bench.py times (default options), against the oracle's own incremental build
(naive sort per haplotype + Algorithm 1 merges), plus the LF-decode certificate;
MEM search on the finished index checked on a sample of the 1 M queries,
haplotype diversity on a sample of the bench's sliding k-mers, the
uneven-genome workload (clusters, N-runs) reduced (against the oracle's
build) and at its size (certified), and the ~6 Gsym served index (certified,
and pinned by backward-search additivity)."""
import os

import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2409_00613_gb300 as rb

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
DEV = torch.device("cuda:0")
FIELDS = ("qid", "start", "end", "k", "kp", "s")
NTH = os.cpu_count() or 4


def host_memory_bytes() -> int:
    """Memory this process may still use on the host: MemAvailable, capped by
    the cgroup limit when there is one."""
    avail = 0
    with open("/proc/meminfo") as f:
        for line in f:
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
    for path in ("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory/memory.limit_in_bytes"):
        try:
            with open(path) as f:
                v = f.read().strip()
            if v != "max":
                avail = min(avail, int(v))
        except (OSError, ValueError):
            pass
    return avail


def gpu_incremental(S, opts=None):
    off = S.offsets
    idx = None
    for a, b in S.batches:
        part = rb.rb3_build_batch(torch.from_numpy(S.seq[off[a]:off[b]].copy()).to(DEV), S.lens[a:b].copy(),
                                  opts=opts)
        if idx is None:
            idx = part
        else:
            rb.rb3_merge_opts(idx, part, opts)
            part.free()
    return idx


@pytest.fixture(scope="module")
def pangenome_full():
    S = synth.pangenome()
    idx = gpu_incremental(S)
    want = oracle.build_incremental(S.seq, S.lens, True, 1, nthreads=NTH)
    return S, idx, want


def test_pangenome_full_bwt_equals_oracle(pangenome_full):
    S, idx, want = pangenome_full
    codes, occ = rb.rb3_export(idx, want_occ=True)
    assert len(codes) == len(want) == S.ds_symbols()
    assert np.array_equal(codes, want)
    T = oracle.concat(S.seq, S.lens, True)
    assert oracle.certify(codes, T, nthreads=NTH) == 0
    info = rb.rb3_index_info(idx)
    assert np.array_equal(occ, oracle.occ_table(want, info["occ_interval"]))
    assert info["m"] == 100 and info["C"] == list(oracle.counts(want))


def test_pangenome_full_mem_search_sample(pangenome_full):
    S, idx, want = pangenome_full
    Q = synth.mem_queries(S)  # the 1 M benchmark queries
    recs, n = rb.rb3_mem_search(idx, torch.from_numpy(Q.q).to(DEV), torch.from_numpy(Q.qoff).to(DEV), 31, 1,
                                cap=Q.nq * 8)
    got = np.stack([recs[f].astype(np.int64) for f in FIELDS], axis=1)
    g = synth.rng(7)
    sample = np.sort(g.choice(Q.nq, size=10_000, replace=False))
    sub = Q.subset(sample)
    ref = oracle.smem(want, sub.q, sub.qoff, 31, 1, nthreads=NTH)
    # map the sample's records back to their global query ids
    ref[:, 0] = sample[ref[:, 0]]
    mask = np.isin(got[:, 0], sample)
    assert np.array_equal(got[mask], ref)
    # backward search on the same sample
    lohi = rb.rb3_backward_search(idx, sub.q, sub.qoff)
    assert np.array_equal(lohi, oracle.backward_search(want, sub.q, sub.qoff))


def test_pangenome_full_diversity_sample(pangenome_full):
    """Haplotype diversity in the configuration bench.py times (the 20,000
    sliding 51-mers of its leg, default scores, W = 25, filter on) on the
    finished index; 200 sampled queries against the oracle on its own BWT."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    S, idx, want = pangenome_full
    q, qoff = bench.diversity_kmers(S)
    out, n = rb.rb3_haplotype_diversity(idx, torch.from_numpy(q).to(DEV), torch.from_numpy(qoff).to(DEV), 1, 3, 5,
                                        2, 25, True, out=torch.empty((len(qoff) - 1, 25, 4), dtype=torch.int64,
                                                                     device=DEV),
                                        n_out=torch.empty(len(qoff) - 1, dtype=torch.int64, device=DEV))
    out, n = out.cpu().numpy(), n.cpu().numpy()
    sample = np.sort(synth.rng(11).choice(len(n), size=200, replace=False))
    sq = np.concatenate([q[qoff[i]:qoff[i + 1]] for i in sample])
    soff = np.arange(len(sample) + 1, dtype=np.int64) * 51
    ref, nref = oracle.haplotype_diversity_many(want, sq, soff, 1, 3, 5, 2, 25, True)
    assert np.array_equal(n[sample], nref)
    for j, i in enumerate(sample):
        assert np.array_equal(out[i, :n[i]], ref[j, :nref[j]]), i
    assert (n > 0).mean() > 0.5


def test_uneven_genomes_reduced():
    """Uneven-genome shape at reduced size: 6 clusters, lognormal lengths, 1%
    substitutions, 0.5% N-runs of 10-100, batches of 16 genomes."""
    S = synth.uneven(n_founders=6, founder_len=300_000, n_genomes=60, per_cluster=10, median=150_000, sigma=0.35,
                     lo=50_000, hi=300_000, batch=16)
    idx = gpu_incremental(S)
    codes = rb.rb3_export(idx)
    want = oracle.build_incremental(S.seq, S.lens, True, 1, nthreads=NTH)
    assert np.array_equal(codes, want)
    assert oracle.certify(codes, oracle.concat(S.seq, S.lens, True), nthreads=NTH) == 0


def test_uneven_genomes_full():
    """The uneven-genome workload at its size: 2,000 genomes in 20 clusters
    (lognormal lengths, median 3 Mb, 1% substitutions, 0.5% N-runs of 10-100),
    both strands (~12.8 Gsym), appended in 32 batches of 64 genomes through
    rb3_append_batches; the finished BWT is certified by the oracle's LF-decode
    certificate against the text (too large for its naive sort), and its symbol
    counts checked."""
    need = 60 << 30  # strings, exported BWT, text, certificate's marks and rank table
    if host_memory_bytes() < need:
        pytest.skip(f"needs {need >> 30} GiB of host memory for the certificate")
    S = synth.uneven()
    off = S.offsets
    ends = np.array([b for (_, b) in S.batches], dtype=np.int64)
    idx = rb.rb3_index_empty()
    seq = torch.from_numpy(S.seq).to(DEV)
    rb.rb3_append_batches(idx, seq, S.lens.copy(), ends)
    del seq
    info = rb.rb3_index_info(idx)
    assert info["n"] == S.ds_symbols() and info["m"] == 2 * len(S.lens) == 4000
    codes = rb.rb3_export(idx)
    idx.free()
    T = oracle.concat(S.seq, S.lens, True)
    del S, off
    assert list(oracle.counts(codes)) == list(oracle.counts(T))
    assert oracle.certify(codes, T, nthreads=NTH) == 0


def test_occ32_index_past_2_to_32():
    """D = 32 keeps 32-bit counts relative to 2^32-symbol spans.  The served
    index (150 Mb founder, 20 haplotypes, batches of 4: ~6 Gsym) crosses 2^32
    after four batches, so the last merge walks over span 1 and writes span
    bases.  Pins that hold at any size: every backward-search interval of the
    merged index is the sum of the batches' intervals (a pattern without $
    compares with each suffix by its first |P| symbols only, so lo and hi add up
    over the batches), checked on patterns sampled from every batch."""
    S = synth.served_index_strings()
    off = S.offsets
    opts = {"occ_interval": 32}
    parts = []
    idx = rb.rb3_index_empty(opts)
    for a, b in S.batches:
        dev_seq = torch.from_numpy(S.seq[off[a]:off[b]].copy()).to(DEV)
        part = rb.rb3_build_batch(dev_seq, S.lens[a:b].copy(), opts=opts)
        del dev_seq
        rb.rb3_merge_opts(idx, part, opts)
        rb.rb3_drop_build_data(part)
        parts.append(part)
    info = rb.rb3_index_info(idx)
    assert info["n"] == S.ds_symbols() > 2**32 and info["occ_interval"] == 32
    # the whole BWT certified against the text by the oracle's LF-decode certificate
    if host_memory_bytes() >= (30 << 30):
        codes = rb.rb3_export(idx)
        assert oracle.certify(codes, oracle.concat(S.seq, S.lens, True), nthreads=NTH) == 0
        del codes
    g = synth.rng(4242)
    pats = [np.array([c], np.uint8) for c in range(1, 6)]
    for _ in range(4000):
        L = int(g.integers(2, 60))
        s = int(g.integers(0, len(S.seq) - L))
        p = S.seq[s:s + L].copy()
        if g.random() < 0.2:
            p[int(g.integers(0, L))] = int(g.integers(1, 5))
        pats.append(p)
    q = np.concatenate(pats)
    qoff = np.concatenate([[0], np.cumsum([len(p) for p in pats])]).astype(np.int64)
    got = rb.rb3_backward_search(idx, q, qoff)
    want = sum(rb.rb3_backward_search(p, q, qoff) for p in parts)
    assert np.array_equal(got, want)
    assert (got[:, 1] > 2**32).sum() > 100  # intervals in the second span were exercised
    for p in parts:
        p.free()
    # the run-length copy keeps the span bases: the same intervals.  Merged with
    # an empty index: the same again; merged with one empty string (two new
    # sentinels, which sort before every letter): every interval moves up by two
    R = rb.rb3_index_compress(idx, 2048)
    assert rb.rb3_index_info(R)["run_length"]
    assert np.array_equal(rb.rb3_backward_search(R, q, qoff), got)
    rb.rb3_merge(R, rb.rb3_index_empty(opts))
    assert np.array_equal(rb.rb3_backward_search(R, q, qoff), got)
    empty_string = rb.rb3_build_batch(np.zeros(0, np.uint8), np.zeros(1, np.int64), opts=opts)
    rb.rb3_merge(R, empty_string)
    assert rb.rb3_index_info(R)["n"] == info["n"] + 2
    assert np.array_equal(rb.rb3_backward_search(R, q, qoff), got + 2)
    # three 5 kb windows merged into the run-length index directly (its walk
    # ranks spans on both sides of 2^32, its span bases are rewritten) and into
    # the plain one: the run-length result is the compressed plain result --
    # the BWT, every span header's ranks (span bases added) and the run count
    rb.rb3_merge(idx, empty_string)
    g2 = synth.rng(4343)
    starts = g2.integers(0, len(S.seq) - 5000, size=3)
    sseq = np.concatenate([S.seq[s:s + 5000] for s in starts]).astype(np.uint8)
    for x in (idx, R):
        rb.rb3_merge(x, rb.rb3_build_batch(torch.from_numpy(sseq).to(DEV), np.full(3, 5000, np.int64), opts=opts))
    R2 = rb.rb3_index_compress(idx, 2048)
    n = info["n"] + 2 + 2 * (15000 + 3)  # both strands, each string with its sentinel
    assert rb.rb3_index_info(R)["n"] == n
    codes = [torch.empty(n, dtype=torch.uint8, device=DEV) for _ in range(2)]
    occ = [torch.empty((n // 2048 + 1, 6), dtype=torch.int64, device=DEV) for _ in range(2)]
    for x, c, o in zip((R, R2), codes, occ):
        rb.rb3_export(x, codes=c, occ=o)
    torch.cuda.synchronize()
    assert torch.equal(codes[0], codes[1]) and torch.equal(occ[0], occ[1])
    assert rb.rb3_index_bytes(R) == rb.rb3_index_bytes(R2)
    del codes, occ
    R2.free()
    R.free()
    idx.free()
