"""GPU parity of local haplotype diversity (Section "Estimating local haplotype
diversity", Algorithm 5): every query's records (k, k', s, H), their order and
their number against the CPU oracle, bit-exact, on plain and run-length
indexes, with and without the redundancy filter, under several scores and
bands; edge cases and refusals."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SCORES = [(1, 3, 5, 2, 25), (2, 3, 5, 3, 8), (3, 3, 5, 2, 32), (1, 3, 5, 2, 1), (2, 4, 6, 2, 3)]


def diversity_queries(S, seed, nq, lo=6, hi=40):
    """Windows of the strings with substitutions, short indels and N, random
    bases, an empty query and an all-N query."""
    g = synth.rng(seed)
    pats = [np.zeros(0, np.uint8), np.full(5, 5, np.uint8)]
    off = S.offsets
    while len(pats) < nq:
        L = int(g.integers(lo, hi + 1))
        if g.random() < 0.15:
            pats.append(synth.random_bases(g, L))
            continue
        h = int(g.integers(0, len(S.lens)))
        if S.lens[h] <= L:
            continue
        st = int(off[h] + g.integers(0, S.lens[h] - L))
        p = S.seq[st:st + L].copy()
        p[p == 0] = 1
        for _ in range(int(g.poisson(0.6))):
            j = int(g.integers(0, L))
            r = g.random()
            if r < 0.6:
                p[j] = int(g.integers(1, 6))
            elif r < 0.8:
                p = np.delete(p, j)
                L -= 1
            else:
                p = np.insert(p, j, int(g.integers(1, 5)))
                L += 1
            if L <= 1:
                break
        pats.append(p.astype(np.uint8))
    q = np.concatenate(pats).astype(np.uint8)
    qoff = np.concatenate([[0], np.cumsum([len(p) for p in pats])]).astype(np.int64)
    return q, qoff


def index_case():
    S = synth.pangenome(seed=811, founder_len=2500, n_hap=6, batch=3)
    B = oracle.bwt(oracle.concat(S.seq, S.lens, True))
    return S, B


def check_all(B, got, n_got, q, qoff, a, b, go, ge, W, red):
    for i in range(len(qoff) - 1):
        P = q[qoff[i]:qoff[i + 1]]
        want = oracle.haplotype_diversity(B, P, a, b, go, ge, W=W, redundancy=red)
        assert n_got[i] == len(want), (i, n_got[i], len(want))
        assert np.array_equal(got[i, :n_got[i]], want), i


@pytest.mark.parametrize("layout", ["d32", "d64", "rle512"])
@pytest.mark.parametrize("scores", SCORES)
def test_diversity_vs_oracle(layout, scores):
    run_layout(layout, scores)


@pytest.mark.parametrize("layout", ["d128", "d256", "rle4096"])
def test_diversity_other_layouts(layout):
    """The remaining rank layouts under two score sets."""
    for scores in (SCORES[0], SCORES[2]):
        run_layout(layout, scores)


def run_layout(layout, scores):
    import torch
    import paper_2409_00613_gb300 as rb
    a, b, go, ge, W = scores
    S, B = index_case()
    D = int(layout[1:]) if layout.startswith("d") else 32
    dev = torch.device("cuda:0")
    off = S.offsets
    half = off[3]
    idx = rb.rb3_build_batch(torch.from_numpy(S.seq[:half].copy()).to(dev), S.lens[:3].copy(),
                             opts={"occ_interval": D})
    rb.rb3_merge(idx, rb.rb3_build_batch(torch.from_numpy(S.seq[half:].copy()).to(dev), S.lens[3:].copy(),
                                         opts={"occ_interval": D}))
    if layout.startswith("rle"):
        idx = rb.rb3_index_compress(idx, int(layout[3:]))
    q, qoff = diversity_queries(S, 812 + a + 7 * W, 120)
    for red in (True, False):
        got, n_got = rb.rb3_haplotype_diversity(idx, q, qoff, a, b, go, ge, W, red)
        check_all(B, got, n_got, q, qoff, a, b, go, ge, W, red)
    # device buffers in and out give the same records
    dq, doff = torch.from_numpy(q).to(dev), torch.from_numpy(qoff).to(dev)
    dout = torch.full((len(qoff) - 1, W, 4), -7, dtype=torch.int64, device=dev)
    dn = torch.empty(len(qoff) - 1, dtype=torch.int64, device=dev)
    rb.rb3_haplotype_diversity(idx, dq, doff, a, b, go, ge, W, True, out=dout, n_out=dn)
    got, n_got = rb.rb3_haplotype_diversity(idx, q, qoff, a, b, go, ge, W, True)
    assert np.array_equal(dn.cpu().numpy(), n_got)
    for i in range(len(n_got)):
        assert np.array_equal(dout[i, :n_got[i]].cpu().numpy(), got[i, :n_got[i]])


def test_diversity_paper_example_and_refusals():
    """The worked example of the section (T = CAAGCAG, query AGCA, a = 3):
    AAGCA scores 4a - q - e but is dropped by the filter; nq = 0; refusals."""
    import torch
    import paper_2409_00613_gb300 as rb
    dev = torch.device("cuda:0")
    code = {"A": 1, "C": 2, "G": 3, "T": 4}
    T = np.array([code[c] for c in "CAAGCAG"], np.uint8)
    idx = rb.rb3_build_batch(torch.from_numpy(T).to(dev), np.array([7], np.int64))
    B = oracle.bwt(oracle.concat(T, np.array([7]), True))
    P = np.array([code[c] for c in "AGCA"], np.uint8)
    qoff = np.array([0, 4], np.int64)
    for red in (False, True):
        got, n = rb.rb3_haplotype_diversity(idx, P, qoff, 3, 3, 5, 2, 32, red)
        want = oracle.haplotype_diversity(B, P, 3, 3, 5, 2, W=32, redundancy=red)
        assert np.array_equal(got[0, :n[0]], want)
        keys = {tuple(r[:3]) for r in want.tolist()}
        assert ((2, 14, 1) in keys) == (not red)
    out, n = rb.rb3_haplotype_diversity(idx, np.zeros(0, np.uint8), np.zeros(1, np.int64))
    assert out.shape[0] == 0 and n.shape[0] == 0
    bad = [dict(W=0), dict(W=33), dict(a=0), dict(gap_ext=0), dict(b=-1), dict(gap_open=70000)]
    for kw in bad:
        with pytest.raises(rb.RB3Error) as e:
            rb.rb3_haplotype_diversity(idx, P, qoff, **kw)
        assert e.value.code == rb.RB3_E_INVAL
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_haplotype_diversity(idx, np.array([1, 0, 2], np.uint8), np.array([0, 3], np.int64))
    assert e.value.code == rb.RB3_E_INVAL
    ss = rb.rb3_build_batch(torch.from_numpy(T).to(dev), np.array([7], np.int64), opts={"single_strand": 1})
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_haplotype_diversity(ss, P, qoff)
    assert e.value.code == rb.RB3_E_INVAL


def overflow_text():
    """65,536 strings: every 8-mer over ACGT followed by one random 20-mer X.
    After the whole of X (a = 5, q = 0, e = 1: H = 100), deleting text symbols
    to its left keeps every left extension of up to 99 symbols positive, and X
    is preceded by all 4^8 contexts: the closure reaches 4 + 16 + ... + 4^8 >
    65,534 distinct nodes at that step, beyond the largest table."""
    g = synth.rng(814)
    X = synth.random_bases(g, 20)
    ctx = (np.arange(65536)[:, None] >> (2 * np.arange(8)[::-1])[None, :]) & 3
    seq = np.concatenate([ctx.astype(np.uint8) + 1, np.tile(X, (65536, 1))], axis=1).reshape(-1)
    return seq.astype(np.uint8), np.full(65536, 28, np.int64), X


def test_diversity_table_overflow_is_reported():
    """The query X on overflow_text() outgrows every table (the small, the
    large and the 65,534-cell one in global memory): it reports -1 and
    RB3_E_CAPACITY; the query beside it keeps its result (all N: no cell
    scores above 0, since every extension mismatches and gaps only lower the
    root's 0)."""
    import torch
    import paper_2409_00613_gb300 as rb
    dev = torch.device("cuda:0")
    seq, lens, X = overflow_text()
    idx = rb.rb3_build_batch(torch.from_numpy(seq).to(dev), lens)
    q = np.concatenate([X, np.full(9, 5, np.uint8)])
    qoff = np.array([0, 20, 29], np.int64)
    out = np.zeros((2, 4, 4), np.int64)
    n = np.full(2, 7, np.int64)
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_haplotype_diversity(idx, q, qoff, 5, 3, 0, 1, 4, True, out=out, n_out=n)
    assert e.value.code == rb.RB3_E_CAPACITY
    assert n[0] == -1 and n[1] == 0


def test_diversity_large_tables_exact():
    """Queries whose steps outgrow the 256-cell and 2,048-cell tables (a long
    exact window with free gap opens) are answered exactly by the next table."""
    import torch
    import paper_2409_00613_gb300 as rb
    dev = torch.device("cuda:0")
    g = synth.rng(813)
    T = synth.random_bases(g, 8000)
    idx = rb.rb3_build_batch(torch.from_numpy(T).to(dev), np.array([8000], np.int64))
    B = oracle.bwt(oracle.concat(T, np.array([8000]), True))
    pats = [T[4000:4300].copy(), T[4000:5400].copy(), T[100:112].copy()]
    q = np.concatenate(pats)
    qoff = np.concatenate([[0], np.cumsum([len(p) for p in pats])]).astype(np.int64)
    out, n = rb.rb3_haplotype_diversity(idx, q, qoff, 2, 3, 0, 1, 4, True)
    for i, p in enumerate(pats):
        want = oracle.haplotype_diversity(B, p, 2, 3, 0, 1, W=4)
        assert n[i] == len(want) and np.array_equal(out[i, :n[i]], want), i