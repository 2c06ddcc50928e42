"""Pins for the CPU oracle: each check ties it to something other than itself
(brute force on tiny inputs written independently here, the paper's worked
example, closed-form relations of Table 1 / Algorithm 3, the LF-decode
certificate).  CPU only."""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CODE = {"$": 0, "A": 1, "C": 2, "G": 3, "T": 4, "N": 5}
LETTER = "$ACGTN"


def enc(s):
    return np.array([CODE[c] for c in s], dtype=np.uint8)


def dec(a):
    return "".join(LETTER[int(c)] for c in a)


def golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            rows[k] = v
    return rows


# ---- independent brute-force pieces (Python, tiny inputs) -------------------

def py_sa(T):
    """Sort suffixes as explicit tuples: a letter c is (1, c); the j-th sentinel
    of T is (0, j); a suffix's key runs up to and including its first sentinel."""
    T = [int(c) for c in T]
    elem, j = [], 0
    for c in T:
        if c == 0:
            elem.append((0, j))
            j += 1
        else:
            elem.append((1, c))
    keys = []
    for p in range(len(T)):
        k = []
        for t in range(p, len(T)):
            k.append(elem[t])
            if T[t] == 0:
                break
        keys.append(tuple(k))
    return sorted(range(len(T)), key=lambda p: keys[p])


def py_concat(strings, both=True):
    comp = {"A": "T", "C": "G", "G": "C", "T": "A", "N": "N"}
    out = ""
    for s in strings:
        out += s + "$"
        if both:
            out += "".join(comp[c] for c in reversed(s)) + "$"
    return out


def rand_list(g, n_str, max_len, n_frac=0.0, allow_empty=True):
    S = synth.random_strings(g, n_str, max_len, n_frac=n_frac, allow_empty=allow_empty)
    return S, ["".join(LETTER[c] for c in S.seq[o:o + l]) for o, l in zip(S.offsets[:-1], S.lens)]


# ---- concatenation ------------------------------------------------------------

def test_ds_concat_golden():
    gd = golden("ds_concat_worked_example.txt")
    s = gd["input"][0]
    T = oracle.concat(enc(s), np.array([len(s)]), both=True)
    assert dec(T) == gd["ds"][0]


def test_concat_matches_python():
    g = synth.rng(11)
    for both in (True, False):
        for _ in range(20):
            S, strs = rand_list(g, int(g.integers(1, 6)), 9, n_frac=0.1)
            assert dec(oracle.concat(S.seq, S.lens, both)) == py_concat(strs, both)


# ---- O1 suffix array / BWT --------------------------------------------------------

@pytest.mark.parametrize("both", [True, False])
def test_suffix_array_vs_python_sort(both):
    g = synth.rng(12 + both)
    for _ in range(60):
        S, strs = rand_list(g, int(g.integers(1, 5)), 10, n_frac=0.15)
        T = oracle.concat(S.seq, S.lens, both)
        assert list(oracle.suffix_array(T)) == py_sa(T)


def test_all_short_lists_exhaustive():
    """Every list of <= 2 strings of length <= 3 over {A,C,N} (plus empty)."""
    import itertools
    words = [""] + ["".join(w) for L in range(1, 4) for w in itertools.product("ACN", repeat=L)]
    cnt = 0
    for a in words:
        for b in [None] + words[::5]:
            strs = [a] if b is None else [a, b]
            seq = enc("".join(strs))
            T = oracle.concat(seq, np.array([len(s) for s in strs]), True)
            SA = py_sa(T)
            B = np.array([T[p - 1] if p > 0 else T[-1] for p in SA], dtype=np.uint8)
            assert np.array_equal(oracle.bwt(T), B)
            cnt += 1
    assert cnt > 300


def test_bwt_lf_closed_form():
    """Table 1: pi(k) = S^{-1}(S(k)-1) = pi_B(B[k],k) whenever B[k] != $; the $
    rows map onto rows 0..m-1 (Section "Locating with FM-index": LF does not
    follow the text at a sentinel)."""
    g = synth.rng(13)
    for _ in range(30):
        S, _ = rand_list(g, int(g.integers(1, 6)), 30, n_frac=0.05)
        T = oracle.concat(S.seq, S.lens, True)
        SA = oracle.suffix_array(T)
        B = oracle.bwt_from_sa(T, SA)
        n = len(T)
        inv = np.empty(n, dtype=np.int64)
        inv[SA] = np.arange(n)
        C = np.array([np.sum(B < a) for a in range(6)])
        seen = np.zeros(6, dtype=np.int64)
        dollar_targets = []
        for k in range(n):
            a = int(B[k])
            pik = C[a] + seen[a]
            seen[a] += 1
            if a != 0:
                assert pik == inv[(SA[k] - 1) % n]
            else:
                dollar_targets.append(pik)
        assert sorted(dollar_targets) == list(range(int(np.sum(T == 0))))


def test_counts_and_occ_table():
    g = synth.rng(14)
    S, _ = rand_list(g, 7, 200, n_frac=0.02)
    T = oracle.concat(S.seq, S.lens, True)
    B = oracle.bwt(T)
    C = oracle.counts(B)
    for a in range(6):
        assert C[a + 1] - C[a] == np.sum(T == a)
    for D in (1, 7, 64, 128):
        occ = oracle.occ_table(B, D)
        ref = np.zeros((len(B) // D + 1, 6), dtype=np.int64)
        cum = np.zeros((len(B) + 1, 6), dtype=np.int64)
        for a in range(6):
            cum[1:, a] = np.cumsum(B == a)
        ref[:] = cum[np.arange(len(B) // D + 1) * D]
        assert np.array_equal(occ, ref)


# ---- O2 certificate / Retrieve ------------------------------------------------------

def test_retrieve_decodes_every_string():
    g = synth.rng(15)
    S, strs = rand_list(g, 6, 40, n_frac=0.05)
    T = oracle.concat(S.seq, S.lens, True)
    B = oracle.bwt(T)
    ds = py_concat(strs, True).split("$")[:-1]
    for i, s in enumerate(ds):
        assert dec(oracle.retrieve(B, i)) == s


def test_certificate_accepts_true_bwt_and_rejects_plants():
    g = synth.rng(16)
    for trial in range(40):
        S, _ = rand_list(g, int(g.integers(1, 6)), 25, n_frac=0.05)
        T = oracle.concat(S.seq, S.lens, True)
        B = oracle.bwt(T)
        assert oracle.certify(B, T) == 0
        # plant: swap two different symbols
        diff = np.flatnonzero(B != B[0])
        if len(diff):
            Bb = B.copy()
            j = int(diff[g.integers(0, len(diff))])
            Bb[0], Bb[j] = Bb[j], Bb[0]
            assert oracle.certify(Bb, T) != 0
        # plant: BWT of the list in another order
        if len(S.lens) > 1 and len(set(map(tuple, np.split(S.seq, S.offsets[1:-1])))) > 1:
            perm = np.arange(len(S.lens))[::-1]
            off = S.offsets
            seq2 = np.concatenate([S.seq[off[i]:off[i + 1]] for i in perm])
            T2 = oracle.concat(seq2, S.lens[perm], True)
            B2 = oracle.bwt(T2)
            if not np.array_equal(B2, B):
                assert oracle.certify(B2, T) != 0
        # plant: a symbol changed (counts break)
        Bc = B.copy()
        Bc[len(B) // 2] = (Bc[len(B) // 2] % 5) + 1 if Bc[len(B) // 2] != 0 else 1
        assert oracle.certify(Bc, T) != 0


# ---- O3 Algorithm 1 ---------------------------------------------------------------

@pytest.mark.parametrize("both", [True, False])
def test_merge_equals_build_of_concatenation(both):
    g = synth.rng(17 + both)
    for trial in range(80):
        S, _ = rand_list(g, int(g.integers(1, 7)), 30, n_frac=0.05)
        cut = int(g.integers(0, len(S.lens) + 1))
        A, Bl = S.subset(0, cut), S.subset(cut, len(S.lens))
        TA = oracle.concat(A.seq, A.lens, both)
        TB = oracle.concat(Bl.seq, Bl.lens, both)
        Tall = oracle.concat(S.seq, S.lens, both)
        M, pos = oracle.merge(oracle.bwt(TA), oracle.bwt(TB), want_pos=True)
        assert np.array_equal(M, oracle.bwt(Tall))
        assert np.all(np.diff(pos) > 0)


def test_merge_into_empty_and_of_empty():
    g = synth.rng(19)
    S, _ = rand_list(g, 4, 30)
    T = oracle.concat(S.seq, S.lens, True)
    B = oracle.bwt(T)
    assert np.array_equal(oracle.merge(np.zeros(0, np.uint8), B), B)
    assert np.array_equal(oracle.merge(B, np.zeros(0, np.uint8)), B)


def test_build_incremental_groups():
    g = synth.rng(20)
    S, _ = rand_list(g, 9, 60, n_frac=0.02)
    ref = oracle.bwt(oracle.concat(S.seq, S.lens, True))
    for grp in (1, 2, 4, 9):
        assert np.array_equal(oracle.build_incremental(S.seq, S.lens, True, grp, nthreads=2), ref)


def test_pangenome_incremental_certified():
    """A small pangenome (near-identical haplotypes): incremental build passes the
    certificate and equals the one-shot O1 build."""
    S = synth.pangenome(seed=99, founder_len=3000, n_hap=6, batch=2)
    T = oracle.concat(S.seq, S.lens, True)
    B = oracle.build_incremental(S.seq, S.lens, True, 2, nthreads=2)
    assert oracle.certify(B, T) == 0
    assert np.array_equal(B, oracle.bwt(T))


# ---- backward search / Algorithm 3 ------------------------------------------------

def test_backward_search_vs_brute():
    g = synth.rng(21)
    for both in (True, False):
        S, _ = rand_list(g, 5, 60, n_frac=0.05)
        T = oracle.concat(S.seq, S.lens, both)
        B = oracle.bwt(T)
        pats = []
        for _ in range(80):
            L = int(g.integers(1, 7))
            if g.random() < 0.6 and len(S.seq) > L:
                s = int(g.integers(0, len(S.seq) - L))
                pats.append(S.seq[s:s + L].copy())
            else:
                pats.append(synth.random_bases(g, L))
        q = np.concatenate(pats)
        qoff = np.concatenate([[0], np.cumsum([len(p) for p in pats])])
        lohi = oracle.backward_search(B, q, qoff)
        for (lo, hi), p in zip(lohi, pats):
            assert lo == oracle.lo_brute(T, p)
            assert hi - lo == oracle.occ_brute(T, p)


def test_occ_strand_symmetry():
    """Section "Double-strand BWT": occ(P) = occ(rc(P)) in a DS text."""
    g = synth.rng(22)
    S, _ = rand_list(g, 4, 80)
    T = oracle.concat(S.seq, S.lens, True)
    comp = np.array([0, 4, 3, 2, 1, 5], dtype=np.uint8)
    for _ in range(100):
        L = int(g.integers(1, 6))
        p = synth.random_bases(g, L)
        assert oracle.occ_brute(T, p) == oracle.occ_brute(T, comp[p[::-1]])


def test_extension_bi_intervals():
    """Algorithm 3 against the bi-interval definition (lo(P), lo(rc P), occ(P))."""
    g = synth.rng(23)
    comp = np.array([0, 4, 3, 2, 1, 5], dtype=np.uint8)
    S, _ = rand_list(g, 4, 50, n_frac=0.05)
    T = oracle.concat(S.seq, S.lens, True)
    B = oracle.bwt(T)

    def bi(p):
        return (oracle.lo_brute(T, p), oracle.lo_brute(T, comp[p[::-1]]), oracle.occ_brute(T, p))

    for _ in range(150):
        L = int(g.integers(0, 5))
        if L and g.random() < 0.7:
            s = int(g.integers(0, len(S.seq) - L))
            p = S.seq[s:s + L].copy()
        else:
            p = synth.random_bases(g, L)
        x = bi(p) if L else (0, 0, len(T))
        a = int(g.integers(1, 6))
        assert oracle.ext(B, x, a, forward=False) == bi(np.concatenate([[a], p]).astype(np.uint8))
        assert oracle.ext(B, x, a, forward=True) == bi(np.concatenate([p, [a]]).astype(np.uint8))


# ---- O4 Algorithm 4 vs O5 definition ----------------------------------------------

def test_smem_paper_worked_example():
    gd = golden("smem_worked_example.txt")
    text, query = gd["text"][0], gd["query"][0]
    T = oracle.concat(enc(text), np.array([len(text)]), True)
    B = oracle.bwt(T)
    q = enc(query)
    qoff = np.array([0, len(q)])
    got = oracle.smem(B, q, qoff, 1, 1)
    want = np.array([[int(v) for v in gd["smem"]]])
    assert np.array_equal(got, want)
    assert np.array_equal(oracle.smem_brute(T, q, qoff, 1, 1), want)
    # the contained MEM (5,1,2): text offset 5, pattern offset 1, length 2 matches
    t_off, p_off, L = (int(v) for v in gd["contained_mem"])
    assert text[t_off:t_off + L] == query[p_off:p_off + L]
    assert not any(r[1] == p_off for r in got)


@pytest.mark.parametrize("ell,smin", [(1, 1), (2, 1), (3, 2), (4, 1), (2, 3), (6, 1)])
def test_smem_alg4_equals_definition(ell, smin):
    g = synth.rng(100 + 10 * ell + smin)
    comp = np.array([0, 4, 3, 2, 1, 5], dtype=np.uint8)
    for trial in range(12):
        S, _ = rand_list(g, int(g.integers(1, 5)), 40, n_frac=0.03, allow_empty=True)
        T = oracle.concat(S.seq, S.lens, True)
        B = oracle.bwt(T)
        qs = []
        for _ in range(8):
            L = int(g.integers(0, 25))
            if g.random() < 0.7 and len(S.seq) > L + 1:
                s = int(g.integers(0, len(S.seq) - L))
                p = S.seq[s:s + L].copy()
                m = g.random(L) < 0.08
                p[m] = synth.random_bases(g, int(m.sum()))
                if g.random() < 0.5:
                    p = comp[p[::-1]]
            else:
                p = synth.random_bases(g, L)
            qs.append(p.astype(np.uint8))
        q = np.concatenate(qs) if qs else np.zeros(0, np.uint8)
        qoff = np.concatenate([[0], np.cumsum([len(p) for p in qs])]).astype(np.int64)
        a = oracle.smem(B, q, qoff, ell, smin)
        b = oracle.smem_brute(T, q, qoff, ell, smin)
        assert np.array_equal(a, b), (ell, smin, trial)
        a_mt = oracle.smem(B, q, qoff, ell, smin, nthreads=3)
        assert np.array_equal(a, a_mt)


# ---- locate -------------------------------------------------------------------

@pytest.mark.parametrize("both", [True, False])
def test_locate_pins(both):
    """Section "Locating with FM-index": the oracle's (string, offset) of every
    row against the input strings written out here: the suffix of row i, read
    from the brute-force suffix array, is the named string from the named
    offset followed by its sentinel; every (string, offset) occurs once; and
    LF moves a row to the row of the same string one offset earlier."""
    g = synth.rng(4711 + both)
    S, strs = rand_list(g, 9, 40, n_frac=0.05)
    comp = {"A": "T", "C": "G", "G": "C", "T": "A", "N": "N"}
    ds = []
    for s_ in strs:
        ds.append(s_)
        if both:
            ds.append("".join(comp[c] for c in reversed(s_)))
    T = oracle.concat(S.seq, S.lens, both)
    SA = np.array(py_sa(T), dtype=np.int64)
    loc = oracle.locate(T, SA, np.arange(len(T)))
    text = dec(T)
    seen = set()
    for i, (t, off) in enumerate(loc):
        want = ds[t][off:] + "$"
        assert text[SA[i]:SA[i] + len(want)] == want
        seen.add((int(t), int(off)))
    assert seen == {(t, o) for t in range(len(ds)) for o in range(len(ds[t]) + 1)}
    B = oracle.bwt_from_sa(T, SA.astype(np.int64))
    C = oracle.counts(B)  # C_B(a) for a = $..N, then n
    row_of = {(int(t), int(o)): i for i, (t, o) in enumerate(loc)}
    for i, (t, off) in enumerate(loc):
        if off == 0:
            continue
        a = int(B[i])
        lf = C[a] + int(np.count_nonzero(B[:i] == a))
        assert lf == row_of[(int(t), int(off) - 1)]


def py_runs(B, span):
    """Runs by a plain scan: a run ends where the symbol changes or a span ends."""
    out = []
    for i, a in enumerate(B):
        if out and out[-1][0] == a and not (span and i % span == 0):
            out[-1][1] += 1
        else:
            out.append([a, 1])
    return out


def test_runs_pins():
    """The run-length form: a hand-worked case, then a plain scan, the
    expansion back to B, maximality inside a span, and each span's lengths
    summing to its size, on random BWTs with long runs (near-identical
    strings) and short ones."""
    sym, ln = oracle.runs(np.array([1, 1, 2, 2, 2, 0, 1], np.uint8))
    assert sym.tolist() == [1, 2, 0, 1] and ln.tolist() == [2, 3, 1, 1]
    sym, ln = oracle.runs(np.array([1, 1, 2, 2, 2, 0, 1], np.uint8), 4)
    assert sym.tolist() == [1, 2, 2, 0, 1] and ln.tolist() == [2, 2, 1, 1, 1]
    assert [len(x) for x in oracle.runs(np.zeros(0, np.uint8), 8)] == [0, 0]
    g = synth.rng(2718)
    for trial in range(12):
        if trial % 2:
            S = synth.pangenome(seed=100 + trial, founder_len=int(g.integers(50, 400)), n_hap=4, batch=4)
            B = oracle.bwt(oracle.concat(S.seq, S.lens, True))
        else:
            S, _ = rand_list(g, int(g.integers(1, 12)), int(g.integers(1, 60)), n_frac=0.1)
            B = oracle.bwt(oracle.concat(S.seq, S.lens, bool(trial & 2)))
        for span in (0, 1, 2, 8, 64):
            sym, ln = oracle.runs(B, span)
            assert [[int(a), int(b)] for a, b in zip(sym, ln)] == py_runs(B.tolist(), span)
            assert np.array_equal(np.repeat(sym, ln), B)
            ends = np.cumsum(ln)
            starts = ends - ln
            same = sym[1:] == sym[:-1]
            if span:
                assert np.all((starts[1:][same] % span) == 0)  # equal neighbours only across a cut
                assert np.all(starts // span == (ends - 1) // span)  # no run crosses a cut
            else:
                assert not np.any(same)


# ---- Section "Estimating local haplotype diversity" (Algorithm 5) ---------------

def py_diversity(strings, P, a, b, q, e):
    """String by string: for every distinct substring x over ACGT of the
    double-strand text, the semi-global affine-gap score of P against x,
    filled from the ends of both (P[i..] against x[j..]) with a cell kept only
    while its score is positive (the empty pair starts at 0).  A positive
    alignment holds fewer than m*a/e deletions, which bounds |x|."""
    comp = {"A": "T", "C": "G", "G": "C", "T": "A", "N": "N"}
    m, NEG = len(P), -(1 << 40)
    max_len = m + (m * a) // e + 1
    subs = set()
    for s in strings:
        for t in (s, "".join(comp[c] for c in reversed(s))):
            for i in range(len(t)):
                for j in range(i + 1, min(len(t), i + max_len) + 1):
                    if "N" in t[i:j]:
                        break
                    subs.add(t[i:j])
    best = {}
    for x in subs:
        L = len(x)
        H = [[NEG] * (L + 2) for _ in range(m + 2)]
        E = [[NEG] * (L + 2) for _ in range(m + 2)]
        F = [[NEG] * (L + 2) for _ in range(m + 2)]
        live = [[False] * (L + 2) for _ in range(m + 2)]
        H[m][L], live[m][L] = 0, True
        for i in range(m, -1, -1):
            for j in range(L, -1, -1):
                if i == m and j == L:
                    continue
                g = ev = fv = NEG
                if i < m and j < L and live[i + 1][j + 1]:
                    g = H[i + 1][j + 1] + (a if P[i] == x[j] else -b)
                if i < m and live[i + 1][j]:
                    ev = max(H[i + 1][j] - q, E[i + 1][j]) - e
                if j < L and live[i][j + 1] and H[i][j + 1] > 0:
                    fv = max(H[i][j + 1] - q, F[i][j + 1]) - e
                H[i][j], E[i][j], F[i][j] = max(g, ev, fv), ev, fv
                live[i][j] = H[i][j] > 0
        if m and H[0][0] > 0:
            best[x] = max(best.get(x, NEG), H[0][0])
    return best


def diversity_from_strings(T, best):
    comp = {"A": "T", "C": "G", "G": "C", "T": "A"}
    cells = {}
    for x, h in best.items():
        key = (oracle.lo_brute(T, enc(x)), oracle.lo_brute(T, enc("".join(comp[c] for c in reversed(x)))),
               oracle.occ_brute(T, enc(x)))
        cells[key] = max(cells.get(key, -(1 << 40)), h)
    return cells


def test_diversity_paper_worked_example():
    gd = golden("diversity_worked_example.txt")
    text, query = gd["text"][0], gd["query"][0]
    a, b, q, e = (int(v) for v in gd["scores"])
    T = oracle.concat(enc(text), np.array([len(text)]), True)
    B = oracle.bwt(T)
    comp = {"A": "T", "C": "G", "G": "C", "T": "A"}

    def bi(x):
        rc = "".join(comp[c] for c in reversed(x))
        return (oracle.lo_brute(T, enc(x)), oracle.lo_brute(T, enc(rc)), oracle.occ_brute(T, enc(x)))

    (xs, hs), (xg, hg) = gd["exact"], gd["gapped"]
    full = {tuple(r[:3]): r[3] for r in oracle.haplotype_diversity(B, enc(query), a, b, q, e, W=0,
                                                                   redundancy=False).tolist()}
    assert full[bi(xs)] == int(hs) and full[bi(xg)] == int(hg)
    assert max(full.values()) == int(hs)
    kept = oracle.haplotype_diversity(B, enc(query), a, b, q, e, W=0)
    keys = [tuple(r[:3]) for r in kept.tolist()]
    assert keys[0] == bi(xs) and bi(xg) not in keys


@pytest.mark.parametrize("scores", [(1, 3, 5, 2), (2, 1, 2, 1), (3, 3, 5, 2), (3, 2, 1, 1), (2, 4, 0, 1)])
def test_diversity_unbanded_equals_string_brute_force(scores):
    """No band, no filter: the cells after the whole query equal, bi-interval
    by bi-interval, the best pruned score over the strings of that interval."""
    a, b, q, e = scores
    g = synth.rng(700 + a + 10 * b + 100 * q)
    n_cells = 0
    for trial in range(8):
        S, strs = rand_list(g, int(g.integers(1, 4)), 24, n_frac=0.03, allow_empty=True)
        T = oracle.concat(S.seq, S.lens, True)
        B = oracle.bwt(T)
        for _ in range(4):
            m = int(g.integers(1, 9))
            if g.random() < 0.6 and len(S.seq) > m:
                st = int(g.integers(0, len(S.seq) - m))
                P = S.seq[st:st + m].copy()
                P[P == 0] = 1
                if g.random() < 0.5:
                    P[int(g.integers(0, m))] = int(g.integers(1, 6))
            else:
                P = synth.random_bases(g, m)
            want = diversity_from_strings(T, py_diversity(strs, dec(P), a, b, q, e))
            got = oracle.haplotype_diversity(B, P, a, b, q, e, W=0, redundancy=False)
            assert {tuple(r[:3]): r[3] for r in got.tolist()} == want
            hs = got[:, 3].tolist()
            assert hs == sorted(hs, reverse=True)
            n_cells += len(got)
    assert n_cells >= 10


def test_diversity_band_and_redundancy_invariants():
    """With a band of W cells: at most W results, each a cell of the unbanded
    run scoring no more there; a wide band changes nothing.  The filter keeps
    the best cell and drops exactly the cells whose k- or k'-interval lies in
    that of a cell kept before them."""
    g = synth.rng(771)
    S = synth.pangenome(seed=772, founder_len=300, n_hap=5, batch=5)
    T = oracle.concat(S.seq, S.lens, True)
    B = oracle.bwt(T)
    for _ in range(8):
        m = int(g.integers(8, 30))
        st = int(g.integers(0, len(S.seq) - m))
        P = S.seq[st:st + m].copy()
        P[P == 0] = 1
        P[int(g.integers(0, m))] = int(g.integers(1, 5))
        full = oracle.haplotype_diversity(B, P, W=0, redundancy=False)
        fmap = {tuple(r[:3]): r[3] for r in full.tolist()}
        for W in (1, 3, 25):
            band = oracle.haplotype_diversity(B, P, W=W, redundancy=False)
            assert len(band) <= W
            for r in band.tolist():
                assert tuple(r[:3]) in fmap and r[3] <= fmap[tuple(r[:3])]
        assert np.array_equal(oracle.haplotype_diversity(B, P, W=100000, redundancy=False), full)
        check_filter(full.tolist(), oracle.haplotype_diversity(B, P, W=0).tolist())
    # cheap gaps on random texts: many overlapping cells, among them chains
    # where a cell lies inside a dropped one but in no kept one
    for trial in range(30):
        S = synth.random_strings(g, int(g.integers(1, 4)), 30, allow_empty=False)
        T = oracle.concat(S.seq, S.lens, True)
        B = oracle.bwt(T)
        P = synth.random_bases(g, int(g.integers(3, 10)))
        full = oracle.haplotype_diversity(B, P, 3, 2, 1, 1, W=0, redundancy=False).tolist()
        check_filter(full, oracle.haplotype_diversity(B, P, 3, 2, 1, 1, W=0).tolist())


def check_filter(full, kept):
    """Walking the unfiltered list best first: a cell is kept iff neither of
    its intervals lies inside the same interval of a cell kept before it."""
    inside = lambda x, y: (x[0] >= y[0] and x[0] + x[2] <= y[0] + y[2]) or \
        (x[1] >= y[1] and x[1] + x[2] <= y[1] + y[2])
    kept_set = {tuple(r) for r in kept}
    seen = []
    for r in full:
        if tuple(r) in kept_set:
            assert not any(inside(r, y) for y in seen)
            seen.append(r)
        else:
            assert any(inside(r, y) for y in seen)
    assert seen == kept


def test_diversity_degenerate_queries():
    """Empty query: no alignment.  A query of N only: every symbol mismatches,
    so nothing stays positive.  An exact occurrence scores a*m and comes first."""
    S = synth.pangenome(seed=773, founder_len=200, n_hap=3, batch=3)
    T = oracle.concat(S.seq, S.lens, True)
    B = oracle.bwt(T)
    assert len(oracle.haplotype_diversity(B, np.zeros(0, np.uint8))) == 0
    assert len(oracle.haplotype_diversity(B, np.full(6, 5, np.uint8), W=0)) == 0
    P = S.seq[10:40].copy()
    top = oracle.haplotype_diversity(B, P, a=2)[0]
    assert top[3] == 2 * len(P)
    assert (top[0], top[2]) == (oracle.lo_brute(T, P), oracle.occ_brute(T, P))


# ---- Section "Finding inexact matches with BWA-SW" (Algorithm 5, DAWG to DAWG) ----

def py_bwasw(T, strings, P, a, b, q, e):
    """Pair by pair: for every distinct substring x of P and y of the
    double-strand text T (of the list `strings`), the pruned end-to-end score
    of x against y (py_diversity with x as the query), keyed by x's SA
    interval in the text P$ and y's bi-interval, the best pair of each key
    kept."""
    TP = oracle.concat(enc(P), np.array([len(P)]), False)
    xs = {P[i:j] for i in range(len(P)) for j in range(i + 1, len(P) + 1)}
    cells = {}
    for x in xs:
        ukey = (oracle.lo_brute(TP, enc(x)), oracle.occ_brute(TP, enc(x)))
        for key, h in diversity_from_strings(T, py_diversity(strings, x, a, b, q, e)).items():
            k = ukey + key
            cells[k] = max(cells.get(k, -(1 << 40)), h)
    return cells


@pytest.mark.parametrize("scores", [(1, 3, 5, 2), (2, 1, 2, 1), (3, 2, 1, 1)])
def test_bwasw_unbanded_equals_pair_brute_force(scores):
    """No band: every (query node, text node) cell with H > 0 equals the best
    pruned score over the string pairs of that pair of intervals."""
    a, b, q, e = scores
    g = synth.rng(880 + a + 10 * b)
    n_cells = 0
    for trial in range(6):
        S, strs = rand_list(g, int(g.integers(1, 3)), 16, n_frac=0.03, allow_empty=False)
        T = oracle.concat(S.seq, S.lens, True)
        B = oracle.bwt(T)
        m = int(g.integers(1, 7))
        if g.random() < 0.6 and len(S.seq) > m:
            st = int(g.integers(0, len(S.seq) - m))
            P = S.seq[st:st + m].copy()
            P[P == 0] = 1
            if g.random() < 0.5:
                P[int(g.integers(0, m))] = int(g.integers(1, 6))
        else:
            P = synth.random_bases(g, m)
        got = oracle.bwasw(B, P, a, b, q, e, W=0)
        want = py_bwasw(T, strs, dec(P), a, b, q, e)
        assert {tuple(r[:5]): r[5] for r in got.tolist()} == want
        n_cells += len(got)
    assert n_cells >= 10


def test_bwasw_band_and_worked_example():
    """Band: at most W cells per query node, none above its unbanded score.
    The section's example text CAAGCAG with query AGCA: the query node of
    AGCA (which also holds AG and AGC, occurring once in P) reaches AGCA in the
    text with 4a, and the node of A reaches the text's A with a."""
    g = synth.rng(885)
    S = synth.pangenome(seed=886, founder_len=200, n_hap=4, batch=4)
    T = oracle.concat(S.seq, S.lens, True)
    B = oracle.bwt(T)
    for _ in range(4):
        P = S.seq[int(g.integers(0, 300)):][:12].copy()
        P[P == 0] = 1
        full = {tuple(r[:5]): r[5] for r in oracle.bwasw(B, P, W=0).tolist()}
        for W in (1, 4):
            band = oracle.bwasw(B, P, W=W)
            per_node = {}
            for r in band.tolist():
                per_node[(r[0], r[1])] = per_node.get((r[0], r[1]), 0) + 1
                assert tuple(r[:5]) in full and r[5] <= full[tuple(r[:5])]
            assert max(per_node.values()) <= W
    text = "CAAGCAG"
    T = oracle.concat(enc(text), np.array([7]), True)
    B = oracle.bwt(T)
    TP = oracle.concat(enc("AGCA"), np.array([4]), False)
    got = {tuple(r[:5]): r[5] for r in oracle.bwasw(B, enc("AGCA"), 3, 3, 5, 2, W=0).tolist()}
    comp = {"A": "T", "C": "G", "G": "C", "T": "A"}

    def key(x, y):
        rc = "".join(comp[c] for c in reversed(y))
        return (oracle.lo_brute(TP, enc(x)), oracle.occ_brute(TP, enc(x)), oracle.lo_brute(T, enc(y)),
                oracle.lo_brute(T, enc(rc)), oracle.occ_brute(T, enc(y)))

    assert got[key("AGCA", "AGCA")] == 12
    assert got[key("A", "A")] == 3
    assert key("AG", "AGCA")[:2] == key("AGCA", "AGCA")[:2]
    # an N in the query is a node of its own DAWG that mismatches every text symbol
    # (ANCA against AGCA stays positive from the end: 3, 6, 3, 6)
    got = {tuple(r[:5]): r[5] for r in oracle.bwasw(B, enc("ANCA"), 3, 3, 5, 2, W=0).tolist()}
    assert got == py_bwasw(T, [text], "ANCA", 3, 3, 5, 2)
    TP = oracle.concat(enc("ANCA"), np.array([4]), False)
    assert got[key("ANCA", "AGCA")] == 3 * 3 - 3


def test_bwasw_node_of_whole_query_equals_linear_runs():
    """The query node holding all of P also holds every prefix of P that
    occurs once in P (same SA interval in P$); its cells are, text node by
    text node, the best of the linear-query runs of those strings."""
    g = synth.rng(890)
    for trial in range(10):
        S, _ = rand_list(g, int(g.integers(1, 3)), 30, allow_empty=False)
        T = oracle.concat(S.seq, S.lens, True)
        B = oracle.bwt(T)
        P = synth.random_bases(g, int(g.integers(3, 9)))
        TP = oracle.concat(P, np.array([len(P)]), False)
        node = (oracle.lo_brute(TP, P), 1)
        members = [P[:j] for j in range(1, len(P) + 1) if oracle.occ_brute(TP, P[:j]) == 1]
        assert all(oracle.lo_brute(TP, x) == node[0] for x in members)
        want = {}
        for x in members:
            for r in oracle.haplotype_diversity(B, x, 3, 2, 1, 1, W=0, redundancy=False).tolist():
                want[tuple(r[:3])] = max(want.get(tuple(r[:3]), -1), r[3])
        got = {tuple(r[2:5]): r[5] for r in oracle.bwasw(B, P, 3, 2, 1, 1, W=0).tolist() if (r[0], r[1]) == node}
        assert got == want


def test_diversity_many_equals_one_by_one():
    """The batched entry (one rank table) gives each query's records as the
    one-query call does."""
    g = synth.rng(895)
    S = synth.pangenome(seed=896, founder_len=400, n_hap=4, batch=4)
    B = oracle.bwt(oracle.concat(S.seq, S.lens, True))
    pats = [np.zeros(0, np.uint8)] + [S.seq[s:s + 25].copy() for s in g.integers(0, len(S.seq) - 25, 30)]
    for p in pats:
        p[p == 0] = 1
    q = np.concatenate(pats)
    qoff = np.concatenate([[0], np.cumsum([len(p) for p in pats])]).astype(np.int64)
    for W in (1, 5, 25):
        out, n = oracle.haplotype_diversity_many(B, q, qoff, W=W)
        for i, p in enumerate(pats):
            want = oracle.haplotype_diversity(B, p, W=W)
            assert n[i] == len(want) and np.array_equal(out[i, :n[i]], want)
