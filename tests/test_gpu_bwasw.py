"""GPU parity of BWA-SW between the query's prefix DAWG and the text's
(Algorithm 5 with the query as a DAWG): every record (query node, text node,
H) against the oracle's DAWG-to-DAWG Algorithm 5 on its own BWT, bit-exact,
under several score sets, bands and index layouts; refusals and capacity."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2409_00613_gb300 as rb

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def text():
    S = synth.pangenome(seed=71, founder_len=3000, n_hap=6, batch=3)
    off = S.offsets
    idx = rb.rb3_build_batch(torch.from_numpy(S.seq[:off[3]].copy()).to(DEV), S.lens[:3].copy())
    rb.rb3_merge(idx, rb.rb3_build_batch(torch.from_numpy(S.seq[off[3]:].copy()).to(DEV), S.lens[3:].copy()))
    B = oracle.bwt(oracle.concat(S.seq, S.lens, True))
    assert np.array_equal(rb.rb3_export(idx), B)
    return S, idx, B


def _queries(S, n=40, seed=0):
    g = synth.rng(9000 + seed)
    qs = []
    for i in range(n):
        L = int(g.integers(1, 160))
        st = int(g.integers(0, len(S.seq) - L))
        p = S.seq[st:st + L].copy()
        if i % 5 == 1:  # substitutions
            m = g.random(L) < 0.05
            p[m] = (p[m] % 4) + 1
        elif i % 5 == 2:  # an insertion and a deletion
            p = np.concatenate([p[:L // 3], synth.random_bases(g, 2), p[L // 3 + 1:]]).astype(np.uint8)
        elif i % 5 == 3:  # N
            p[g.random(len(p)) < 0.05] = 5
        elif i % 5 == 4:  # random
            p = synth.random_bases(g, L)
        qs.append(p)
    qs += [np.zeros(0, np.uint8), np.array([3], np.uint8), np.tile(np.array([1, 2], np.uint8), 40),
           np.full(30, 5, np.uint8), np.full(50, 1, np.uint8)]
    st = int(g.integers(0, len(S.seq) - 600))
    qs.append(S.seq[st:st + 600].copy())
    return qs


def _pack(qs):
    off = np.zeros(len(qs) + 1, np.int64)
    off[1:] = np.cumsum([len(p) for p in qs])
    return (np.concatenate(qs).astype(np.uint8) if qs else np.zeros(0, np.uint8)), off


def _check(recs, qs, B, a, b, q, e, W):
    for i, p in enumerate(qs):
        got = recs[recs[:, 0] == i][:, 1:]
        want = oracle.bwasw(B, p, a, b, q, e, W)
        assert got.shape == want.shape and np.array_equal(got, want), (i, len(p), got.shape, want.shape)


@pytest.mark.parametrize("scores", [(1, 3, 5, 2, 25), (2, 2, 3, 1, 8), (1, 1, 0, 1, 32), (1, 3, 5, 2, 1)])
def test_bwasw_vs_oracle(text, scores):
    S, idx, B = text
    qs = _queries(S, seed=scores[4])
    q, qoff = _pack(qs)
    recs = rb.rb3_bwasw(idx, q, qoff, *scores)
    assert len(recs) > 1000
    _check(recs, qs, B, *scores)
    # device buffers give the same records
    dq, doff = torch.from_numpy(q).to(DEV), torch.from_numpy(qoff).to(DEV)
    out = torch.empty((len(recs) + 5, 7), dtype=torch.int64, device=DEV)
    n = rb.rb3_bwasw(idx, dq, doff, *scores, cap=len(recs) + 5, out=out)
    assert n == len(recs) and np.array_equal(out[:n].cpu().numpy(), recs)


@pytest.mark.parametrize("layout", ["d64", "d256", "rle512"])
def test_bwasw_other_layouts(text, layout):
    S, _, B = text
    off = S.offsets
    D = 64 if layout == "d64" else (256 if layout == "d256" else 32)
    idx = rb.rb3_build_batch(torch.from_numpy(S.seq.copy()).to(DEV), S.lens.copy(), opts={"occ_interval": D})
    if layout.startswith("rle"):
        idx = rb.rb3_index_compress(idx, 512)
    qs = _queries(S, n=15, seed=3)
    q, qoff = _pack(qs)
    _check(rb.rb3_bwasw(idx, q, qoff, 1, 3, 5, 2, 25), qs, B, 1, 3, 5, 2, 25)


def test_bwasw_longest_query_and_refusals(text):
    S, idx, B = text
    g = synth.rng(9100)
    off = S.offsets
    h = int(g.integers(0, len(S.lens)))
    st = int(off[h] + g.integers(0, S.lens[h] - 2047 + 1))
    p = S.seq[st:st + 2047].copy()  # inside one haplotype
    recs = rb.rb3_bwasw(idx, p, np.array([0, 2047], np.int64), 1, 3, 5, 2, 25)
    # the whole query occurs: the node of P itself holds its exact match, H = 2047 a
    assert recs[:, 6].max() == 2047 and (recs[:, 6] > 0).all()
    keys = recs[:, 1] * 4096 + recs[:, 2]
    assert (np.diff(keys) >= 0).all()  # sorted by query node
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_bwasw(idx, np.ones(2048, np.uint8), np.array([0, 2048], np.int64))
    assert e.value.code == rb.RB3_E_INVAL
    for bad in (dict(W=0), dict(W=33), dict(a=0), dict(gap_ext=0)):
        with pytest.raises(rb.RB3Error):
            rb.rb3_bwasw(idx, p[:10], np.array([0, 10], np.int64), **bad)
    with pytest.raises(rb.RB3Error):
        rb.rb3_bwasw(idx, np.array([1, 0, 2], np.uint8), np.array([0, 3], np.int64))
    ss = rb.rb3_build_batch(S.seq[:100].copy(), np.array([100], np.int64), opts={"single_strand": 1})
    with pytest.raises(rb.RB3Error):
        rb.rb3_bwasw(ss, p[:10], np.array([0, 10], np.int64))
    # capacity: the number needed, then the same records with room for them
    qs = _queries(S, n=5, seed=4)
    q, qoff = _pack(qs)
    full = rb.rb3_bwasw(idx, q, qoff)
    out = np.empty((3, 7), np.int64)
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_bwasw(idx, q, qoff, cap=3, out=out)
    assert e.value.code == rb.RB3_E_CAPACITY


def test_bwasw_node_overflow_is_reported():
    """The query X of the diversity overflow text outgrows every cell table at
    the node of the whole of X: RB3_E_CAPACITY."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "dv", os.path.join(os.path.dirname(os.path.abspath(__file__)), "test_gpu_diversity.py"))
    dvmod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(dvmod)
    seq, lens, X = dvmod.overflow_text()
    idx = rb.rb3_build_batch(torch.from_numpy(seq).to(DEV), lens)
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_bwasw(idx, X, np.array([0, 20], np.int64), 5, 3, 0, 1, 4)
    assert e.value.code == rb.RB3_E_CAPACITY
