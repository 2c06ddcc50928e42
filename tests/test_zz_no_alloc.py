"""The allocation-free SMEM entry point (for callers that cannot allocate device
memory while they search) gives the same records, in the same order, as
rb3_mem_search; two calls in a row share and reuse its fixed scratch.  This
file is collected last on purpose."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2409_00613_gb300 as rb

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
FIELDS = ("qid", "start", "end", "k", "kp", "s")


def _strings():
    return synth.pangenome(seed=61, founder_len=20_000, n_hap=8, batch=4)


def _index(S):
    off = S.offsets
    idx = rb.rb3_build_batch(torch.from_numpy(S.seq[:off[4]].copy()).to(DEV), S.lens[:4].copy())
    rb.rb3_merge(idx, rb.rb3_build_batch(torch.from_numpy(S.seq[off[4]:].copy()).to(DEV), S.lens[4:].copy()))
    return idx


def _index_and_queries():
    S = _strings()
    Q = synth.mem_queries(S, seed=62, nq=3000, median=150, lo=1, hi=2000, sub=0.01)
    return _index(S), Q


def _records(out, n):
    return out[: n * 40].cpu().numpy().view(rb.SMEM_DTYPE)


def test_noalloc_matches_mem_search_on_two_calls():
    idx, Q = _index_and_queries()
    q = torch.from_numpy(Q.q).to(DEV)
    qoff = torch.from_numpy(Q.qoff).to(DEV)
    for ell, smin in ((31, 1), (19, 2)):
        want, n_want = rb.rb3_mem_search(idx, q, qoff, ell, smin)
        assert n_want > 100
        cap = n_want + 10
        for call in range(2):
            out = torch.full((cap * 40,), 0xAB, dtype=torch.uint8, device=DEV)
            n = rb.rb3_mem_search_noalloc(idx, q, qoff, ell, smin, out, cap)
            assert n == n_want, (ell, smin, call)
            got = _records(out, n)
            for f in FIELDS:
                assert np.array_equal(got[f], want[f]), (f, ell, smin, call)


def test_noalloc_matches_the_oracle():
    """One call checked against the oracle's Algorithm 4 on the oracle's own BWT."""
    S = _strings()
    idx = _index(S)
    B = oracle.bwt(oracle.concat(S.seq, S.lens, True))
    assert np.array_equal(rb.rb3_export(idx), B)
    Q = synth.mem_queries(S, seed=63, nq=400, median=120, lo=1, hi=1500, sub=0.01)
    q = torch.from_numpy(Q.q).to(DEV)
    qoff = torch.from_numpy(Q.qoff).to(DEV)
    ref = oracle.smem(B, Q.q, Q.qoff, 25, 1)
    cap = len(ref) + 8
    out = torch.empty(cap * 40, dtype=torch.uint8, device=DEV)
    n = rb.rb3_mem_search_noalloc(idx, q, qoff, 25, 1, out, cap)
    assert n == len(ref) and n > 50
    got = _records(out, n)
    assert np.array_equal(np.stack([got[f] for f in FIELDS], axis=1), ref)


def test_noalloc_at_its_limits():
    """131,072 queries of 1,023 bases: exactly 524,288 chunks, the largest call
    (the scans run over many tiles); equal to rb3_mem_search."""
    S = _strings()
    idx = _index(S)
    nq, L = 131_072, 1_023
    Q = synth.mem_queries(S, seed=64, nq=nq, median=L, sigma=0.0, lo=L, hi=L, sub=0.02, random_frac=0.2)
    assert Q.nq == nq and int(Q.qoff[-1]) == nq * L
    q = torch.from_numpy(Q.q).to(DEV)
    qoff = torch.from_numpy(Q.qoff).to(DEV)
    want, n_want = rb.rb3_mem_search(idx, q, qoff, 31, 1)
    cap = n_want + 1
    out = torch.empty(cap * 40, dtype=torch.uint8, device=DEV)
    n = rb.rb3_mem_search_noalloc(idx, q, qoff, 31, 1, out, cap)
    assert n == n_want and n > nq
    got = _records(out, n)
    for f in FIELDS:
        assert np.array_equal(got[f], want[f]), f


def test_noalloc_limits_and_capacity():
    idx, Q = _index_and_queries()
    q = torch.from_numpy(Q.q).to(DEV)
    qoff = torch.from_numpy(Q.qoff).to(DEV)
    _, n_want = rb.rb3_mem_search(idx, q, qoff, 31, 1)
    out = torch.empty(40 * 4, dtype=torch.uint8, device=DEV)
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_mem_search_noalloc(idx, q, qoff, 31, 1, out, 4)
    assert e.value.code == rb.RB3_E_CAPACITY
    big = torch.zeros(131_073 + 1, dtype=torch.int64, device=DEV)
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_mem_search_noalloc(idx, q, big, 31, 1, out, 4)
    assert e.value.code == rb.RB3_E_INVAL


def test_noalloc_refuses_chunk_limit_and_bad_offsets():
    idx, _ = _index_and_queries()
    out = torch.empty(40 * 4, dtype=torch.uint8, device=DEV)
    # 130,000 queries of 1,025 bases: 133.25 M bases (under 2^27) but 650,000 chunks
    nq, L = 130_000, 1_025
    q = torch.ones(nq * L, dtype=torch.uint8, device=DEV)
    qoff = torch.arange(nq + 1, dtype=torch.int64, device=DEV) * L
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_mem_search_noalloc(idx, q, qoff, 31, 1, out, 4)
    assert e.value.code == rb.RB3_E_INVAL and "chunks" in str(e.value)
    # more bases than 524,288 chunks of 256 can hold
    n_big = 524_288 * 256 + 1
    qb = torch.ones(n_big, dtype=torch.uint8, device=DEV)
    qo = torch.tensor([0, n_big], dtype=torch.int64, device=DEV)
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_mem_search_noalloc(idx, qb, qo, 31, 1, out, 4)
    assert e.value.code == rb.RB3_E_INVAL
    del qb
    # offsets that run backwards inside [qoff[0], qoff[nq]]: refused before any search
    q3 = torch.ones(1000, dtype=torch.uint8, device=DEV)
    for bad in ([0, 1000, 10], [0, 600, 300, 1000]):
        qo = torch.tensor(bad, dtype=torch.int64, device=DEV)
        with pytest.raises(rb.RB3Error) as e:
            rb.rb3_mem_search_noalloc(idx, q3, qo, 31, 1, out, 4)
        assert e.value.code == rb.RB3_E_INVAL and "qoff" in str(e.value)
    # a good call right after the refusals
    qo = torch.tensor([0, 400, 1000], dtype=torch.int64, device=DEV)
    q3[:] = torch.from_numpy(_strings().seq[:1000].copy()).to(DEV)
    n = rb.rb3_mem_search_noalloc(idx, q3, qo, 31, 1, out, 4)
    assert n >= 1
