"""The allocation-free SMEM entry point (for callers that cannot allocate device
memory while they search) gives the same records, in the same order, as
rb3_mem_search; two calls in a row share and reuse its fixed scratch.  This
file is collected last on purpose."""
import numpy as np
import pytest
import torch

import synth
import paper_2409_00613_gb300 as rb

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _index_and_queries():
    S = synth.pangenome(seed=61, founder_len=20_000, n_hap=8, batch=4)
    off = S.offsets
    idx = rb.rb3_build_batch(torch.from_numpy(S.seq[:off[4]].copy()).to(DEV), S.lens[:4].copy())
    rb.rb3_merge(idx, rb.rb3_build_batch(torch.from_numpy(S.seq[off[4]:].copy()).to(DEV), S.lens[4:].copy()))
    Q = synth.mem_queries(S, seed=62, nq=3000, median=150, lo=1, hi=2000, sub=0.01)
    return idx, Q


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
            got = out[: n * 40].cpu().numpy().view(rb.SMEM_DTYPE)
            for f in ("qid", "start", "end", "k", "kp", "s"):
                assert np.array_equal(got[f], want[f]), (f, ell, smin, call)


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
