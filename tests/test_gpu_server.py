"""Served SMEM search with continuous batching: every request's SMEMs are the
same alone (one request per micro-batch, one slot) and in the mix (bursts
admitted into shared micro-batches on several slots), and equal to
rb3_mem_search on the query by itself."""
import time

import numpy as np
import pytest
import torch

import synth
import paper_2409_00613_gb300 as rb

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
FIELDS = ("start", "end", "k", "kp", "s")


def _index():
    S = synth.pangenome(seed=81, founder_len=80_000, n_hap=8, batch=4)
    off = S.offsets
    idx = rb.rb3_build_batch(torch.from_numpy(S.seq[:off[4]].copy()).to(DEV), S.lens[:4].copy())
    rb.rb3_merge(idx, rb.rb3_build_batch(torch.from_numpy(S.seq[off[4]:].copy()).to(DEV), S.lens[4:].copy()))
    return S, idx


def _collect(srv, n, timeout=120.0):
    got, t0 = [], time.time()
    while len(got) < n:
        c = rb.rb3_server_poll(srv, 4096, 20000)
        got.extend(c.tolist())
        assert time.time() - t0 < timeout, "server did not complete the requests"
    return np.array(got, dtype=rb.COMPLETION_DTYPE)


def test_server_same_alone_and_in_the_mix():
    S, idx = _index()
    _, Q = synth.served_requests(S, rate=1000.0, n_req=150, lo=100, hi=30_000)
    ref, n = rb.rb3_mem_search(idx, Q.q, Q.qoff, 31, 1)
    per = [ref[ref["qid"] == i] for i in range(Q.nq)]
    queries = [Q.q[Q.qoff[i]:Q.qoff[i + 1]] for i in range(Q.nq)]

    def check(srv, comp, tagmap):
        for c in comp:
            assert c["status"] == 0 and c["t_done_ns"] >= c["t_submit_ns"]
            recs = rb.rb3_server_take(srv, c["req_id"], c["n_smem"])
            want = per[tagmap[c["req_id"]]]
            assert len(recs) == len(want)
            for f in FIELDS:
                assert np.array_equal(recs[f], want[f])

    alone = rb.rb3_server_create(idx, slots=1, max_batch_requests=1)
    tags = {}
    for i, qq in enumerate(queries):
        rid = rb.rb3_server_submit(alone, qq, i)
        tags[rid] = i
        comp = _collect(alone, 1)
        assert comp["batch_requests"][0] == 1
        check(alone, comp, tags)
    alone.close()

    mixed = rb.rb3_server_create(idx, slots=4, max_batch_bases=200_000)
    tags = {}
    for i, qq in enumerate(queries):
        tags[rb.rb3_server_submit(mixed, qq, i)] = i
    comp = _collect(mixed, len(queries))
    assert comp["batch_requests"].max() > 1  # requests were batched together
    assert rb.rb3_server_batches(mixed) < len(queries)
    check(mixed, comp, tags)
    mixed.close()


def test_server_rejects_bad_symbols():
    S, idx = _index()
    srv = rb.rb3_server_create(idx)
    with pytest.raises(rb.RB3Error):
        rb.rb3_server_submit(srv, np.array([1, 2, 0], np.uint8))
    srv.close()


def test_server_plain_kernel_same_records():
    """Micro-batches run with the one-query-per-thread kernel (search_form 1)
    give the same records as the default form."""
    S, idx = _index()
    _, Q = synth.served_requests(S, rate=1000.0, n_req=80, lo=100, hi=20_000)
    ref, _ = rb.rb3_mem_search(idx, Q.q, Q.qoff, 31, 1)
    srv = rb.rb3_server_create(idx, slots=3, search_form=1, max_batch_bases=100_000)
    tags = {rb.rb3_server_submit(srv, Q.q[Q.qoff[i]:Q.qoff[i + 1]], i): i for i in range(Q.nq)}
    for c in _collect(srv, Q.nq):
        assert c["status"] == 0
        recs = rb.rb3_server_take(srv, c["req_id"], c["n_smem"])
        want = ref[ref["qid"] == tags[c["req_id"]]]
        for f in FIELDS:
            assert np.array_equal(recs[f], want[f])
    srv.close()
    with pytest.raises(rb.RB3Error):
        rb.rb3_server_create(idx, search_form=7)


def test_server_replay_open_loop():
    """The native replay submits every request at its arrival time and
    reports each completion after its arrival; an impossible rate (all at
    once) still completes, in micro-batches of more than one request."""
    S, idx = _index()
    _, Q = synth.served_requests(S, rate=1000.0, n_req=400, lo=100, hi=20_000)
    for rate in (2000.0, 1e9):
        arr = np.cumsum(synth.rng(5).exponential(1.0 / rate, size=Q.nq))
        srv = rb.rb3_server_create(idx, slots=4)
        done, batch = rb.rb3_server_replay(srv, Q.q, Q.qoff, arr)
        st = rb.rb3_server_stats(srv)
        nb = rb.rb3_server_batches(srv)
        srv.close()
        assert (done >= arr).all() and (batch >= 1).all()
        # the slots' accounts: every request and base once, in the batches run
        assert st["batches"] == nb and st["requests"] == Q.nq and st["bases"] == int(Q.qoff[-1])
        assert min(st["gather_ns"], st["search_ns"], st["publish_ns"]) >= 0 and st["search_ns"] > 0
        if rate > 1e6:
            assert batch.max() > 1
    with pytest.raises(rb.RB3Error):
        srv = rb.rb3_server_create(idx)
        try:
            rb.rb3_server_replay(srv, Q.q, Q.qoff, arr[::-1].copy())
        finally:
            srv.close()
