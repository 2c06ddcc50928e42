"""The merge split over ranks (rb3_merge_partition / rb3_merge_positions /
rb3_merge_apply), host side, on CPU: two gloo ranks split a small merge's
input strings with the library's partition, each rank fills the merged rows of
its own strings' suffixes (the walk, which needs a GPU, is stood in for by the
oracle's Algorithm 1 positions restricted to those rows), the ranks add their
arrays with one all-reduce, and the result is checked: every row is written
by exactly one rank, the sum is Algorithm 1's whole position array, and the
stable interleave at those rows is the oracle's merged BWT."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
import paper_2409_00613_gb300 as rb


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(seed):
    g = synth.rng(seed)
    S = synth.random_strings(g, 13, 400, n_frac=0.02, allow_empty=True)
    off = S.offsets
    A, B = S.subset(0, 5), S.subset(5, 13)
    B1 = oracle.bwt(oracle.concat(A.seq, A.lens, True))
    T2 = oracle.concat(B.seq, B.lens, True)
    SA2 = oracle.suffix_array(T2)
    B2 = oracle.bwt_from_sa(T2, SA2)
    M, pos = oracle.merge(B1, B2, want_pos=True)
    # the input string of every row of B2 (DS string d = input string d // 2)
    ends = np.flatnonzero(T2 == 0)
    ds = np.searchsorted(ends, SA2)
    return B, B1, B2, M, pos, ds // 2


def _interleave(B1, B2, pos):
    out = np.empty(len(B1) + len(B2), dtype=np.uint8)
    mask = np.zeros(len(out), dtype=bool)
    mask[pos] = True
    out[mask] = B2
    out[~mask] = B1
    return out


def _rank_main(rank, world, port, seed, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        B, B1, B2, M, pos_all, string_of_row = _case(seed)
        owner = rb.rb3_merge_partition(B.lens, world)
        mine = owner[string_of_row] == rank
        part = torch.from_numpy(np.where(mine, pos_all, 0).astype(np.int64))
        written = torch.from_numpy(mine.astype(np.int64))
        dist.all_reduce(part, op=dist.ReduceOp.SUM)
        dist.all_reduce(written, op=dist.ReduceOp.SUM)
        ok = (bool((written.numpy() == 1).all()) and np.array_equal(part.numpy(), pos_all)
              and np.array_equal(_interleave(B1, B2, part.numpy()), M))
        q.put((rank, ok, int(mine.sum())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_merge_positions_over_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, 4100 + world, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for _, ok, _ in res), res
    assert sum(n for _, _, n in res) == len(_case(4100 + world)[2])
    assert all(n > 0 for _, _, n in res)  # every rank walked something


def test_partition_balances_and_is_deterministic():
    g = synth.rng(9)
    lens = g.integers(0, 5_000_000, size=200)
    for parts in (1, 2, 3, 8):
        owner = rb.rb3_merge_partition(lens, parts)
        assert owner.min() >= 0 and owner.max() < parts
        assert np.array_equal(owner, rb.rb3_merge_partition(lens, parts))
        load = np.bincount(owner, weights=lens + 1, minlength=parts)
        # longest-first greedy: no part exceeds the mean by more than the longest string
        assert load.max() - (lens + 1).sum() / parts <= lens.max() + 1
    assert len(rb.rb3_merge_partition(np.zeros(0, np.int64), 4)) == 0
    with pytest.raises(rb.RB3Error):
        rb.rb3_merge_partition(np.array([3, -1]), 2)
