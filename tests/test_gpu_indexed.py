"""GPU parity of merges whose new strings are already (wholly or in long
stretches) in the index: exact duplicates, reverse-complement duplicates,
strings whose long suffix or prefix equals an indexed string's, near
duplicates, copies inside one batch and strings held by many copies.  In these
merges the new suffixes tie with indexed ones over up to a megabase, which is
where Algorithm 1's walk and the segment seeds do all of their work.  The
expected BWT is the oracle's incremental build (each string's double-strand
BWT by naive sort, then Algorithm 1 merges one string at a time), bit-exact."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2409_00613_gb300 as rb

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
RC = np.array([0, 4, 3, 2, 1, 5], dtype=np.uint8)


def rc(s):
    return RC[s[::-1]]


def _strings(*parts):
    seq = np.concatenate(parts).astype(np.uint8) if parts else np.zeros(0, np.uint8)
    return seq, np.array([len(p) for p in parts], dtype=np.int64)


def _build(parts, opts):
    seq, lens = _strings(*parts)
    return rb.rb3_build_batch(torch.from_numpy(seq).to(DEV), lens, opts=opts)


def _expected(parts, both=True):
    seq, lens = _strings(*parts)
    return oracle.build_incremental(seq, lens, both, group=1)


@pytest.fixture(scope="module")
def base():
    g = synth.rng(synth.SEED_BASE + 501)
    P0 = synth.random_bases(g, 1_000_000)
    P1 = synth.random_bases(g, 1_000_000)
    R = synth.random_bases(g, 5_000)
    return P0, P1, R


def _cases(P0, P1, R):
    snp = P0.copy()
    snp[500_000] = (snp[500_000] % 4) + 1
    return {
        "exact duplicate": [P1],
        "reverse-complement duplicate": [rc(P0)],
        "900 kb suffix to the sentinel": [np.concatenate([R[:1000], P0[100_000:]])],
        "700 kb prefix": [np.concatenate([P1[:700_000], R[:3000]])],
        "one SNP in the middle": [snp],
        "two copies in the batch": [P0, P0],
        "duplicate beside a fresh string": [R, P1, R[::-1].copy()],
    }


_WANT = {}


@pytest.mark.parametrize("D", [32, 64])
@pytest.mark.parametrize("seg_len", [0, 512])
def test_merge_of_indexed_strings(base, D, seg_len):
    P0, P1, R = base
    opts = {"occ_interval": D, "seg_len": seg_len}
    for name, new in _cases(P0, P1, R).items():
        idx = _build([P0, P1], opts)
        rb.rb3_merge_opts(idx, _build(new, opts), opts)
        got = rb.rb3_export(idx)
        if name not in _WANT:
            _WANT[name] = _expected([P0, P1] + new)
        want = _WANT[name]
        assert len(got) == len(want), name
        assert np.array_equal(got, want), name
        idx.free()


def test_merge_of_a_string_held_by_many_copies():
    """70 copies of a 40 kb string in the index, one more merged in (with a
    fresh string and a 30 kb prefix of it): every prefix of every new suffix of
    the copy occurs at least 70 times in the index."""
    g = synth.rng(synth.SEED_BASE + 502)
    Q = synth.random_bases(g, 40_000)
    mid = synth.random_bases(g, 2_000)
    new = [Q, mid, Q[:30_000].copy()]
    opts = {"occ_interval": 32, "seg_len": 512}
    idx = _build([Q] * 70, opts)
    rb.rb3_merge_opts(idx, _build(new, opts), opts)
    got = rb.rb3_export(idx)
    assert np.array_equal(got, _expected([Q] * 70 + new))
    assert oracle.certify(got, oracle.concat(*_strings(*([Q] * 70 + new)), True)) == 0


def test_merge_of_indexed_strings_single_strand(base):
    P0, P1, R = base
    opts = {"occ_interval": 32, "seg_len": 512, "single_strand": 1}
    for new in ([P1], [np.concatenate([R[:1000], P0[200_000:]])], [P0, P0]):
        idx = _build([P0, P1], opts)
        rb.rb3_merge_opts(idx, _build(new, opts), opts)
        assert np.array_equal(rb.rb3_export(idx), _expected([P0, P1] + new, both=False))
        idx.free()
