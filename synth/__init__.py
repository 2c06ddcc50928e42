"""Seeded synthetic inputs shaped like the paper's workloads.

The paper's data (human100/320, AllTheBacteria, SRR/DRR read sets) is not
available, so these generators stand in for it with the same shapes:
near-identical haplotypes of one founder (a pangenome), uneven bacterial-like
genomes with N-runs, short and long query reads.  Both the CUDA path's tests and
the oracle take their inputs from here; this module holds none of the method's
arithmetic (no concatenation, suffix order, rank or search).  Sequences are
uint8 codes A=1 C=2 G=3 T=4 N=5, strings back to back with int64 lengths.

Queries drawn from the reverse strand are reverse-complemented here; that is
input synthesis only (any query string is a valid input).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 240900613
_RC = np.array([0, 4, 3, 2, 1, 5], dtype=np.uint8)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Strings:
    """Strings back to back: seq[off[i]:off[i]+lens[i]]."""
    seq: np.ndarray
    lens: np.ndarray
    batches: list = field(default_factory=list)  # [(first string, end string)]

    @property
    def offsets(self) -> np.ndarray:
        off = np.zeros(len(self.lens) + 1, dtype=np.int64)
        np.cumsum(self.lens, out=off[1:])
        return off

    def subset(self, s0: int, s1: int) -> "Strings":
        off = self.offsets
        return Strings(self.seq[off[s0]:off[s1]], self.lens[s0:s1].copy())

    def ds_symbols(self) -> int:
        return int(2 * (self.lens.sum() + len(self.lens)))


@dataclass
class Queries:
    q: np.ndarray      # uint8 codes back to back
    qoff: np.ndarray   # int64, nq+1

    @property
    def nq(self) -> int:
        return len(self.qoff) - 1

    def subset(self, idx) -> "Queries":
        idx = np.asarray(idx, dtype=np.int64)
        lens = self.qoff[idx + 1] - self.qoff[idx]
        off = np.zeros(len(idx) + 1, dtype=np.int64)
        np.cumsum(lens, out=off[1:])
        parts = [self.q[self.qoff[i]:self.qoff[i + 1]] for i in idx]
        q = np.concatenate(parts) if parts else np.zeros(0, np.uint8)
        return Queries(q.astype(np.uint8), off)


def random_bases(g: np.random.Generator, n: int) -> np.ndarray:
    return g.integers(1, 5, size=n, dtype=np.uint8)


def _substitute(g, s: np.ndarray, rate: float) -> np.ndarray:
    """Replace each ACGT base with probability `rate` by a different ACGT base."""
    idx = np.flatnonzero(g.random(len(s)) < rate)
    if len(idx):
        old = s[idx]
        ok = old <= 4
        idx, old = idx[ok], old[ok]
        shift = g.integers(1, 4, size=len(idx), dtype=np.uint8)
        s[idx] = ((old - 1 + shift) % 4 + 1).astype(np.uint8)
    return s


def _substitute_sparse(g, s: np.ndarray, rate: float) -> np.ndarray:
    """Like _substitute, with the substituted positions drawn directly (a
    binomial count of uniform positions, repeats merged) instead of one
    uniform number per base: the same law up to the rare repeats, and cheap on
    megabase strings."""
    n = int(g.binomial(len(s), rate)) if len(s) else 0
    idx = np.unique(g.integers(0, len(s), size=n)) if n else np.zeros(0, np.int64)
    if len(idx):
        old = s[idx]
        ok = old <= 4
        idx, old = idx[ok], old[ok]
        shift = g.integers(1, 4, size=len(idx), dtype=np.uint8)
        s[idx] = ((old - 1 + shift) % 4 + 1).astype(np.uint8)
    return s


def _trunc_geometric(g, size: int, p: float = 0.5, hi: int = 10) -> np.ndarray:
    out = g.geometric(p, size=size)
    bad = out > hi
    while bad.any():
        out[bad] = g.geometric(p, size=int(bad.sum()))
        bad = out > hi
    return out.astype(np.int64)


def mutate(g, ref: np.ndarray, snp_rate: float, indel_rate: float) -> np.ndarray:
    """A haplotype of `ref`: SNPs (new base != old) and 50/50 insertions /
    deletions of geometric(0.5) length truncated to 1..10 (random inserted bases)."""
    hap = _substitute(g, ref.copy(), snp_rate)
    pos = np.flatnonzero(g.random(len(ref)) < indel_rate)
    if len(pos) == 0:
        return hap
    lens = _trunc_geometric(g, len(pos))
    ins = g.random(len(pos)) < 0.5
    pieces, prev = [], 0
    for p, L, is_ins in zip(pos.tolist(), lens.tolist(), ins.tolist()):
        if p < prev:
            continue
        pieces.append(hap[prev:p])
        if is_ins:
            pieces.append(random_bases(g, L))
            prev = p
        else:
            prev = min(p + L, len(hap))
    pieces.append(hap[prev:])
    return np.concatenate(pieces).astype(np.uint8)


# ---------------------------------------------------------------------------
# Workloads.  Seed = SEED_BASE + workload number.
# ---------------------------------------------------------------------------

def tiny(seed: int = SEED_BASE + 0, n_str: int = 64, length: int = 1000, nq: int = 1000, qlen: int = 20):
    """64 uniform ACGT strings of 1,000 bp; batch A = strings 0-31, batch B = 32-63;
    1,000 forward-strand queries of 20 bp at a uniform string and offset."""
    g = rng(seed)
    seq = random_bases(g, n_str * length)
    S = Strings(seq, np.full(n_str, length, dtype=np.int64), [(0, n_str // 2), (n_str // 2, n_str)])
    sid = g.integers(0, n_str, size=nq)
    off = g.integers(0, length - qlen + 1, size=nq)
    starts = sid * length + off
    q = seq[(starts[:, None] + np.arange(qlen)[None, :]).ravel()].copy()
    qoff = np.arange(nq + 1, dtype=np.int64) * qlen
    return S, Queries(q, qoff)


def pangenome(seed: int = SEED_BASE + 1, founder_len: int = 5_000_000, n_hap: int = 50,
              snp: float = 1e-3, indel: float = 1e-4, batch: int = 10) -> Strings:
    """Uniform ACGT founder; n_hap haplotypes with SNPs and short indels; batches of
    `batch` haplotypes (both strands are added by the index builder)."""
    g = rng(seed)
    founder = random_bases(g, founder_len)
    haps = [mutate(g, founder, snp, indel) for _ in range(n_hap)]
    lens = np.array([len(h) for h in haps], dtype=np.int64)
    batches = [(b, min(b + batch, n_hap)) for b in range(0, n_hap, batch)]
    return Strings(np.concatenate(haps), lens, batches)


def uneven(seed: int = SEED_BASE + 2, n_founders: int = 20, founder_len: int = 7_000_000,
           n_genomes: int = 2000, per_cluster: int = 100, median: float = 3e6, sigma: float = 0.35,
           lo: int = 1_000_000, hi: int = 7_000_000, sub: float = 0.01, n_frac: float = 0.005,
           nrun=(10, 100), batch: int = 64) -> Strings:
    """Bacterial-like genomes: genome g is a random window (lognormal length, clipped)
    of founder g // per_cluster with `sub` substitutions and N-runs covering about
    `n_frac` of its bases (run lengths uniform in nrun)."""
    g = rng(seed)
    founders = [random_bases(g, founder_len) for _ in range(n_founders)]
    L = np.clip(np.exp(np.log(median) + sigma * g.standard_normal(n_genomes)), lo, hi).astype(np.int64)
    L = np.minimum(L, founder_len)
    out = []
    mean_run = 0.5 * (nrun[0] + nrun[1])
    for i in range(n_genomes):
        f = founders[(i // per_cluster) % n_founders]
        st = int(g.integers(0, founder_len - L[i] + 1))
        s = _substitute_sparse(g, f[st:st + L[i]].copy(), sub)
        nr = int(round(n_frac * L[i] / mean_run))
        if nr:
            rl = g.integers(nrun[0], nrun[1] + 1, size=nr)
            rs = g.integers(0, max(1, L[i] - nrun[1]), size=nr)
            for a, b in zip(rs.tolist(), rl.tolist()):
                s[a:a + b] = 5
        out.append(s)
    lens = np.array([len(s) for s in out], dtype=np.int64)
    batches = [(b, min(b + batch, n_genomes)) for b in range(0, n_genomes, batch)]
    return Strings(np.concatenate(out), lens, batches)


def _sample_windows(g, S: Strings, lens: np.ndarray, sub_rates: np.ndarray) -> Queries:
    """Windows of the given lengths at a random string, offset and strand, then
    substitutions at the per-query rate."""
    off = S.offsets
    nq = len(lens)
    sid = g.integers(0, len(S.lens), size=nq)
    slen = S.lens[sid]
    lens = np.minimum(lens, slen)
    st = (g.random(nq) * (slen - lens + 1)).astype(np.int64)
    strand = g.random(nq) < 0.5
    qoff = np.zeros(nq + 1, dtype=np.int64)
    np.cumsum(lens, out=qoff[1:])
    q = np.empty(int(qoff[-1]), dtype=np.uint8)
    chunk = 65536
    for c0 in range(0, nq, chunk):
        c1 = min(nq, c0 + chunk)
        l = lens[c0:c1]
        rel = np.arange(int(l.sum()), dtype=np.int64) - np.repeat(qoff[c0:c1] - qoff[c0], l)
        base = np.repeat(off[sid[c0:c1]] + st[c0:c1], l)
        rev = np.repeat(strand[c0:c1], l)
        ll = np.repeat(l, l)
        idx = np.where(rev, base + ll - 1 - rel, base + rel)
        w = S.seq[idx]
        w = np.where(rev, _RC[w], w).astype(np.uint8)
        rates = np.repeat(sub_rates[c0:c1], l)
        m = (g.random(len(w)) < rates) & (w <= 4)
        if m.any():
            shift = g.integers(1, 4, size=int(m.sum()), dtype=np.uint8)
            w[m] = ((w[m] - 1 + shift) % 4 + 1).astype(np.uint8)
        q[qoff[c0]:qoff[c1]] = w
    return Queries(q, qoff)


def mem_queries(S: Strings, seed: int = SEED_BASE + 3, nq: int = 1_000_000, median: float = 150.0,
                sigma: float = 1.0, lo: int = 31, hi: int = 10_000, sub: float = 0.01,
                random_frac: float = 0.10) -> Queries:
    """Queries for batched MEM search: lognormal lengths (median 150, sigma 1,
    clipped to [31, 10000]); 90% windows of a random haplotype / offset / strand
    with 1% substitutions, 10% uniform-random ACGT of the same length law."""
    g = rng(seed)
    lens = np.clip(np.exp(np.log(median) + sigma * g.standard_normal(nq)), lo, hi).astype(np.int64)
    is_rand = g.random(nq) < random_frac
    Qs = _sample_windows(g, S, lens, np.full(nq, sub))
    # overwrite the random ones in place (same lengths)
    ql = Qs.qoff[1:] - Qs.qoff[:-1]
    rmask = np.repeat(is_rand, ql)
    nr = int(rmask.sum())
    if nr:
        Qs.q[rmask] = random_bases(g, nr)
    return Qs


def served_requests(S: Strings, rate: float, n_req: int, seed: int = SEED_BASE + 4,
                    lo: int = 100, hi: int = 100_000, sub=(0.001, 0.05)):
    """Open-loop Poisson arrivals at `rate` req/s; lengths log-uniform in [lo, hi];
    per-request substitution rate uniform in `sub`.  Returns (arrival seconds, Queries)."""
    g = rng(seed + int(rate))
    t = np.cumsum(g.exponential(1.0 / rate, size=n_req))
    lens = np.exp(g.uniform(np.log(lo), np.log(hi), size=n_req)).astype(np.int64)
    rates = g.uniform(sub[0], sub[1], size=n_req)
    return t, _sample_windows(g, S, lens, rates)


def served_index_strings(seed: int = SEED_BASE + 4, founder_len: int = 150_000_000, n_hap: int = 20,
                         batch: int = 4) -> Strings:
    """The served index: 20 haplotypes of a 150 Mb founder (SNPs 1e-3, indels 1e-4)."""
    return pangenome(seed=seed, founder_len=founder_len, n_hap=n_hap, batch=batch)


def random_strings(g, n_str: int, max_len: int, n_frac: float = 0.0, allow_empty: bool = True) -> Strings:
    """Small random lists for edge-case tests: lengths uniform in [0 or 1, max_len],
    optional N symbols at rate n_frac."""
    lens = g.integers(0 if allow_empty else 1, max_len + 1, size=n_str).astype(np.int64)
    seq = random_bases(g, int(lens.sum()))
    if n_frac > 0:
        seq[g.random(len(seq)) < n_frac] = 5
    return Strings(seq, lens, [(0, n_str)])
