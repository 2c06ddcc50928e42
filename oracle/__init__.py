"""CPU oracle for the BWT build / merge / search path (H. Li, arXiv 2409.00613).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only code
that may import this package.  The CUDA library and its Python binding never
import it and share no code with it.

The arithmetic lives in ``rb3_oracle.c`` (plain C, int64 everywhere); this
module only marshals numpy arrays through ctypes.  Symbol codes are
$=0 A=1 C=2 G=3 T=4 N=5.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py`` (brute force on tiny inputs, the paper's worked
SMEM and haplotype-diversity examples, closed-form LF/symmetry relations and
the LF-decode certificate).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rb3_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc.so")
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile rb3_oracle.c into oracle/_build/liborc.so with gcc."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        L.orc_concat.restype = ctypes.c_int64
        L.orc_concat.argtypes = [_u8p, _i64p, ctypes.c_int64, ctypes.c_int, _u8p]
        L.orc_suffix_array.argtypes = [_u8p, ctypes.c_int64, _i64p]
        L.orc_bwt_from_sa.argtypes = [_u8p, ctypes.c_int64, _i64p, _u8p]
        L.orc_bwt.argtypes = [_u8p, ctypes.c_int64, _u8p]
        L.orc_counts.argtypes = [_u8p, ctypes.c_int64, _i64p]
        L.orc_occ_table.argtypes = [_u8p, ctypes.c_int64, ctypes.c_int64, _i64p]
        L.orc_retrieve.restype = ctypes.c_int64
        L.orc_retrieve.argtypes = [_u8p, ctypes.c_int64, ctypes.c_int64, _u8p, ctypes.c_int64]
        L.orc_certify.restype = ctypes.c_int
        L.orc_certify.argtypes = [_u8p, ctypes.c_int64, _u8p, ctypes.c_int64, ctypes.c_int]
        L.orc_merge.argtypes = [_u8p, ctypes.c_int64, _u8p, ctypes.c_int64, _u8p, _i64p, ctypes.c_int]
        L.orc_build_incremental.restype = ctypes.c_int64
        L.orc_build_incremental.argtypes = [_u8p, _i64p, ctypes.c_int64, ctypes.c_int, ctypes.c_int64,
                                            _u8p, ctypes.c_int]
        L.orc_backward_search.argtypes = [_u8p, ctypes.c_int64, _u8p, _i64p, ctypes.c_int64, _i64p]
        L.orc_ext.argtypes = [_u8p, ctypes.c_int64, _i64p, ctypes.c_int, ctypes.c_int]
        L.orc_smem.restype = ctypes.c_int64
        L.orc_smem.argtypes = [_u8p, ctypes.c_int64, _u8p, _i64p, ctypes.c_int64, ctypes.c_int64,
                               ctypes.c_int64, _i64p, ctypes.c_int64]
        L.orc_smem_mt.restype = ctypes.c_int64
        L.orc_smem_mt.argtypes = [_u8p, ctypes.c_int64, _u8p, _i64p, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_int64, _i64p, ctypes.c_int64, ctypes.c_int]
        L.orc_occ_brute.restype = ctypes.c_int64
        L.orc_occ_brute.argtypes = [_u8p, ctypes.c_int64, _u8p, ctypes.c_int64]
        L.orc_lo_brute.restype = ctypes.c_int64
        L.orc_lo_brute.argtypes = [_u8p, ctypes.c_int64, _u8p, ctypes.c_int64]
        L.orc_smem_brute.restype = ctypes.c_int64
        L.orc_smem_brute.argtypes = [_u8p, ctypes.c_int64, _u8p, _i64p, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_int64, _i64p, ctypes.c_int64]
        L.orc_diversity.restype = ctypes.c_int64
        L.orc_diversity.argtypes = [_u8p, ctypes.c_int64, _u8p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _i64p,
                                    ctypes.c_int64]
        L.orc_diversity_many.restype = None
        L.orc_diversity_many.argtypes = [_u8p, ctypes.c_int64, _u8p, _i64p, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                         _i64p, _i64p]
        L.orc_bwasw.restype = ctypes.c_int64
        L.orc_bwasw.argtypes = [_u8p, ctypes.c_int64, _u8p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _i64p, ctypes.c_int64]
        L.orc_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(_u8p)


def _i64(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(_i64p)


def max_threads() -> int:
    return int(lib().orc_max_threads())


def concat(seq, lens, both: bool = True) -> np.ndarray:
    """T = P0 $ [rc(P0) $] P1 $ ... (codes), from strings back to back."""
    seq, ps = _u8(seq)
    lens, pl = _i64(lens)
    n = lib().orc_concat(ps, pl, len(lens), int(both), None)
    T = np.empty(n, dtype=np.uint8)
    lib().orc_concat(ps, pl, len(lens), int(both), T.ctypes.data_as(_u8p))
    return T


def suffix_array(T) -> np.ndarray:
    T, pt = _u8(T)
    SA = np.empty(len(T), dtype=np.int64)
    lib().orc_suffix_array(pt, len(T), SA.ctypes.data_as(_i64p))
    return SA


def bwt(T) -> np.ndarray:
    T, pt = _u8(T)
    B = np.empty(len(T), dtype=np.uint8)
    lib().orc_bwt(pt, len(T), B.ctypes.data_as(_u8p))
    return B


def bwt_from_sa(T, SA) -> np.ndarray:
    T, pt = _u8(T)
    SA, psa = _i64(SA)
    B = np.empty(len(T), dtype=np.uint8)
    lib().orc_bwt_from_sa(pt, len(T), psa, B.ctypes.data_as(_u8p))
    return B


def counts(B) -> np.ndarray:
    """C_B(a) for a = 0..6 (C[6] = n)."""
    B, pb = _u8(B)
    C = np.empty(7, dtype=np.int64)
    lib().orc_counts(pb, len(B), C.ctypes.data_as(_i64p))
    return C


def occ_table(B, D: int) -> np.ndarray:
    """(n//D + 1, 6) array: rank_B(a, j*D)."""
    B, pb = _u8(B)
    out = np.empty((len(B) // D + 1, 6), dtype=np.int64)
    lib().orc_occ_table(pb, len(B), D, out.ctypes.data_as(_i64p))
    return out


def retrieve(B, i: int) -> np.ndarray:
    B, pb = _u8(B)
    out = np.empty(len(B) + 1, dtype=np.uint8)
    L = lib().orc_retrieve(pb, len(B), i, out.ctypes.data_as(_u8p), len(out))
    return out[:L].copy()


def certify(B, T, nthreads: int = 0) -> int:
    """0 iff B is the BWT of the string list concatenated in T."""
    B, pb = _u8(B)
    T, pt = _u8(T)
    return int(lib().orc_certify(pb, len(B), pt, len(T), nthreads))


def merge(B1, B2, nthreads: int = 0, want_pos: bool = False):
    """Algorithm 1: BWT of (strings of B1) followed by (strings of B2)."""
    B1, p1 = _u8(B1)
    B2, p2 = _u8(B2)
    M = np.empty(len(B1) + len(B2), dtype=np.uint8)
    pos = np.empty(len(B2), dtype=np.int64) if want_pos else None
    lib().orc_merge(p1, len(B1), p2, len(B2), M.ctypes.data_as(_u8p),
                    pos.ctypes.data_as(_i64p) if want_pos else None, nthreads)
    return (M, pos) if want_pos else M


def build_incremental(seq, lens, both: bool = True, group: int = 1, nthreads: int = 0) -> np.ndarray:
    """BWT of the list built group by group (O1 per group, Algorithm 1 merges)."""
    seq, ps = _u8(seq)
    lens, pl = _i64(lens)
    n = int(np.sum(lens + 1)) * (2 if both else 1)
    B = np.empty(n, dtype=np.uint8)
    got = lib().orc_build_incremental(ps, pl, len(lens), int(both), group, B.ctypes.data_as(_u8p),
                                      nthreads)
    assert got == n
    return B


def backward_search(B, q, qoff) -> np.ndarray:
    B, pb = _u8(B)
    q, pq = _u8(q)
    qoff, po = _i64(qoff)
    nq = len(qoff) - 1
    out = np.empty((nq, 2), dtype=np.int64)
    lib().orc_backward_search(pb, len(B), pq, po, nq, out.ctypes.data_as(_i64p))
    return out


def locate(T, SA, rows) -> np.ndarray:
    """Section "Locating with FM-index": the suffix of BWT row i starts at text
    position S(i); reported as (index of the string it lies in, offset on that
    string), strings numbered in the order of their sentinels in T.  Written
    out from that definition (numpy), not from Algorithm 2's sampling."""
    T = np.asarray(T)
    ends = np.flatnonzero(T == 0)  # the sentinel ending each string, in order
    p = np.asarray(SA, dtype=np.int64)[np.asarray(rows, dtype=np.int64)]
    t = np.searchsorted(ends, p)  # first sentinel at or after p
    start = np.where(t == 0, 0, ends[np.maximum(t - 1, 0)] + 1)
    return np.stack([t.astype(np.int64), p - start], axis=1)


def runs(B, span: int = 0):
    """Section "BWT construction" (Fig. 2): the run-length form of the BWT, its
    maximal runs of one symbol, as (symbols, lengths); with span > 0 every run
    is also cut at the positions that are multiples of span (the blocks of the
    static encoding).  Written out from that definition (numpy)."""
    B = np.asarray(B, dtype=np.uint8)
    n = len(B)
    if n == 0:
        return np.zeros(0, np.uint8), np.zeros(0, np.int64)
    starts = np.ones(n, dtype=bool)  # position i starts a run
    starts[1:] = B[1:] != B[:-1]
    if span > 0:
        starts[::span] = True
    first = np.flatnonzero(starts)
    lengths = np.diff(np.append(first, n)).astype(np.int64)
    return B[first].copy(), lengths


def ext(B, kks, a: int, forward: bool):
    B, pb = _u8(B)
    x = np.array(kks, dtype=np.int64)
    lib().orc_ext(pb, len(B), x.ctypes.data_as(_i64p), int(a), int(forward))
    return tuple(int(v) for v in x)


def smem(B, q, qoff, min_len: int, min_occ: int = 1, nthreads: int = 1) -> np.ndarray:
    """Algorithm 4 over every query: (N, 6) int64 records (qid,start,end,k,k',s)."""
    B, pb = _u8(B)
    q, pq = _u8(q)
    qoff, po = _i64(qoff)
    nq = len(qoff) - 1
    L = lib()
    if nthreads == 1:
        n = L.orc_smem(pb, len(B), pq, po, nq, min_len, min_occ, None, 0)
        out = np.empty((max(n, 1), 6), dtype=np.int64)
        L.orc_smem(pb, len(B), pq, po, nq, min_len, min_occ, out.ctypes.data_as(_i64p), n)
    else:
        n = L.orc_smem_mt(pb, len(B), pq, po, nq, min_len, min_occ, None, 0, nthreads)
        out = np.empty((max(n, 1), 6), dtype=np.int64)
        L.orc_smem_mt(pb, len(B), pq, po, nq, min_len, min_occ, out.ctypes.data_as(_i64p), n, nthreads)
    return out[:n]


def haplotype_diversity(B, P, a: int = 1, b: int = 3, q: int = 5, e: int = 2, W: int = 25,
                        redundancy: bool = True) -> np.ndarray:
    """Section "Estimating local haplotype diversity": Algorithm 5 (BWA-SW) on
    the linear query P, end to start, against the text's prefix DAWG, with the
    top-W band; (N, 4) int64 records (k, k', s, H) of the end-to-end
    alignments with H > 0, best first, redundant bi-intervals filtered.  The
    readings the paper leaves open are listed at orc_diversity."""
    B, pb = _u8(B)
    P, pp = _u8(P)
    L = lib()
    n = L.orc_diversity(pb, len(B), pp, len(P), a, b, q, e, W, int(redundancy), None, 0)
    out = np.empty((max(n, 1), 4), dtype=np.int64)
    L.orc_diversity(pb, len(B), pp, len(P), a, b, q, e, W, int(redundancy), out.ctypes.data_as(_i64p), n)
    return out[:n].copy()


def haplotype_diversity_many(B, q, qoff, a: int = 1, b: int = 3, gq: int = 5, e: int = 2, W: int = 25,
                             redundancy: bool = True):
    """haplotype_diversity for every query q[qoff[i]:qoff[i+1]] with one
    rank table over B (W >= 1): (out (nq, W, 4), n_out (nq,))."""
    assert W >= 1
    B, pb = _u8(B)
    q, pq = _u8(q)
    qoff, po = _i64(qoff)
    nq = len(qoff) - 1
    out = np.zeros((max(nq, 1), W, 4), dtype=np.int64)
    n_out = np.zeros(max(nq, 1), dtype=np.int64)
    lib().orc_diversity_many(pb, len(B), pq, po, nq, a, b, gq, e, W, int(redundancy), out.ctypes.data_as(_i64p),
                             n_out.ctypes.data_as(_i64p))
    return out[:nq], n_out[:nq]


def bwasw(B, P, a: int = 1, b: int = 3, q: int = 5, e: int = 2, W: int = 25) -> np.ndarray:
    """Section "Finding inexact matches with BWA-SW": Algorithm 5 between the
    prefix DAWG of P (built from the BWT of the one-string text P$) and that
    of the indexed text; (N, 6) int64 records (uk, us, k, k', s, H): a query
    node (the SA interval (uk, us) of its strings in P$) and a text node with
    H > 0, the band of W cells per query node (0: no band), sorted by query
    node, then H descending, k, k', s."""
    B, pb = _u8(B)
    P = np.asarray(P, dtype=np.uint8)
    BP, pbp = _u8(bwt(concat(P, np.array([len(P)], np.int64), False)))
    L = lib()
    n = L.orc_bwasw(pb, len(B), pbp, len(BP), a, b, q, e, W, None, 0)
    out = np.empty((max(n, 1), 6), dtype=np.int64)
    L.orc_bwasw(pb, len(B), pbp, len(BP), a, b, q, e, W, out.ctypes.data_as(_i64p), n)
    out = out[:n]
    order = np.lexsort((out[:, 4], out[:, 3], out[:, 2], -out[:, 5], out[:, 1], out[:, 0]))
    return out[order].copy()


def occ_brute(T, P) -> int:
    T, pt = _u8(T)
    P, pp = _u8(P)
    return int(lib().orc_occ_brute(pt, len(T), pp, len(P)))


def lo_brute(T, P) -> int:
    T, pt = _u8(T)
    P, pp = _u8(P)
    return int(lib().orc_lo_brute(pt, len(T), pp, len(P)))


def smem_brute(T, q, qoff, min_len: int, min_occ: int = 1) -> np.ndarray:
    T, pt = _u8(T)
    q, pq = _u8(q)
    qoff, po = _i64(qoff)
    nq = len(qoff) - 1
    n = lib().orc_smem_brute(pt, len(T), pq, po, nq, min_len, min_occ, None, 0)
    out = np.empty((max(n, 1), 6), dtype=np.int64)
    lib().orc_smem_brute(pt, len(T), pq, po, nq, min_len, min_occ, out.ctypes.data_as(_i64p), n)
    return out[:n]
