"""ctypes binding of librb3 (include/rb3.h).  Argument marshalling only: every
step of the computation runs in the library's CUDA kernels.  Function names
are the C ABI's.  Array arguments may be torch tensors (CUDA or CPU), numpy
arrays or raw integer addresses; streams are torch streams, raw cudaStream_t
integers or None (legacy default stream)."""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

RB3_OK, RB3_E_INVAL, RB3_E_NOMEM, RB3_E_CUDA, RB3_E_TIMEOUT, RB3_E_CAPACITY, RB3_E_IO = range(7)
_NAMES = {0: "RB3_OK", 1: "RB3_E_INVAL", 2: "RB3_E_NOMEM", 3: "RB3_E_CUDA", 4: "RB3_E_TIMEOUT",
          5: "RB3_E_CAPACITY", 6: "RB3_E_IO"}


class RB3Error(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class rb3_opts(ctypes.Structure):
    _fields_ = [("occ_interval", ctypes.c_int32), ("single_strand", ctypes.c_int32),
                ("seg_len", ctypes.c_int64), ("seed_cap", ctypes.c_int64),
                ("merge_form", ctypes.c_int32), ("search_form", ctypes.c_int32),
                ("chunk_len", ctypes.c_int64), ("walk_ctas_per_sm", ctypes.c_int32),
                ("sa_sample", ctypes.c_int32), ("batch_mb", ctypes.c_int32), ("hot_depth", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


class rb3_server_opts(ctypes.Structure):
    _fields_ = [("min_len", ctypes.c_int32), ("slots", ctypes.c_int32), ("min_occ", ctypes.c_int64),
                ("max_batch_bases", ctypes.c_int64), ("max_batch_requests", ctypes.c_int64),
                ("search_form", ctypes.c_int64), ("hot_depth", ctypes.c_int64), ("reserved", ctypes.c_int64 * 2)]


COMPLETION_DTYPE = np.dtype([("req_id", "<i8"), ("tag", "<i8"), ("n_smem", "<i8"), ("status", "<i4"),
                             ("batch_requests", "<i4"), ("t_submit_ns", "<i8"), ("t_done_ns", "<i8")])

SMEM_DTYPE = np.dtype([("qid", "<i8"), ("start", "<i4"), ("end", "<i4"), ("k", "<i8"), ("kp", "<i8"),
                       ("s", "<i8")])
assert SMEM_DTYPE.itemsize == 40

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_lib = None


def lib():
    """Loads librb3.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        sig = {
            "rb3_opts_default": (None, [_vp]),
            "rb3_build_batch": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp, ctypes.POINTER(_vp)]),
            "rb3_index_empty": (ctypes.c_int, [_vp, ctypes.POINTER(_vp)]),
            "rb3_merge": (ctypes.c_int, [_vp, _vp, _vp]),
            "rb3_merge_opts": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
            "rb3_merge_partition": (ctypes.c_int, [_vp, _i64, _i32, _vp]),
            "rb3_merge_positions": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i32, _vp, _vp]),
            "rb3_merge_apply": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
            "rb3_append_batches": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp, _i64, _vp, _vp]),
            "rb3_backward_search": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp, _vp]),
            "rb3_diversity_stats": (ctypes.c_int, [_vp, _i32]),
            "rb3_haplotype_diversity": (ctypes.c_int, [_vp, _vp, _vp, _i64, _i32, _i32, _i32, _i32, _i32, _i32,
                                                       _vp, _vp, _vp]),
            "rb3_mem_search": (ctypes.c_int, [_vp, _vp, _vp, _i64, _i32, _i64, _vp, _i64,
                                              ctypes.POINTER(_i64), _vp]),
            "rb3_mem_search_opts": (ctypes.c_int, [_vp, _vp, _vp, _i64, _i32, _i64, _vp, _vp, _i64,
                                                   ctypes.POINTER(_i64), _vp]),
            "rb3_mem_search_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _i64, _i32, _i64, _vp, _i64,
                                                      ctypes.POINTER(_i64), _vp]),
            "rb3_export": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
            "rb3_locate": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp]),
            "rb3_index_info": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                              ctypes.POINTER(_i64), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
            "rb3_drop_build_data": (ctypes.c_int, [_vp]),
            "rb3_index_compress": (ctypes.c_int, [_vp, _i32, _vp, ctypes.POINTER(_vp)]),
            "rb3_index_bytes": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
            "rb3_device_peak": (ctypes.c_int, [ctypes.POINTER(_i64), _i32]),
            "rb3_selftest_wait": (ctypes.c_int, [_i32, _vp]),
            "rb3_walk_stats": (ctypes.c_int, [_vp, _i32]),
            "rb3_search_stats": (ctypes.c_int, [_vp, _i32]),
            "rb3_index_save": (ctypes.c_int, [_vp, ctypes.c_char_p]),
            "rb3_index_load": (ctypes.c_int, [ctypes.c_char_p, _vp, ctypes.POINTER(_vp)]),
            "rb3_index_free": (None, [_vp]),
            "rb3_last_error": (ctypes.c_char_p, []),
            "rb3_encode_ascii": (ctypes.c_int, [ctypes.c_char_p, _i64, _vp]),
            "rb3_profile_enable": (ctypes.c_int, [ctypes.c_int]),
            "rb3_profile_reset": (ctypes.c_int, []),
            "rb3_profile_read": (ctypes.c_int, [ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double),
                                                ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_double), _i32,
                                                ctypes.POINTER(_i32)]),
            "rb3_profile_timeline": (ctypes.c_int, [ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double),
                                                    ctypes.POINTER(ctypes.c_double), _i64, ctypes.POINTER(_i64)]),
            "rb3_launch_count": (_i64, []),
            "rb3_tune_merge": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_double), _vp]),
            "rb3_bwasw": (ctypes.c_int, [_vp, _vp, _vp, _i64, _i32, _i32, _i32, _i32, _i32, _vp, _i64, _vp, _vp]),
            "rb3_tune_build": (ctypes.c_int, [_vp, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _vp, _vp, _vp]),
            "rb3_tune_search": (ctypes.c_int, [_vp, _vp, _vp, _i64, _i32, _i64, _vp, _vp,
                                               ctypes.POINTER(ctypes.c_double), _vp]),
            "rb3_server_opts_default": (None, [_vp]),
            "rb3_server_create": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(_vp)]),
            "rb3_server_submit": (ctypes.c_int, [_vp, _vp, _i64, _i64, ctypes.POINTER(_i64)]),
            "rb3_server_poll": (ctypes.c_int, [_vp, _vp, _i64, ctypes.POINTER(_i64), _i32]),
            "rb3_server_take": (ctypes.c_int, [_vp, _i64, _vp, _i64, ctypes.POINTER(_i64)]),
            "rb3_server_replay": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp, _vp, _vp]),
            "rb3_server_batches": (_i64, [_vp]),
            "rb3_server_stats": (ctypes.c_int, [_vp, _vp]),
            "rb3_server_destroy": (None, [_vp]),
            "rb3_probe_random_gather": (ctypes.c_int, [_i32, _i32, _i32, _i64, ctypes.POINTER(ctypes.c_double),
                                                       ctypes.POINTER(ctypes.c_double), _vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code: int):
    if code != RB3_OK:
        raise RB3Error(code, lib().rb3_last_error().decode(errors="replace"))


def _ptr(x):
    """Address of a tensor / array / int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr() if x.numel() else None
    if isinstance(x, np.ndarray):
        return x.ctypes.data if x.size else None
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _len(x) -> int:
    return int(x.numel()) if hasattr(x, "numel") else int(len(x))


def _opts(o):
    if o is None:
        return None
    if isinstance(o, rb3_opts):
        return o
    r = rb3_opts()
    for k, v in dict(o).items():
        setattr(r, k, int(v))
    return r


class Index:
    """Owns one rb3_index handle; freed with rb3_index_free."""

    def __init__(self, handle: int):
        self.handle = handle

    def free(self):
        if self.handle:
            lib().rb3_index_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return ctypes.c_void_p(self.handle)


def rb3_opts_default() -> rb3_opts:
    o = rb3_opts()
    lib().rb3_opts_default(ctypes.byref(o))
    return o


def rb3_build_batch(seq, lens, n_seq=None, opts=None, stream=None) -> Index:
    n_seq = _len(lens) if n_seq is None else n_seq
    out = _vp()
    o = _opts(opts)
    _check(lib().rb3_build_batch(_ptr(seq), _ptr(lens), n_seq, ctypes.byref(o) if o else None, _stream(stream),
                                 ctypes.byref(out)))
    return Index(out.value)


def rb3_index_empty(opts=None) -> Index:
    out = _vp()
    o = _opts(opts)
    _check(lib().rb3_index_empty(ctypes.byref(o) if o else None, ctypes.byref(out)))
    return Index(out.value)


def rb3_merge(dst: Index, src: Index, stream=None):
    _check(lib().rb3_merge(dst.handle, src.handle, _stream(stream)))


def rb3_merge_opts(dst: Index, src: Index, opts=None, stream=None):
    o = _opts(opts)
    _check(lib().rb3_merge_opts(dst.handle, src.handle, ctypes.byref(o) if o else None, _stream(stream)))


def rb3_merge_partition(lens, parts: int) -> np.ndarray:
    """owner[i] in [0, parts) of every input string (host only; see include/rb3.h)."""
    lens = np.ascontiguousarray(lens, dtype=np.int64)
    owner = np.zeros(len(lens), dtype=np.int32)
    _check(lib().rb3_merge_partition(_ptr(lens), len(lens), int(parts), _ptr(owner)))
    return owner


def rb3_merge_positions(dst: Index, src: Index, pos, owner=None, part: int = 0, opts=None, stream=None):
    """Writes into the device tensor pos the merged rows of src's rows owned by `part`
    (every row when owner is None), 0 elsewhere."""
    o = _opts(opts)
    own = None if owner is None else np.ascontiguousarray(owner, dtype=np.int32)
    _check(lib().rb3_merge_positions(dst.handle, src.handle, ctypes.byref(o) if o else None, _ptr(own), int(part),
                                     _ptr(pos), _stream(stream)))
    return pos


def rb3_merge_apply(dst: Index, src: Index, pos, stream=None):
    _check(lib().rb3_merge_apply(dst.handle, src.handle, _ptr(pos), _stream(stream)))


def rb3_merge_sharded(dst: Index, src: Index, lens, opts=None, group=None, stream=None):
    """The merge split over the ranks of a torch.distributed group, each rank
    holding its own copy of dst and src on its GPU: the ranks walk their share
    of src's input strings (lengths lens), add up their position arrays with one
    all-reduce, and each applies the whole array to its copy of dst."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    owner = rb3_merge_partition(lens, world)
    n2 = rb3_index_info(src)["n"]
    pos = torch.zeros(n2, dtype=torch.int64, device=torch.device("cuda", torch.cuda.current_device()))
    rb3_merge_positions(dst, src, pos, owner, rank, opts, stream)
    dist.all_reduce(pos, op=dist.ReduceOp.SUM, group=group)
    torch.cuda.synchronize()  # the all-reduce's stream may differ from `stream`
    rb3_merge_apply(dst, src, pos, stream)


def rb3_append_batches(dst: Index, seq, lens, batch_end, opts=None, stream=None):
    """Build each batch and merge it into dst, builds overlapping merges."""
    o = _opts(opts)
    lens_a = np.ascontiguousarray(lens, dtype=np.int64) if not hasattr(lens, "data_ptr") else lens
    ends = np.ascontiguousarray(batch_end, dtype=np.int64)
    _check(lib().rb3_append_batches(dst.handle, _ptr(seq), _ptr(lens_a), _len(lens_a), _ptr(ends), len(ends),
                                    ctypes.byref(o) if o else None, _stream(stream)))


def rb3_backward_search(idx: Index, q, qoff, nq=None, lo_hi=None, stream=None):
    nq = _len(qoff) - 1 if nq is None else nq
    if lo_hi is None:
        lo_hi = np.empty((nq, 2), dtype=np.int64)
    _check(lib().rb3_backward_search(idx.handle, _ptr(q), _ptr(qoff), nq, _ptr(lo_hi), _stream(stream)))
    return lo_hi


def rb3_bwasw(idx: Index, q, qoff, a: int = 1, b: int = 3, gap_open: int = 5, gap_ext: int = 2, W: int = 25,
              cap=None, nq=None, out=None, stream=None):
    """BWA-SW of every query's prefix DAWG against the index (see include/rb3.h):
    (N, 7) int64 records (qid, uk, us, k, k', s, H) sorted by (qid, uk, us, band
    rank).  Grows a host output buffer once when cap is not given."""
    nq = _len(qoff) - 1 if nq is None else nq
    n_out = _i64(0)
    if cap is None:
        cap = 1 << 16
    for _ in range(2):
        buf = np.empty((max(cap, 1), 7), dtype=np.int64) if out is None else out
        code = lib().rb3_bwasw(idx.handle, _ptr(q), _ptr(qoff), nq, int(a), int(b), int(gap_open), int(gap_ext),
                               int(W), _ptr(buf), int(cap), ctypes.byref(n_out), _stream(stream))
        if code == RB3_E_CAPACITY and out is None and n_out.value > cap:
            cap = n_out.value
            continue
        _check(code)
        return buf[:n_out.value] if out is None else n_out.value
    _check(code)


def rb3_haplotype_diversity(idx: Index, q, qoff, a: int = 1, b: int = 3, gap_open: int = 5, gap_ext: int = 2,
                            W: int = 25, redundancy: bool = True, nq=None, out=None, n_out=None, stream=None):
    """Returns (out, n_out): out[i, :n_out[i]] are query i's (k, k', s, H)
    records, best first.  Raises RB3Error (RB3_E_CAPACITY) when a query step
    overflows its cell table; n_out of that query is then -1."""
    nq = _len(qoff) - 1 if nq is None else nq
    if out is None:
        out = np.empty((nq, W, 4), dtype=np.int64)
    if n_out is None:
        n_out = np.empty(nq, dtype=np.int64)
    _check(lib().rb3_haplotype_diversity(idx.handle, _ptr(q), _ptr(qoff), nq, a, b, gap_open, gap_ext, W,
                                         int(redundancy), _ptr(out), _ptr(n_out), _stream(stream)))
    return out, n_out


def rb3_diversity_stats(reset: bool = False) -> dict:
    """Rank-all reads and table cells of rb3_haplotype_diversity since the
    last reset."""
    out = np.zeros(2, dtype=np.int64)
    _check(lib().rb3_diversity_stats(_ptr(out), int(reset)))
    return {"rank_reads": int(out[0]), "cells": int(out[1])}


def rb3_mem_search_opts(idx: Index, q, qoff, min_len: int, min_occ: int = 1, opts=None, out=None, cap=None,
                        nq=None, stream=None):
    """Returns (records, n).  Without `out` a host array is allocated and grown
    once on RB3_E_CAPACITY."""
    nq = _len(qoff) - 1 if nq is None else nq
    o = _opts(opts)
    n_out = _i64(0)
    auto = out is None
    if auto:
        cap = 1 << 16 if cap is None else cap
        out = np.empty(cap, dtype=SMEM_DTYPE)
    elif cap is None:
        cap = _len(out) if not hasattr(out, "element_size") else out.numel() * out.element_size() // 40
    r = lib().rb3_mem_search_opts(idx.handle, _ptr(q), _ptr(qoff), nq, int(min_len), int(min_occ),
                                  ctypes.byref(o) if o else None, _ptr(out), cap, ctypes.byref(n_out),
                                  _stream(stream))
    if r == RB3_E_CAPACITY and auto:
        cap = int(n_out.value)
        out = np.empty(cap, dtype=SMEM_DTYPE)
        r = lib().rb3_mem_search_opts(idx.handle, _ptr(q), _ptr(qoff), nq, int(min_len), int(min_occ),
                                      ctypes.byref(o) if o else None, _ptr(out), cap, ctypes.byref(n_out),
                                      _stream(stream))
    _check(r)
    n = int(n_out.value)
    return (out[:n] if auto else out), n


def rb3_mem_search(idx: Index, q, qoff, min_len: int, min_occ: int = 1, out=None, cap=None, nq=None, stream=None):
    return rb3_mem_search_opts(idx, q, qoff, min_len, min_occ, None, out, cap, nq, stream)


def rb3_mem_search_noalloc(idx: Index, q, qoff, min_len: int, min_occ: int, out, cap: int, nq=None, stream=None):
    """Allocation-free SMEM search for callers that cannot allocate device memory
    while searching (see include/rb3.h).  q, qoff, out: device tensors.  Returns n."""
    nq = _len(qoff) - 1 if nq is None else nq
    n_out = _i64(0)
    _check(lib().rb3_mem_search_noalloc(idx.handle, _ptr(q), _ptr(qoff), nq, int(min_len), int(min_occ), _ptr(out),
                                        int(cap), ctypes.byref(n_out), _stream(stream)))
    return int(n_out.value)


def rb3_tune_merge(dst: Index, src: Index, opts=None, stream=None):
    """(best rb3_opts, ms of the best walk phase) for merging src into dst."""
    o = _opts(opts) or rb3_opts_default()
    best = rb3_opts()
    ms = ctypes.c_double()
    _check(lib().rb3_tune_merge(dst.handle, src.handle, ctypes.byref(o), ctypes.byref(best), ctypes.byref(ms),
                                _stream(stream)))
    return best, ms.value


def rb3_tune_build(seq, lens, batch_end, opts=None, index_mb: int = 0, stream=None):
    """(best rb3_opts, [(D, build+merge ms, projected index MiB)]) for an incremental build."""
    o = _opts(opts) or rb3_opts_default()
    lens_a = np.ascontiguousarray(lens, dtype=np.int64) if not hasattr(lens, "data_ptr") else lens
    ends = np.ascontiguousarray(batch_end, dtype=np.int64)
    best = rb3_opts()
    ms = (ctypes.c_double * 3)()
    mb = (ctypes.c_double * 3)()
    _check(lib().rb3_tune_build(_ptr(seq), _ptr(lens_a), _len(lens_a), _ptr(ends), len(ends), ctypes.byref(o),
                                int(index_mb), ctypes.byref(best), ms, mb, _stream(stream)))
    return best, [(D, ms[i], mb[i]) for i, D in enumerate((32, 64, 128))]


def rb3_tune_search(idx: Index, q, qoff, min_len: int, min_occ: int = 1, opts=None, stream=None):
    """(best rb3_opts, ms) of the chunked SMEM search on these (device) queries."""
    o = _opts(opts) or rb3_opts_default()
    best = rb3_opts()
    ms = ctypes.c_double()
    _check(lib().rb3_tune_search(idx.handle, _ptr(q), _ptr(qoff), _len(qoff) - 1, int(min_len), int(min_occ),
                                 ctypes.byref(o), ctypes.byref(best), ctypes.byref(ms), _stream(stream)))
    return best, ms.value


def rb3_index_info(idx: Index) -> dict:
    n, m, D, fl = _i64(), _i64(), _i32(), _i32()
    C = (_i64 * 7)()
    _check(lib().rb3_index_info(idx.handle, ctypes.byref(n), ctypes.byref(m), C, ctypes.byref(D), ctypes.byref(fl)))
    return {"n": n.value, "m": m.value, "C": list(C), "occ_interval": D.value,
            "single_strand": bool(fl.value & 1), "has_build_data": bool(fl.value & 2),
            "run_length": bool(fl.value & 4), "sa_sample": fl.value >> 8}


def rb3_index_compress(idx: Index, span: int = 0, stream=None) -> Index:
    """Run-length copy of idx (read-only; queries run on it unchanged)."""
    out = _vp()
    _check(lib().rb3_index_compress(idx.handle, span, _stream(stream), ctypes.byref(out)))
    return Index(out.value)


def rb3_walk_stats(reset: bool = False) -> dict:
    """Counts of the merge walks since the last reset (see include/rb3.h)."""
    v = (_i64 * 4)()
    _check(lib().rb3_walk_stats(v, int(reset)))
    return {"seeds": v[0], "seed_block_reads": v[1], "walk_block_reads": v[2], "walked_again": v[3]}


def rb3_search_stats(reset: bool = False) -> dict:
    """Counts of the step-machine SMEM search since the last reset (see include/rb3.h)."""
    v = (_i64 * 2)()
    _check(lib().rb3_search_stats(v, int(reset)))
    return {"extensions": v[0], "block_reads": v[1]}


def rb3_selftest_wait(limit: int, stream=None):
    """Runs the bounded-wait self-test; raises RB3Error (RB3_E_TIMEOUT) as designed."""
    _check(lib().rb3_selftest_wait(int(limit), _stream(stream)))


def rb3_device_peak(reset: bool = False) -> int:
    """High-water mark (bytes) of the library's device allocations since the last reset."""
    v = _i64()
    _check(lib().rb3_device_peak(ctypes.byref(v), int(reset)))
    return v.value


def rb3_index_bytes(idx: Index) -> dict:
    b, r = _i64(), _i64()
    _check(lib().rb3_index_bytes(idx.handle, ctypes.byref(b), ctypes.byref(r)))
    return {"device_bytes": b.value, "runs": r.value}


def rb3_locate(idx: Index, rows, out=None, stream=None):
    """(string index, offset) of each BWT row; rows: int64 (host array or device tensor)."""
    r = rows if hasattr(rows, "data_ptr") else np.ascontiguousarray(rows, dtype=np.int64)
    n = _len(r)
    if out is None:
        out = np.empty((n, 2), dtype=np.int64)
    _check(lib().rb3_locate(idx.handle, _ptr(r), n, _ptr(out), _stream(stream)))
    return out


def rb3_export(idx: Index, codes=None, occ=None, stream=None, want_occ: bool = False):
    info = rb3_index_info(idx)
    if codes is None:
        codes = np.empty(info["n"], dtype=np.uint8)
    if occ is None and want_occ:
        occ = np.empty((info["n"] // info["occ_interval"] + 1, 6), dtype=np.int64)
    _check(lib().rb3_export(idx.handle, _ptr(codes), _ptr(occ), _stream(stream)))
    return (codes, occ) if want_occ else codes


def rb3_drop_build_data(idx: Index):
    _check(lib().rb3_drop_build_data(idx.handle))


def rb3_index_save(idx: Index, path: str):
    _check(lib().rb3_index_save(idx.handle, os.fsencode(path)))


def rb3_index_load(path: str, stream=None) -> Index:
    out = _vp()
    _check(lib().rb3_index_load(os.fsencode(path), _stream(stream), ctypes.byref(out)))
    return Index(out.value)


def rb3_index_free(idx: Index):
    idx.free()


def rb3_last_error() -> str:
    return lib().rb3_last_error().decode(errors="replace")


def rb3_encode_ascii(s) -> np.ndarray:
    b = s.encode() if isinstance(s, str) else bytes(s)
    out = np.empty(len(b), dtype=np.uint8)
    _check(lib().rb3_encode_ascii(b, len(b), out.ctypes.data if len(b) else None))
    return out


def rb3_profile_enable(on: bool = True):
    _check(lib().rb3_profile_enable(int(on)))


def rb3_profile_reset():
    _check(lib().rb3_profile_reset())


def rb3_profile_read() -> dict:
    """{name: (ms, calls, algorithmic bytes)} accumulated since the last reset."""
    cap = 128
    names = (ctypes.c_char_p * cap)()
    ms = (ctypes.c_double * cap)()
    calls = (_i64 * cap)()
    byts = (ctypes.c_double * cap)()
    n = _i32()
    _check(lib().rb3_profile_read(names, ms, calls, byts, cap, ctypes.byref(n)))
    return {names[i].decode(): (ms[i], calls[i], byts[i]) for i in range(min(n.value, cap))}


def rb3_profile_timeline() -> list:
    """[(name, start_ms, duration_ms)] of every phase since the last reset, start
    relative to the reset."""
    n = _i64()
    _check(lib().rb3_profile_timeline(None, None, None, 0, ctypes.byref(n)))
    cap = n.value
    names = (ctypes.c_char_p * max(cap, 1))()
    st = (ctypes.c_double * max(cap, 1))()
    du = (ctypes.c_double * max(cap, 1))()
    _check(lib().rb3_profile_timeline(names, st, du, cap, ctypes.byref(n)))
    return [(names[i].decode(), st[i], du[i]) for i in range(min(n.value, cap))]


def rb3_launch_count() -> int:
    return int(lib().rb3_launch_count())


def rb3_probe_random_gather(bytes_per_access: int, dependent: bool, threads_per_sm: int,
                            buffer_bytes: int = 8 << 30, stream=None):
    """(GB/s, M reads/s) of random reads; see include/rb3.h."""
    g, m = ctypes.c_double(), ctypes.c_double()
    _check(lib().rb3_probe_random_gather(int(bytes_per_access), int(dependent), int(threads_per_sm),
                                         int(buffer_bytes), ctypes.byref(g), ctypes.byref(m), _stream(stream)))
    return g.value, m.value


class Server:
    """Owns one rb3_server (served SMEM search with continuous batching)."""

    def __init__(self, handle: int, index: "Index"):
        self.handle = handle
        self.index = index  # keeps the index alive while serving

    def close(self):
        if self.handle:
            lib().rb3_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rb3_server_create(idx: Index, **opts) -> Server:
    o = rb3_server_opts()
    lib().rb3_server_opts_default(ctypes.byref(o))
    for k, v in opts.items():
        setattr(o, k, int(v))
    out = _vp()
    _check(lib().rb3_server_create(idx.handle, ctypes.byref(o), ctypes.byref(out)))
    return Server(out.value, idx)


def rb3_server_submit(srv: Server, q, tag: int = 0) -> int:
    q = np.ascontiguousarray(q, dtype=np.uint8)
    rid = _i64()
    _check(lib().rb3_server_submit(srv.handle, q.ctypes.data if q.size else None, q.size, int(tag), ctypes.byref(rid)))
    return rid.value


def rb3_server_poll(srv: Server, cap: int = 4096, wait_us: int = 0) -> np.ndarray:
    out = np.empty(cap, dtype=COMPLETION_DTYPE)
    n = _i64()
    _check(lib().rb3_server_poll(srv.handle, out.ctypes.data, cap, ctypes.byref(n), int(wait_us)))
    return out[:n.value]


def rb3_server_take(srv: Server, req_id: int, n_smem: int) -> np.ndarray:
    out = np.empty(max(1, n_smem), dtype=SMEM_DTYPE)
    n = _i64()
    _check(lib().rb3_server_take(srv.handle, int(req_id), out.ctypes.data, len(out), ctypes.byref(n)))
    return out[:n.value]


def rb3_server_replay(srv: Server, q, qoff, arrival_s):
    """Open-loop replay (native threads): (done_s, batch) per request, relative to the
    trace start; latency = done_s - arrival_s."""
    q = np.ascontiguousarray(q, dtype=np.uint8)
    qoff = np.ascontiguousarray(qoff, dtype=np.int64)
    arr = np.ascontiguousarray(np.round(np.asarray(arrival_s) * 1e9), dtype=np.int64)
    n = len(qoff) - 1
    done = np.empty(n, dtype=np.int64)
    batch = np.empty(n, dtype=np.int32)
    _check(lib().rb3_server_replay(srv.handle, _ptr(q), _ptr(qoff), n, _ptr(arr), _ptr(done), _ptr(batch)))
    return done / 1e9, batch


def rb3_server_batches(srv: Server) -> int:
    return int(lib().rb3_server_batches(srv.handle))


def rb3_server_stats(srv: Server) -> dict:
    """Slot time since creation (see include/rb3.h): batches, requests, bases and
    ns gathering / searching / publishing, summed over slots."""
    v = (_i64 * 6)()
    _check(lib().rb3_server_stats(srv.handle, v))
    return {"batches": v[0], "requests": v[1], "bases": v[2], "gather_ns": v[3], "search_ns": v[4],
            "publish_ns": v[5]}


def rb3_server_destroy(srv: Server):
    srv.close()
