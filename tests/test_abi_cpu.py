"""CPU-side checks of the boundary: the CUDA library builds, loads and exports
every symbol include/rb3.h declares; without a GPU a compute call fails loudly
(no CPU fallback)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2409_00613_gb300 as rb

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "rb3.h")


def declared():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rb3_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for must in ("rb3_build_batch", "rb3_merge", "rb3_mem_search", "rb3_backward_search", "rb3_export",
                 "rb3_index_save", "rb3_index_load", "rb3_index_free", "rb3_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = rb.lib()
    for name in declared():
        assert hasattr(L, name), name


def test_struct_layouts_match_header():
    assert ctypes.sizeof(rb.rb3_opts) == 4 + 4 + 8 + 8 + 4 + 4 + 8 + 4 + 4 + 4 + 4 * 5
    assert rb.SMEM_DTYPE.itemsize == 40


def test_encode_ascii():
    assert list(rb.rb3_encode_ascii("ACGTacgtNx-")) == [1, 2, 3, 4, 1, 2, 3, 4, 5, 5, 5]


def test_no_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    seq = np.array([1, 2, 3, 4], dtype=np.uint8)
    with pytest.raises(rb.RB3Error) as e:
        rb.rb3_build_batch(seq, np.array([4], dtype=np.int64))
    assert e.value.code in (rb.RB3_E_CUDA, rb.RB3_E_NOMEM)
