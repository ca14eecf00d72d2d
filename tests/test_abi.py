"""The C-ABI library builds, loads and exports every function declared in
include/*.h; host-side argument checks answer without touching a GPU."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2607_14054_gb300 import _abi, buildlib as _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(sos_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return _abi.load()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "sos_filter" in names and len(names) >= 6
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_status_strings(lib):
    assert _abi.sos_abi_version() >= 1
    for code, name in _abi.STATUS_NAMES.items():
        assert _abi.sos_status_str(code) == name


def test_workspace_size_host_checks(lib):
    lengths = np.array([8192, 0, 5, 100000], dtype=np.int64)
    n = _abi.sos_workspace_size(4, 8, lengths.ctypes.data, None)
    assert n > 0
    bigger = _abi.sos_workspace_size(4, 8, np.array([8192, 0, 5, 10**7], dtype=np.int64).ctypes.data, None)
    assert bigger > n
    # invalid: kmax out of range, unsupported tuning, negative length
    assert _abi.sos_workspace_size(4, 9, lengths.ctypes.data, None) == 0
    assert _abi.sos_workspace_size(4, 8, lengths.ctypes.data, (24, 8, 0, 0)) == 0
    bad = np.array([1, -1, 3, 4], dtype=np.int64)
    assert _abi.sos_workspace_size(4, 8, bad.ctypes.data, None) == 0


def test_filter_rejects_bad_arguments_on_host(lib):
    # These return before any CUDA call is made.
    lengths = np.array([16], dtype=np.int64)
    dummy = 1 << 20  # never dereferenced: the checks fire first
    assert _abi.sos_filter(dummy, 0, dummy, 1, 1, dummy, lengths.ctypes.data, 0, dummy, 0,
                           dummy, 1 << 20, None, 0) == -1          # sos NULL
    assert _abi.sos_filter(dummy, dummy, dummy, 1, 9, dummy, lengths.ctypes.data, 0, dummy, 0,
                           dummy, 1 << 20, None, 0) == -6          # kmax > 8
    assert _abi.sos_filter(dummy, dummy, dummy, 1, 2, dummy, lengths.ctypes.data, 0, dummy, 0,
                           dummy, 1 << 20, (16, 5, 0, 0), 0) == -6  # unsupported tuning
    assert _abi.sos_filter(dummy, dummy, dummy, 1, 2, dummy, lengths.ctypes.data, 0, 2 * dummy, 0,
                           dummy, 16, None, 0) == -5               # workspace too small
    assert _abi.sos_filter(dummy, dummy, dummy, 1, 2, dummy, lengths.ctypes.data, 0, dummy + 8, 0,
                           dummy, 1 << 20, None, 0) == -1          # y overlaps x


def test_host_path_sizes_on_host(lib):
    """sos_filter_host_sizes answers on the host: the block is rounded up to
    whole float4s, an eighth of the signal (at least 2^20) by default, the
    staging area holds four block buffers, and negative lengths or too many
    sections are refused."""
    lh = np.array([3_000_000, 5, 0, 700_001], dtype=np.int64)
    st, ws, stg, blk = _abi.sos_filter_host_sizes(4, 8, lh.ctypes.data, 1001, None)
    assert st == 0 and blk == 1004 and ws > 0 and stg >= 4 * 4 * 1004
    st, ws2, stg2, blk2 = _abi.sos_filter_host_sizes(4, 8, lh.ctypes.data, 0, None)
    assert st == 0 and blk2 == 1 << 20 and stg2 >= 4 * 4 * (1 << 20)
    big = np.array([1 << 26], dtype=np.int64)
    st, _, _, blk3 = _abi.sos_filter_host_sizes(1, 2, big.ctypes.data, 0, None)
    assert st == 0 and blk3 == (1 << 26) // 8
    bad = np.array([10, -1], dtype=np.int64)
    assert _abi.sos_filter_host_sizes(2, 2, bad.ctypes.data, 0, None)[0] == -1
    assert _abi.sos_filter_host_sizes(1, 9, big.ctypes.data, 0, None)[0] == -1
