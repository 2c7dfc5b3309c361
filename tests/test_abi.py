"""The C-ABI library builds, loads and exports every symbol include/fcfs.h declares.

Host-side checks only: no kernel is launched here.
"""
import ctypes as C
import os
import re

import pytest

from paper_1010_5562_gb300 import build as B
from paper_1010_5562_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return _lib.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fcfs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fcfs_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, "binding lacks %s" % n


def test_status_strings(lib):
    for code in range(7):
        assert lib.fcfs_status_string(code)
    assert lib.fcfs_version() >= 100


def test_host_argument_checks(lib):
    # NULL outputs and unsupported sizes are rejected before any device work
    assert lib.fcfs_forward(None, None, None, 0, 256, 8, 0, 0, None, None, None, 0, None) == 1
    assert lib.fcfs_forward(None, None, None, 0, 100, 8, 0, 0, 16, 16, None, 0, None) == 6   # T not 2^n
    assert lib.fcfs_forward(None, None, None, 0, 256, 0, 0, 0, 16, 16, None, 0, None) == 6   # K = 0
    assert lib.fcfs_forward(None, None, None, 0, 256, 8, 7, 0, 16, 16, None, 0, None) == 1   # bad precision
    assert lib.fcfs_forward(None, None, None, 0, 256, 8, 0, 0, 16, 16, None, 0, None) == 3   # no workspace
    assert lib.fcfs_forward(None, None, None, 0, 256, 8, 0, 4, 16, 16, None, 0, None) == 1   # bad flags
    # misaligned vertex pointers
    assert lib.fcfs_forward(20, 32, 48, 10, 256, 8, 0, 0, 16, 16, 256, 1 << 20, None) == 1
    assert lib.fcfs_edge_chain(None, None, None, None, None, -1, None, None) == 1
    assert lib.fcfs_edge_chain(None, None, None, None, None, 0, None, None) == 0


def test_workspace_sizes(lib):
    for prec in (0, 1):
        a = lib.fcfs_workspace_size(12576, 4096, 256, prec)
        b = lib.fcfs_workspace_size(0, 4096, 256, prec)
        assert a > b > 0 and a % 256 == 0
    assert lib.fcfs_workspace_size(100, 1000, 8, 0) == 0     # unsupported T


def test_no_cpu_fallback(monkeypatch, tmp_path):
    """Without the library the binding raises instead of computing anything."""
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        _lib.load()
