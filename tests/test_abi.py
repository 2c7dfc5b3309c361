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


def test_grouped_plan_workspaces(lib):
    """Host plans of the grouped forms, through the size functions (no device
    work): the T = 65536, K = 1024 clip takes the pruned FFT along y, whose
    workspace holds conj(H) as K x T complex FP32 and no partial planes; the
    split-FP16 contraction over y holds H as 2 x 2K x (T + 1 rounded up to 64)
    FP16; forcing a grouped form on a small clip grows the workspace."""
    V, T, K = 945450, 65536, 1024
    h_bytes = 2 * (2 * K) * 65600 * 2
    poly_bytes = K * T * 8
    try:
        lib.fcfs_debug_set_hybrid(0)
        direct = lib.fcfs_workspace_size(V, T, K, 1)
        adj_direct = lib.fcfs_adjoint_workspace_size(V, T, K, 1)
        small_direct = lib.fcfs_workspace_size(12576, 4096, 256, 1)
        small_direct32 = lib.fcfs_workspace_size(12576, 4096, 256, 0)
        batch_direct = lib.fcfs_batch_workspace_size(100000, 8, 2048, 128, 1)
        lib.fcfs_debug_set_hybrid(1)
        auto = lib.fcfs_workspace_size(V, T, K, 1)
        assert auto >= poly_bytes and auto >= direct   # FFT form, or the validation plan
        assert lib.fcfs_workspace_size(V, T, K, 0) >= poly_bytes
        # the adjoint groups by y and by x: two permutations of V corners more
        assert lib.fcfs_adjoint_workspace_size(V, T, K, 1) >= adj_direct + 2 * 4 * V
        lib.fcfs_debug_set_hybrid(2)
        assert lib.fcfs_workspace_size(V, T, K, 1) >= h_bytes
        assert lib.fcfs_workspace_size(12576, 4096, 256, 1) > small_direct
        assert lib.fcfs_batch_workspace_size(100000, 8, 2048, 128, 1) > batch_direct
        # the split-FP16 contraction over y needs tensor cores: FP32 stays direct
        assert lib.fcfs_workspace_size(12576, 4096, 256, 0) == small_direct32
        lib.fcfs_debug_set_hybrid(3)
        assert lib.fcfs_workspace_size(12576, 4096, 256, 0) >= 256 * 4096 * 8
        assert lib.fcfs_workspace_size(12576, 4096, 256, 1) >= 256 * 4096 * 8
    finally:
        lib.fcfs_debug_set_hybrid(1)


def test_cosine_host_checks(lib):
    """The cosine-series entry points: sizes and host-detectable errors."""
    cw = lib.fcfs_cosine_workspace_size
    for prec in (0, 1):
        a = cw(12576, 4096, 256, prec)
        b = cw(0, 4096, 256, prec)
        assert a > b > 0 and a % 256 == 0
        # its K x K partial planes are a quarter of the Fourier block's 2K x 2K
        assert a < lib.fcfs_workspace_size(12576, 8192, 256, prec)
    assert cw(100, 32768, 64, 1) > 0          # largest period: sines of period 2T = 65536
    assert cw(100, 65536, 64, 1) == 0         # 2T beyond the tables
    assert cw(100, 1000, 8, 1) == 0           # T not a power of two
    assert cw(100, 256, 0, 1) == 0            # K = 0
    f = lib.fcfs_cosine
    assert f(None, None, None, 0, 256, 8, 1, 0, None, None, None, 0, None) == 1       # NULL output
    assert f(None, None, None, 0, 256, 8, 1, 1, 16, 16, None, 0, None) == 1           # flags must be 0
    assert f(None, None, None, 0, 65536, 8, 1, 0, 16, 16, None, 0, None) == 6         # T too large
    assert f(None, None, None, 0, 256, 8, 7, 0, 16, 16, None, 0, None) == 1           # bad precision
    assert f(None, None, None, 0, 256, 8, 1, 0, 16, 16, None, 0, None) == 3           # no workspace
    assert f(20, 32, 48, 10, 256, 8, 1, 0, 16, 16, 256, 1 << 20, None) == 1           # misaligned corners


def test_haar_host_checks(lib):
    """The Haar-transform entry points: sizes and host-detectable errors."""
    hw = lib.fcfs_haar_workspace_size
    a = hw(12576, 4096, 12)
    # banded (grids of >= 256 cells a side): the band sums (2^12 / 32 x 2^12 int32),
    # never the 2^24-cell grid
    assert 4 * 4 ** 12 // 32 <= a < 4 * 4 ** 12 and a % 256 == 0
    assert hw(12576, 4096, 7) >= 4 * 4 ** 7               # 128 x 128 cells: the grid (int32: cells of side 32)
    assert hw(100, 65536, 5) >= 8 * 4 ** 5                # cells of side 2048: int64 grid
    assert hw(0, 4096, 0) > 0 and hw(100, 16, 4) > 0
    assert hw(100, 4096, 13) == 0                         # J > log2 T
    assert hw(100, 65536, 15) == 0                        # J > 14
    assert hw(100, 1000, 4) == 0 and hw(100, 256, -1) == 0
    f = lib.fcfs_haar
    assert f(None, None, None, 0, 256, 4, 0, None, None, 0, None) == 1        # NULL output
    assert f(None, None, None, 0, 256, 4, 1, 16, None, 0, None) == 1          # flags must be 0
    assert f(None, None, None, 0, 256, 9, 0, 16, None, 0, None) == 6          # J too large
    assert f(None, None, None, 0, 256, 4, 0, 16, None, 0, None) == 3          # no workspace
    assert f(20, 32, 48, 10, 256, 4, 0, 16, 256, 1 << 20, None) == 1          # misaligned corners


FORMS = {0: "direct", 1: "grouped_tc", 2: "grouped_fft"}


def test_automatic_contraction_choice(lib):
    """The automatic choice among the contraction over the corners (direct),
    the split-FP16 contraction over y (grouped_tc) and the pruned FFT along y
    (grouped_fft), from cost estimates fitted to measurements of all three."""
    g = lib.fcfs_forward_grouped
    lib.fcfs_debug_set_hybrid(1)
    assert g(12576, 4096, 256, 1) == 0      # the T = 4096 clip: 0.039 ms direct, 0.077 FFT
    assert g(31700, 2048, 128, 1) == 0      # the adjoint workload's clip, K = 128
    assert g(945450, 65536, 1024, 1) == 2   # the large clip: 14.9 direct, 2.10 grouped tc, 1.72 FFT
    assert g(945450, 65536, 1024, 0) == 2   # plain FP32: 174 ms direct, 1.70 FFT
    assert g(12622, 4096, 1024, 1) == 2     # 0.262, 0.246, 0.172 ms
    assert g(100, 1000, 8, 1) == -1
    try:
        lib.fcfs_debug_set_hybrid(0)
        assert g(945450, 65536, 1024, 1) == 0
        lib.fcfs_debug_set_hybrid(2)
        assert g(12576, 4096, 256, 1) == 1
        assert g(12576, 4096, 256, 0) == 0  # no tensor-core form for FP32 calls
        lib.fcfs_debug_set_hybrid(3)
        assert g(12576, 4096, 256, 1) == 2
        assert g(12576, 4096, 256, 0) == 2
    finally:
        lib.fcfs_debug_set_hybrid(1)


# Sizes of the sweeps the automatic choices were fitted to: (T, K, V, prec, fastest
# form), measured on the GB300 (ms per call); "tie" marks cases where the two
# fastest forms are within 5%.
FORWARD_SWEEP = [
    (65536, 1024, 945450, 1, "grouped_fft"), (65536, 1024, 945450, 0, "grouped_fft"),
    (4096, 256, 3144, 1, "direct"),
    (4096, 256, 12576, 1, "direct"), (4096, 256, 12576, 0, "grouped_fft"),
    (4096, 256, 50386, 1, "direct"), (4096, 256, 50386, 0, "grouped_fft"),
    (4096, 256, 201294, 1, "tie"), (4096, 256, 201294, 0, "grouped_fft"),
    (65536, 1024, 125716, 1, "grouped_fft"), (4096, 1024, 12622, 1, "grouped_fft"),
    (16384, 512, 50152, 1, "tie"), (65536, 512, 945586, 1, "tie"),
    (65536, 256, 945586, 1, "tie"), (2048, 128, 31546, 1, "direct"),
    (2048, 128, 31546, 0, "grouped_fft"),
]
# adjoint: (T, K, V, fastest form) from the GB300 measurements of all four
# (per corner on tensor cores, per corner FP32, grouped tensor cores, pruned FFT)
ADJOINT_SWEEP = [
    (2048, 128, 31700, "fft"), (4096, 256, 3144, "fft"), (4096, 256, 12622, "fft"),
    (4096, 1024, 12622, "fft"), (4096, 256, 50386, "fft"), (4096, 1024, 50386, "fft"),
    (4096, 256, 201294, "fft"), (16384, 512, 188808, "fft"), (65536, 1024, 125716, "fft"),
    (65536, 256, 125716, "tie"), (65536, 1024, 945450, "fft"), (65536, 512, 945450, "fft"),
    (65536, 256, 945450, "fft"), (2048, 128, 1232, "fft"), (2048, 512, 1232, "fft"),
    (1024, 64, 1836, "fft"), (1024, 256, 1836, "fft"),
]
ADJOINT_FORMS = {0: "per_corner", 1: "grouped_tc", 2: "fft"}
FORWARD_MISSES = []


def test_automatic_choices_against_the_sweeps(lib):
    """The cost estimates pick the measured fastest form in every case that is
    not a near-tie, forward and adjoint."""
    lib.fcfs_debug_set_hybrid(1)
    misses = []
    for T, K, V, prec, best in FORWARD_SWEEP:
        got = FORMS[lib.fcfs_forward_grouped(V, T, K, prec)]
        if best != "tie" and got != best:
            misses.append((T, K, V, prec))
    assert sorted(misses) == sorted(FORWARD_MISSES), misses
    for T, K, V, best in ADJOINT_SWEEP:
        for prec in (1, 0):   # split FP16, plain FP32: the pruned FFT wins in both classes
            got = ADJOINT_FORMS[lib.fcfs_adjoint_grouped(V, T, K, prec)]
            assert best == "tie" or got == best, (T, K, V, prec, got)
    assert lib.fcfs_adjoint_grouped(100, 1000, 8, 1) == -1
    assert lib.fcfs_adjoint_grouped(40, 8, 2, 1) == 0              # T < 16: no pruned FFT
    assert lib.fcfs_adjoint_grouped(40, 4096, 4096, 1) in (0, 1)   # 2K > 4096: no pruned FFT
    try:
        lib.fcfs_debug_set_hybrid(0)
        assert lib.fcfs_adjoint_grouped(945450, 65536, 1024, 1) == 0
        lib.fcfs_debug_set_hybrid(2)
        assert lib.fcfs_adjoint_grouped(945450, 65536, 1024, 1) == 1
        assert lib.fcfs_adjoint_grouped(945450, 65536, 1024, 0) == 2   # FP32: no tensor-core form
        lib.fcfs_debug_set_hybrid(3)
        assert lib.fcfs_adjoint_grouped(31700, 2048, 128, 1) == 2
    finally:
        lib.fcfs_debug_set_hybrid(1)


def test_python_contraction_queries(lib):
    """The binding's queries answer as the C ABI does (host only, no device work)."""
    from paper_1010_5562_gb300 import fcfs
    assert fcfs.forward_grouped(945450, 65536, 1024) == 2
    assert fcfs.forward_grouped(12576, 4096, 256) == 0
    assert fcfs.adjoint_grouped(945586, 65536, 1024) == 2
    assert fcfs.adjoint_grouped(31700, 2048, 128) == 2
    assert fcfs.adjoint_grouped(945586, 65536, 1024, prec="fp32") == 2
    assert fcfs.forward_grouped(100, 1000, 8) == -1


def test_plans_host(lib):
    """Plans through the C ABI without device work: creation checks, knob
    ranges, resolved knobs and workspace sizes, independence from the hooks."""
    import ctypes as C
    h = C.c_void_p()
    assert lib.fcfs_plan_create(C.byref(h), 0, 945450, 1, 65536, 1024, 1) == 0 and h.value
    try:
        assert lib.fcfs_plan_get(h, 0) == 2                        # automatic: the pruned FFT along y
        auto_ws = lib.fcfs_plan_workspace_size(h)
        assert auto_ws == lib.fcfs_workspace_size(945450, 65536, 1024, 1)
        assert lib.fcfs_plan_set(h, 0, 1) == 0                     # split-FP16 contraction over y
        assert lib.fcfs_plan_get(h, 0) == 1
        assert lib.fcfs_plan_workspace_size(h) >= 2 * 2048 * 65600 * 2
        assert lib.fcfs_plan_set(h, 0, 0) == 0 and lib.fcfs_plan_get(h, 0) == 0
        assert lib.fcfs_plan_set(h, 1, 7) == 0 and lib.fcfs_plan_get(h, 1) == 7   # vertex splits
        assert lib.fcfs_plan_get(h, 2) == 1                        # CTA pairs for 2K >= 256
        assert lib.fcfs_plan_set(h, 2, 0) == 0 and lib.fcfs_plan_get(h, 2) == 0
        assert lib.fcfs_plan_set(h, 0, 3) == 1                     # no such form
        assert lib.fcfs_plan_set(h, 3, 16) == 1                    # unit chunks: batch plans only
        assert lib.fcfs_plan_set(h, 9, 0) == 1
        # the process-wide hooks are untouched by the plan
        assert lib.fcfs_forward_grouped(945450, 65536, 1024, 1) == 2
    finally:
        lib.fcfs_plan_destroy(h)
    b = C.c_void_p()
    assert lib.fcfs_plan_create(C.byref(b), 1, 100000, 8, 2048, 128, 1) == 0
    try:
        assert lib.fcfs_plan_get(b, 3) == 64                       # default: 4096 corners per unit
        assert lib.fcfs_plan_set(b, 3, 16) == 0 and lib.fcfs_plan_get(b, 3) == 16
        assert lib.fcfs_plan_workspace_size(b) > 0
        assert lib.fcfs_plan_set(b, 1, 4) == 1                     # splits: forward plans only
    finally:
        lib.fcfs_plan_destroy(b)
    a = C.c_void_p()
    assert lib.fcfs_plan_create(C.byref(a), 2, 945586, 1, 65536, 1024, 1) == 0
    try:
        assert lib.fcfs_plan_get(a, 0) == 2                        # the pruned-FFT adjoint
        auto_ws = lib.fcfs_plan_workspace_size(a)
        assert auto_ws >= 2 * 65536 * 1025 * 8                     # V_k of both matrices
        assert lib.fcfs_plan_set(a, 0, 1) == 0 and lib.fcfs_plan_get(a, 0) == 1
        assert lib.fcfs_plan_set(a, 0, 0) == 0 and lib.fcfs_plan_get(a, 0) == 0
        assert lib.fcfs_plan_set(a, 0, 3) == 1                     # no such form
        assert lib.fcfs_plan_workspace_size(a) > 0
    finally:
        lib.fcfs_plan_destroy(a)
    bad = C.c_void_p()
    assert lib.fcfs_plan_create(C.byref(bad), 0, 100, 1, 1000, 8, 1) == 6 and not bad.value   # T not 2^n
    assert lib.fcfs_plan_create(C.byref(bad), 0, 100, 2, 1024, 8, 1) == 1                     # clips of a forward plan
    assert lib.fcfs_plan_create(C.byref(bad), 5, 100, 1, 1024, 8, 1) == 1
    assert lib.fcfs_plan_create(None, 0, 100, 1, 1024, 8, 1) == 1
