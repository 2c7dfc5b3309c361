"""Grouped forward with the pruned FFT along y against the FP64 oracle.

The corners are grouped by y, H is summed per row from x-sorted corner pairs
(FP32), and the off-axis block comes from P FFTs of length L per frequency k
(T = P L) with the output pruned to |l| <= K (Step 4's sparse-image DFT with
output pruning).  The whole path is FP32 on CUDA cores, so it is held to the
plain-FP32 bound max|dF|/area <= 1e-6 whatever precision the call names; the
area and F(0,0) are exact.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import config_clip, make_clip, clip_from_rings, rect_ring

pytestmark = pytest.mark.gpu

TOL = 1e-6
FFT = 3   # fcfs_debug_set_hybrid: force the FFT form


@pytest.fixture(scope="module")
def fc():
    from paper_1010_5562_gb300 import build as B
    B.build()
    from paper_1010_5562_gb300 import fcfs
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    fcfs.set_hybrid(1)
    return fcfs


def run(fc, clip, K, mode, prec="split_f16"):
    x, y, s = (torch.from_numpy(a).cuda() for a in (clip.x, clip.y, clip.s))
    fc.set_hybrid(mode)
    try:
        ws = fc.alloc_workspace(fc.workspace_size(clip.V, clip.T, K, prec), x.device)
        out = torch.full((2 * K + 1, 2 * K + 1), float("nan"), dtype=torch.complex64, device="cuda")
        F, a = fc.forward(x, y, s, clip.T, K, prec=prec, out=out, workspace=ws)
        torch.cuda.synchronize()
        assert fc.get_status(ws) == "FCFS_OK"
    finally:
        fc.set_hybrid(1)
    return F.cpu().numpy().astype(np.complex128), int(a)


CASES = [
    # (T, polygons, seed, smin, smax, K)
    (256, 40, 21, 4, 30, 32),          # L = 64, P = 4
    (256, 40, 22, 4, 30, 128),         # L = T: one FFT per k, every l kept
    (1024, 300, 23, 6, 40, 200),       # K not a power of two
    (2048, 600, 24, 8, 60, 129),       # 2K + 1 > 256 outputs
    (8192, 900, 25, 20, 200, 100),     # quarter-wave tables, L = T / 16
    (65536, 1000, 26, 20, 2000, 130),  # sparse y, P = 16
    (16, 4, 27, 1, 3, 40),             # tiny period, K > T
    (64, 6, 28, 2, 10, 7),             # one item of 64 rows
    (32, 3, 29, 2, 8, 5),              # period below one item: row T folded in the same item
]


@pytest.mark.parametrize("prec", ["fp32", "split_f16"])
@pytest.mark.parametrize("case", CASES, ids=[f"T{c[0]}_K{c[5]}" for c in CASES])
def test_fft_matches_oracle(fc, case, prec):
    T, n, seed, smin, smax, K = case
    clip = make_clip(T, n, seed, smin=smin, smax=smax)
    F, area = run(fc, clip, K, FFT, prec)
    A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    assert area == A
    assert np.all(np.isfinite(F)), "block not fully written"
    assert F[K, K] == complex(np.float32(A), 0.0)
    Fo = oracle.block(clip.x, clip.y, clip.s, clip.T, K)
    err = np.max(np.abs(F - Fo)) / A
    assert err <= TOL, err


def test_fft_bench_clip_deterministic(fc):
    """Workload 2 (T = 4096, V = 12576, K = 256): the whole block within the
    FP32 bound; repeated calls are bit-identical (rows are summed in x order
    whatever order the grouping left the corners in); the axis lines are the
    same exact integer sums as on the direct path."""
    clip, K = config_clip(2)
    F1, a1 = run(fc, clip, K, FFT)
    F2, a2 = run(fc, clip, K, FFT)
    Fd, ad = run(fc, clip, K, 0)
    A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    assert a1 == a2 == ad == A
    assert np.array_equal(F1, F2)
    np.testing.assert_array_equal(F1[K, :], Fd[K, :])
    np.testing.assert_array_equal(F1[:, K], Fd[:, K])
    Fo = oracle.block(clip.x, clip.y, clip.s, clip.T, K)
    assert np.max(np.abs(F1 - Fo)) / A <= TOL


def test_fft_dense_rows_fallback(fc):
    """10000 rectangles 5 wide on y in [0, 50]: two rows of 20000 corners, more
    than one item sorts in shared memory, so those items take the exact
    fixed-point sums.  The clip is ill-conditioned for any FP32 evaluation of
    the y stage: its two rows carry H[k, 50] = -H[k, 0] exactly, and at low l
    G = H[k, 0] (1 - e^{-j 2 pi 50 l / T}) is ~200x smaller than either term,
    so the FFT's roundings of the two terms (relative ~1e-7 of |H|) reach ~2e-6
    of this clip's small area (the direct paths: ~5e-5).  Held to 5e-6 on
    sampled coefficients."""
    T, K = 65536, 128
    clip = clip_from_rings(T, [rect_ring(6 * i, 0, 6 * i + 5, 50) for i in range(10000)])
    F, a = run(fc, clip, K, FFT)
    A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    assert a == A
    assert np.all(np.isfinite(F))
    rng = np.random.default_rng(4)
    pick = np.unique(np.concatenate([[0, 1, -1, K, -K], rng.integers(-K, K + 1, 24)]))
    Fo = oracle.block_entries(clip.x, clip.y, clip.s, clip.T, pick, pick)
    assert np.max(np.abs(F[np.ix_(pick + K, pick + K)] - Fo)) / A <= 5e-6


@pytest.mark.parametrize("mode,tol", [(FFT, TOL), (2, 1e-5)], ids=["grouped_fft", "grouped_tc"])
def test_wide_rows_sorted_whole(fc, mode, tol):
    """Rows of more than 128 corners (150 rectangles side by side on y in
    [100, 164): 300 corners on rows 100 and 164) take the bitonic sort of their
    whole item; the other items, with rows of a few corners, the sort by rank
    within the rows.  Both H formats (polyphase FP32, FP16 rows) against the
    oracle over the whole block."""
    T, K = 4096, 96
    rings = [rect_ring(20 + 25 * i, 100, 40 + 25 * i, 164) for i in range(150)]
    base = make_clip(T, 300, 31, smin=8, smax=60)
    for m in range(base.n_polys):
        xs, ys = base.ring(m)
        if ys.min() > 300:   # keep the random polygons clear of the wide rows
            rings.append((xs, ys))
    clip = clip_from_rings(T, rings)
    F, a = run(fc, clip, K, mode)
    A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    assert a == A
    Fo = oracle.block(clip.x, clip.y, clip.s, clip.T, K)
    assert np.max(np.abs(F - Fo)) / A <= tol


def test_fft_rows_on_the_clip_border(fc):
    """Corners on y = T (folded onto row 0) and on x = T and x = 0."""
    T, K = 512, 60
    rings = [rect_ring(0, 500, 30, 512), rect_ring(480, 0, 512, 40), rect_ring(100, 0, 140, 512),
             rect_ring(200, 200, 260, 300)]
    clip = clip_from_rings(T, rings)
    F, a = run(fc, clip, K, FFT)
    A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    assert a == A
    Fo = oracle.block(clip.x, clip.y, clip.s, clip.T, K)
    assert np.max(np.abs(F - Fo)) / A <= TOL


@pytest.mark.parametrize("prec", ["fp32", "split_f16"])
def test_config5_fft_sampled(fc, prec):
    """Workload 5 (T = 65536, V = 945450, K = 1024), the automatic choice: 12
    full rows of the 2049 x 2049 block against the oracle."""
    clip, K = config_clip(5)
    assert fc.forward_grouped(clip.V, clip.T, K, prec=prec) == 2
    F, a = run(fc, clip, K, 1, prec)
    A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    assert a == A
    assert np.all(np.isfinite(F))
    rows = np.array([-K, -1023, -517, -64, -1, 0, 1, 2, 3, 100, 511, K])
    Fo = oracle.block_entries(clip.x, clip.y, clip.s, clip.T, rows, oracle.freqs(K))
    err = np.max(np.abs(F[rows + K, :] - Fo)) / A
    assert err <= TOL, err


def test_fft_launches(fc):
    """prep, count, scan, scatter, H, FFT, binning, axis DFT, axis output."""
    clip, K = config_clip(2)
    x, y, s = (torch.from_numpy(a).cuda() for a in (clip.x, clip.y, clip.s))
    fc.set_hybrid(FFT)
    try:
        ws = fc.alloc_workspace(fc.workspace_size(clip.V, clip.T, K, "fp32"), x.device)
        n0 = fc.launch_count()
        fc.forward(x, y, s, clip.T, K, prec="fp32", workspace=ws)
        assert fc.launch_count() - n0 == 9
    finally:
        fc.set_hybrid(1)
