"""Row-binned contraction (corners grouped by y, the off-axis block contracted
over the T + 1 values of y) against the FP64 oracle and the direct contraction.

It is taken automatically for single-clip split-FP16 calls on CTA pairs when
a cost estimate of the two contractions favours it (the large-clip workload
among others); here it is also forced on smaller clips.  Bounds as for the split-FP16 path: max|dF|/area <= 1e-5, the
area and F(0,0) exact.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import config_clip, make_clip, clip_from_rings, rect_ring

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def fc():
    from paper_1010_5562_gb300 import build as B
    B.build()
    from paper_1010_5562_gb300 import fcfs
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    fcfs.set_splits(0)
    fcfs.set_hybrid(1)
    return fcfs


def to_dev(clip):
    return (torch.from_numpy(clip.x).cuda(), torch.from_numpy(clip.y).cuda(),
            torch.from_numpy(clip.s).cuda())


def run(fc, clip, K, mode, splits=0):
    """One split-FP16 forward with the grouping mode set (workspace sized after it)."""
    x, y, s = to_dev(clip)
    fc.set_hybrid(mode)
    fc.set_splits(splits)
    try:
        ws = fc.alloc_workspace(fc.workspace_size(clip.V, clip.T, K, "split_f16"), x.device)
        out = torch.full((2 * K + 1, 2 * K + 1), float("nan"), dtype=torch.complex64, device="cuda")
        F, a = fc.forward(x, y, s, clip.T, K, prec="split_f16", out=out, workspace=ws)
        torch.cuda.synchronize()
        assert fc.get_status(ws) == "FCFS_OK"
    finally:
        fc.set_hybrid(1)
        fc.set_splits(0)
    return F.cpu().numpy().astype(np.complex128), int(a)


CASES = [
    # (T, polygons, seed, smin, smax, K): pair tiles need 2K >= 256
    (256, 40, 11, 4, 30, 128),        # y range of 5 chunks, one pair tile
    (1024, 300, 12, 6, 40, 200),      # 2K = 400: ragged pair tiles
    (2048, 600, 13, 8, 60, 129),      # 2K = 258: a 2-row tail tile
    (8192, 900, 14, 20, 200, 128),    # quarter-wave tables from T = 8192 on (tensor-core plans)
    (65536, 1000, 15, 20, 2000, 130), # quarter-wave tables, sparse y
    (16, 4, 16, 1, 3, 128),           # tiny period: one y chunk, K >> T
]


@pytest.mark.parametrize("case", CASES, ids=[f"T{c[0]}_K{c[5]}" for c in CASES])
def test_hybrid_matches_oracle(fc, case):
    T, n, seed, smin, smax, K = case
    clip = make_clip(T, n, seed, smin=smin, smax=smax)
    Fg, area = run(fc, clip, K, mode=2)
    A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    assert area == A
    assert np.all(np.isfinite(Fg)), "block not fully written"
    assert Fg[K, K] == complex(np.float32(A), 0.0)
    Fo = oracle.block(clip.x, clip.y, clip.s, clip.T, K)
    err = np.max(np.abs(Fg - Fo)) / A
    assert err <= TOL, err


@pytest.mark.parametrize("splits", [0, 1, 3, 7])
def test_hybrid_against_direct_and_deterministic(fc, splits):
    """Workload 2 (T=4096, V=12576, K=256): grouped and direct contractions
    agree to FP32 rounding; H is an exact integer sum, so repeated grouped calls
    (whose corner order inside a y group is arbitrary) are bit-identical."""
    clip, K = config_clip(2)
    Fh1, a1 = run(fc, clip, K, mode=2, splits=splits)
    Fh2, a2 = run(fc, clip, K, mode=2, splits=splits)
    Fd, a0 = run(fc, clip, K, mode=0, splits=splits)
    A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    assert a1 == a2 == a0 == A
    assert np.array_equal(Fh1, Fh2)
    assert np.max(np.abs(Fh1 - Fd)) / A <= 2e-6
    np.testing.assert_array_equal(Fh1[K, :], Fd[K, :])   # axis lines: the same exact integer sums
    np.testing.assert_array_equal(Fh1[:, K], Fd[:, K])
    Fo = oracle.block(clip.x, clip.y, clip.s, clip.T, K)
    assert np.max(np.abs(Fh1 - Fo)) / A <= TOL


def test_hybrid_large_y_groups(fc):
    """10000 rectangles 5 wide and 50 high side by side on y in [0, 50]: the two
    y groups of 20000 corners take the per-y power-of-two scale of the FP16
    split (2^-1 on H, 2^1 on the generated operand).  The grouped contraction
    is within the split-FP16 bound of the oracle (sampled coefficients).

    Features 5 units wide at T = 65536 are hard for the direct contraction: the
    two corners of a horizontal edge differ in phase by 2 pi 5 k / T, and their
    FP16-split operands cancel inside the MMA to a few 1e-4 of their size, so
    its error is ~5e-5 of the area here.  The grouped path sums such corners
    exactly in fixed point first (~6e-7).  A wrong per-y scale would show as
    an O(1) difference between the two."""
    T, K = 65536, 128
    clip = clip_from_rings(T, [rect_ring(6 * i, 0, 6 * i + 5, 50) for i in range(10000)])
    Fh, ah = run(fc, clip, K, mode=2)
    Fd, ad = run(fc, clip, K, mode=0)
    A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    assert ah == ad == A == 10000 * 5 * 50
    assert np.all(np.isfinite(Fh))
    rng = np.random.default_rng(3)
    pick = np.unique(np.concatenate([[0, 1, -1, K, -K], rng.integers(-K, K + 1, 24)]))
    Fo = oracle.block_entries(clip.x, clip.y, clip.s, clip.T, pick, pick)
    err_h = np.max(np.abs(Fh[np.ix_(pick + K, pick + K)] - Fo)) / A
    err_d = np.max(np.abs(Fd[np.ix_(pick + K, pick + K)] - Fo)) / A
    diff = np.max(np.abs(Fh - Fd)) / A
    assert err_h <= TOL, (err_h, err_d, diff)
    assert diff <= err_d + err_h + 1e-5, (err_h, err_d, diff)


def test_hybrid_launches(fc):
    """Grouped: prep, count, scan, scatter, H, contraction, binning, axis DFT,
    reduce.  Workload 4 (K = 128) stays direct automatically: below K = 256 the
    grouped form gains little and adds launches."""
    clip, K = config_clip(4)
    x, y, s = to_dev(clip)
    ws = fc.alloc_workspace(fc.workspace_size(clip.V, clip.T, K, "split_f16"), x.device)
    n0 = fc.launch_count()
    fc.forward(x, y, s, clip.T, K, prec="split_f16", workspace=ws)
    assert fc.launch_count() - n0 in (2, 4)   # fused, or separate axis and reduce kernels
    fc.set_hybrid(2)
    try:
        ws2 = fc.alloc_workspace(fc.workspace_size(clip.V, clip.T, K, "split_f16"), x.device)
        n0 = fc.launch_count()
        fc.forward(x, y, s, clip.T, K, prec="split_f16", workspace=ws2)
        assert fc.launch_count() - n0 == 9
    finally:
        fc.set_hybrid(1)
