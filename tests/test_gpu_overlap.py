"""Stages of a call on a second stream (the axis lines beside the grouped
forward's H and FFT, the adjoint's grouping beside its FFTs): the results do not
depend on it, and a call with its fork and join captures into a CUDA graph."""
import numpy as np
import pytest
import torch

import oracle
from synth import make_clip

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    from paper_1010_5562_gb300 import build as B
    B.build()
    from paper_1010_5562_gb300 import fcfs
    assert torch.cuda.is_available()
    return fcfs


@pytest.fixture(scope="module")
def case():
    # T >= 16384: the axis lines take the FFT path; the grouped FFT forms forced
    clip = make_clip(16384, 3000, 4242, smin=10, smax=200)
    K = 256
    rng = np.random.default_rng(42)
    W = 2 * K + 1
    G = (rng.standard_normal((W, W)) + 1j * rng.standard_normal((W, W))).astype(np.complex64)
    return clip, K, G


def run(fc, clip, K, G, overlap, stream=None):
    x, y, s = (torch.from_numpy(a).cuda() for a in (clip.x, clip.y, clip.s))
    dF = torch.from_numpy(G).cuda()
    fc.set_overlap(overlap)
    fc.set_hybrid(3)
    try:
        F, area = fc.forward(x, y, s, clip.T, K, prec="split_f16")
        gx, gy = fc.adjoint(x, y, s, clip.T, K, dF, prec="split_f16")
        torch.cuda.synchronize()
    finally:
        fc.set_hybrid(1)
        fc.set_overlap(True)
    return F.cpu().numpy(), int(area), gx.cpu().numpy(), gy.cpu().numpy()


def test_overlap_gives_the_same_results(fc, case):
    clip, K, G = case
    a = run(fc, clip, K, G, True)
    b = run(fc, clip, K, G, False)
    assert np.array_equal(a[0], b[0]) and a[1] == b[1]
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
    A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    assert a[1] == A
    pick = np.array([0, 1, -1, 5, -77, K, -K])
    Fo = oracle.block_entries(clip.x, clip.y, clip.s, clip.T, pick, pick)
    assert np.max(np.abs(a[0][np.ix_(pick + K, pick + K)] - Fo)) / A <= 1e-6


def test_overlapped_calls_capture_into_a_graph(fc, case):
    """Forward and adjoint (each forking a side stream and joining it back)
    captured on a side stream of torch, replayed, against the eager calls."""
    clip, K, G = case
    ref = run(fc, clip, K, G, True)
    x, y, s = (torch.from_numpy(a).cuda() for a in (clip.x, clip.y, clip.s))
    dF = torch.from_numpy(G).cuda()
    W = 2 * K + 1
    F = torch.empty((W, W), dtype=torch.complex64, device="cuda")
    area = torch.empty(1, dtype=torch.int64, device="cuda")
    gx = torch.empty(clip.V, dtype=torch.float32, device="cuda")
    gy = torch.empty_like(gx)
    fc.set_hybrid(3)
    try:
        wsf = fc.alloc_workspace(fc.workspace_size(clip.V, clip.T, K, "split_f16"), "cuda")
        wsa = fc.alloc_workspace(fc._lib.load().fcfs_adjoint_workspace_size(clip.V, clip.T, K, 1), "cuda")
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            # warm-up outside the capture (tables, side stream creation)
            fc.forward(x, y, s, clip.T, K, prec="split_f16", out=F, area_out=area, workspace=wsf, stream=st)
            fc.adjoint(x, y, s, clip.T, K, dF, prec="split_f16", gx=gx, gy=gy, workspace=wsa, stream=st)
        st.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            fc.forward(x, y, s, clip.T, K, prec="split_f16", out=F, area_out=area, workspace=wsf, stream=st)
            fc.adjoint(x, y, s, clip.T, K, dF, prec="split_f16", gx=gx, gy=gy, workspace=wsa, stream=st)
        F.zero_()
        gx.zero_()
        gy.zero_()
        g.replay()
        torch.cuda.synchronize()
    finally:
        fc.set_hybrid(1)
    assert np.array_equal(F.cpu().numpy(), ref[0]) and int(area) == ref[1]
    assert np.array_equal(gx.cpu().numpy(), ref[2]) and np.array_equal(gy.cpu().numpy(), ref[3])
