"""Pruned-FFT adjoint on the GPU against the FP64 oracle.

The adjoint's sums over the grouped coordinate b (y for gx, x for gy) run as one
input-pruned FFT of length T per frequency k (P FFTs of length L >= 2K), and
each corner takes one dot of K + 1 terms (fcfs_adjoint_fft.cu).  Error measure:
max_v |g_gpu - g_oracle| / max_v |g_oracle|.  FP32 arithmetic throughout (both
precision classes take the same kernels); the bound is the plain-FP32 target
1e-6, measured 1.2e-7 .. 5.3e-7 on the small clips, 4.0e-7 on workload 4 and
3.6e-7 .. 4.7e-7 on sampled corners of the T = 65536 clip.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import clip_from_rings, config4_target, config_clip, make_clip, rect_ring

pytestmark = pytest.mark.gpu
TOL = 1e-6
FFT_FORM = 3   # fcfs_debug_set_hybrid: force the pruned-FFT form


@pytest.fixture(scope="module")
def fc():
    from paper_1010_5562_gb300 import build as B
    B.build()
    from paper_1010_5562_gb300 import fcfs
    assert torch.cuda.is_available()
    return fcfs


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def cot(K, seed):
    rng = np.random.default_rng(seed)
    W = 2 * K + 1
    G = rng.standard_normal((W, W)) + 1j * rng.standard_normal((W, W))
    return G.astype(np.complex64).astype(np.complex128)


def grad(fc, clip, K, G, mode=FFT_FORM, prec="fp32"):
    fc.set_hybrid(mode)   # the adjoint sizes its workspace inside the call
    try:
        x, y, s = dev(clip.x), dev(clip.y), dev(clip.s)
        dF = torch.from_numpy(G.astype(np.complex64)).cuda()
        gx, gy = fc.adjoint(x, y, s, clip.T, K, dF, prec=prec)
        torch.cuda.synchronize()
        return gx.cpu().numpy().astype(np.float64), gy.cpu().numpy().astype(np.float64)
    finally:
        fc.set_hybrid(1)


def check(fc, clip, K, G, tol=TOL, prec="fp32"):
    gx, gy = grad(fc, clip, K, G, prec=prec)
    rx, ry = oracle.vertex_gradient(clip.x, clip.y, clip.s, clip.T, K, G)
    ex, ey = rel(gx, rx), rel(gy, ry)
    assert ex < tol and ey < tol, (clip.T, K, ex, ey)
    return gx, gy


@pytest.mark.parametrize("prec", ["fp32", "split_f16"])
@pytest.mark.parametrize("K", [1, 7, 64, 129, 200])
def test_fft_adjoint_random_cotangent(fc, K, prec):
    """T = 512: K = 1 (L = 2, P = 256 residues, 2048 per buffer), 64 (L = 128),
    129 (L = 512 > 2K + 1), 200 (L = T, one residue); the form is the same for
    both precision classes."""
    clip = make_clip(512, 30, 900 + K, smin=6, smax=40)
    check(fc, clip, K, cot(K, 100 + K), prec=prec)


@pytest.mark.parametrize("K", [4, 8])
def test_fft_adjoint_tiny_period(fc, K):
    """T = 16, the smallest period of the form: one dot tile per matrix; K = 8
    gives L = T (P = 1) and l = +-8 sharing the residue 8."""
    clip = clip_from_rings(16, [rect_ring(1, 2, 5, 9), rect_ring(9, 0, 16, 4)])
    check(fc, clip, K, cot(K, 16 + K))


def test_fft_adjoint_border_corners(fc):
    """Corners at x = T and y = T: their V_k(T) is V_k(0) + lin_k T (the
    periodic part repeats, the linear side term does not)."""
    T = 1024
    clip = clip_from_rings(T, [rect_ring(T - 10, T - 10, T, T), rect_ring(0, 5, 30, T), rect_ring(500, 0, T, 3)])
    assert int(np.sum(clip.x == T)) > 0 and int(np.sum(clip.y == T)) > 0
    check(fc, clip, 64, cot(64, 3))


def test_fft_adjoint_unsupported_sizes_fall_back(fc):
    """T < 16 or L > T: forcing the form leaves the automatic choice, still exact."""
    clip = clip_from_rings(4, [rect_ring(1, 1, 2, 3)])
    check(fc, clip, 20, cot(20, 4), tol=1e-5)
    assert fc.adjoint_grouped(clip.V, 4, 20) != 2


def test_fft_adjoint_config4_pupil_loss(fc):
    """Workload 4 (T = 2048, ~31.7k corners, K = 128): the pupil-filtered loss
    gradient, corners and edges, against the oracle; the automatic form."""
    clip, K = config_clip(4)
    tgt, _ = config4_target(clip)
    T = clip.T
    F = oracle.block(clip.x, clip.y, clip.s, T, K)
    Ft = oracle.block(tgt.x, tgt.y, tgt.s, T, K)
    _, G = oracle.pupil_loss(F, Ft, K)
    assert fc.adjoint_grouped(clip.V, T, K, prec="fp32") == 2
    gx, gy = grad(fc, clip, K, G, mode=1)
    rx, ry = oracle.vertex_gradient(clip.x, clip.y, clip.s, T, K, G)
    assert rel(gx, rx) < TOL and rel(gy, ry) < TOL, (rel(gx, rx), rel(gy, ry))
    gE = fc.edge_chain(dev(gx.astype(np.float32)), dev(gy.astype(np.float32)), dev(clip.ev0), dev(clip.ev1),
                       dev(clip.eaxis))
    rE = oracle.edge_gradient(rx, ry, clip.ev0, clip.ev1, clip.eaxis)
    # an edge moves two corners of opposite sign: its derivative is a difference
    # of two corner derivatives, so its error is bounded on the corners' scale
    dE = np.max(np.abs(gE.cpu().numpy().astype(np.float64) - rE))
    assert dE / max(np.max(np.abs(rx)), np.max(np.abs(ry))) < 2 * TOL, dE
    assert rel(gE.cpu().numpy().astype(np.float64), rE) < 1e-5


def test_fft_adjoint_config5_sampled(fc):
    """Workload 5 (T = 65536, ~945k corners, K = 1024), a seeded cotangent over
    the whole block: 64 sampled corners against the oracle (each corner's
    derivative depends only on that corner)."""
    clip, K = config_clip(5)
    G = cot(K, 5)
    gx, gy = grad(fc, clip, K, G, mode=1)
    rng = np.random.default_rng(55)
    idx = np.sort(rng.choice(clip.V, 64, replace=False))
    rx, ry = oracle.vertex_gradient(clip.x[idx], clip.y[idx], clip.s[idx], clip.T, K, G)
    ex, ey = rel(gx[idx], rx), rel(gy[idx], ry)
    assert ex < TOL and ey < TOL, (ex, ey)


def test_fft_adjoint_dense_groups(fc):
    """10000 rectangles 5 wide on y in [0, 50]: 20000 corners at y = 0 and at
    y = 50 fall into single dot tiles, which take their corners in 40 passes
    over the tile's values.  Sampled corners against the oracle."""
    T, K = 65536, 128
    clip = clip_from_rings(T, [rect_ring(6 * i, 0, 6 * i + 5, 50) for i in range(10000)])
    G = cot(K, 9)
    gx, gy = grad(fc, clip, K, G)
    rng = np.random.default_rng(9)
    idx = np.sort(rng.choice(clip.V, 64, replace=False))
    rx, ry = oracle.vertex_gradient(clip.x[idx], clip.y[idx], clip.s[idx], T, K, G)
    assert rel(gx[idx], rx) < 1e-5 and rel(gy[idx], ry) < 1e-5, (rel(gx[idx], rx), rel(gy[idx], ry))


def test_fft_adjoint_deterministic_and_forms_agree(fc):
    """Each corner's sum runs in a fixed order: repeated calls are bit-identical.
    The form agrees with the tensor-core forms (grouped and per corner)."""
    clip = make_clip(2048, 400, 77, smin=8, smax=120)
    K = 96
    G = cot(K, 77)
    a = grad(fc, clip, K, G)
    b = grad(fc, clip, K, G)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for mode in (0, 2):
        c = grad(fc, clip, K, G, mode=mode, prec="split_f16")
        assert rel(a[0], c[0]) < 1e-5 and rel(a[1], c[1]) < 1e-5


def test_fft_adjoint_launches(fc):
    """prep, grouping (count, scan, scatter), the tables (with the transposed
    cotangent), the FFTs, the dots."""
    clip, K = config_clip(4)
    x, y, s = dev(clip.x), dev(clip.y), dev(clip.s)
    dF = torch.zeros((2 * K + 1, 2 * K + 1), dtype=torch.complex64, device="cuda")
    fc.set_hybrid(FFT_FORM)
    try:
        n0 = fc.launch_count()
        fc.adjoint(x, y, s, clip.T, K, dF, prec="split_f16")
        assert fc.launch_count() - n0 == 7
    finally:
        fc.set_hybrid(1)
