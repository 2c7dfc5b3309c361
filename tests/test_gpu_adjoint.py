"""Adjoint (corner and edge derivatives) on the GPU against the FP64 oracle.

Error measure: max_v |g_gpu - g_oracle| / max_v |g_oracle| over all corners (and
over all edges for the chained derivative).  The FP32 adjoint sums (2K+2)-term
FP32 dot products per row and a compensated sum over row tiles; the bound 1e-5
leaves a factor of ~10 over the measured error.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import config_clip, config4_target, make_clip

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def fc():
    from paper_1010_5562_gb300 import build as B
    B.build()
    from paper_1010_5562_gb300 import fcfs
    assert torch.cuda.is_available()
    return fcfs


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_grad(fc, clip, K, G, prec="fp32"):
    x, y, s = dev(clip.x), dev(clip.y), dev(clip.s)
    dF = torch.from_numpy(G.astype(np.complex64)).cuda()
    gx, gy = fc.adjoint(x, y, s, clip.T, K, dF, prec=prec)
    torch.cuda.synchronize()
    return gx.cpu().numpy().astype(np.float64), gy.cpu().numpy().astype(np.float64)


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


PRECS = ["fp32", "split_f16"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("K", [1, 7, 40, 64, 100, 200])
def test_random_cotangent(fc, K, prec):
    """The split-FP16 path runs the contraction on the tensor cores (row tiles
    of 128 coefficient rows; K = 64, 100, 200 give full, partial and one-row
    last tiles); 30 polygons leave a partial tile of 256 corners."""
    clip = make_clip(512, 30, 700 + K, smin=6, smax=40)
    rng = np.random.default_rng(K)
    W = 2 * K + 1
    G = rng.standard_normal((W, W)) + 1j * rng.standard_normal((W, W))
    gx, gy = gpu_grad(fc, clip, K, G, prec)
    rx, ry = oracle.vertex_gradient(clip.x, clip.y, clip.s, clip.T, K, G)
    assert rel(gx, rx) < TOL and rel(gy, ry) < TOL, (rel(gx, rx), rel(gy, ry))


@pytest.mark.parametrize("prec", PRECS)
def test_config4_pupil_loss_gradient(fc, prec):
    """Workload 4: T=2048, ~31.7k corners, K=128, L = sum over k^2+l^2 <= K^2 of
    |F - F_target|^2 with the target's edges jittered by U{-2..2}."""
    clip, K = config_clip(4)
    tgt, _ = config4_target(clip)
    T = clip.T
    F = oracle.block(clip.x, clip.y, clip.s, T, K)
    Ft = oracle.block(tgt.x, tgt.y, tgt.s, T, K)
    _, G = oracle.pupil_loss(F, Ft, K)
    gx, gy = gpu_grad(fc, clip, K, G, prec)
    rx, ry = oracle.vertex_gradient(clip.x, clip.y, clip.s, T, K, G)
    assert rel(gx, rx) < TOL and rel(gy, ry) < TOL, (rel(gx, rx), rel(gy, ry))
    # chained to edge positions on the GPU
    gE = fc.edge_chain(dev(gx.astype(np.float32)), dev(gy.astype(np.float32)), dev(clip.ev0), dev(clip.ev1),
                       dev(clip.eaxis))
    rE = oracle.edge_gradient(rx, ry, clip.ev0, clip.ev1, clip.eaxis)
    assert rel(gE.cpu().numpy().astype(np.float64), rE) < TOL


def test_autograd_edge_gradient_and_finite_differences(fc):
    """Edge gradients through torch.autograd match the oracle, and a +-1 move of
    an edge changes the GPU loss by the predicted amount."""
    clip, K = config_clip(4, scale=0.05)
    tgt, _ = config4_target(clip)
    T = clip.T
    ev0, ev1, eaxis, s = dev(clip.ev0), dev(clip.ev1), dev(clip.eaxis), dev(clip.s)
    mask = torch.from_numpy(oracle.pupil_mask(K)).cuda()
    Ft, _ = fc.forward(dev(tgt.x), dev(tgt.y), s, T, K, prec="fp32")
    pos = torch.from_numpy(clip.edge_positions().astype(np.float32)).cuda().requires_grad_(True)
    F = fc.block(pos, ev0, ev1, eaxis, s, T, K)
    L = ((F - Ft).abs() ** 2 * mask).sum()
    L.backward()
    gE = pos.grad.cpu().numpy().astype(np.float64)
    Fo = oracle.block(clip.x, clip.y, clip.s, T, K)
    Fto = oracle.block(tgt.x, tgt.y, tgt.s, T, K)
    _, G = oracle.pupil_loss(Fo, Fto, K)
    rx, ry = oracle.vertex_gradient(clip.x, clip.y, clip.s, T, K, G)
    rE = oracle.edge_gradient(rx, ry, clip.ev0, clip.ev1, clip.eaxis)
    # includes the FP32 forward error of F in the cotangent (measured 1.4e-6; 2.5e-6
    # with the split-FP16 forward)
    assert rel(gE, rE) < 1e-5

    def loss_at(p):
        with torch.no_grad():
            Fp = fc.block(p, ev0, ev1, eaxis, s, T, K)
            return float(((Fp - Ft).abs().double() ** 2 * mask).sum())

    base = pos.detach().clone()
    worst = 0.0
    for e in range(0, clip.ev0.shape[0], max(1, clip.ev0.shape[0] // 12)):
        pp, pm = base.clone(), base.clone()
        pp[e] += 1.0
        pm[e] -= 1.0
        fd = (loss_at(pp) - loss_at(pm)) / 2.0
        worst = max(worst, abs(fd - gE[e]) / np.max(np.abs(gE)))
    # a unit central difference of a smooth function of the edge position;
    # its truncation error (third derivative) bounds the agreement
    assert worst < 2e-2, worst


def test_edge_chain_empty_and_direct(fc):
    gx = torch.tensor([1.0, 2.0, 3.0, 4.0], device="cuda")
    gy = torch.tensor([10.0, 20.0, 30.0, 40.0], device="cuda")
    ev0 = torch.tensor([0, 1, 2, 3], dtype=torch.int32, device="cuda")
    ev1 = torch.tensor([1, 2, 3, 0], dtype=torch.int32, device="cuda")
    ax = torch.tensor([1, 0, 1, 0], dtype=torch.int8, device="cuda")
    gE = fc.edge_chain(gx, gy, ev0, ev1, ax).cpu().tolist()
    assert gE == [30.0, 5.0, 70.0, 5.0]


@pytest.mark.parametrize("prec", PRECS)
def test_config5_adjoint_sampled(fc, prec):
    """Workload 5 (T=65536, ~945k corners, K=1024): the FP32 adjoint of a seeded
    random cotangent on the full block, checked on 48 sampled corners (the
    oracle's derivative of each corner depends only on that corner)."""
    clip, K = config_clip(5)
    W = 2 * K + 1
    rng = np.random.default_rng(5)
    G = (rng.standard_normal((W, W)) + 1j * rng.standard_normal((W, W))).astype(np.complex64)
    gx, gy = gpu_grad(fc, clip, K, G.astype(np.complex128), prec)
    idx = np.sort(rng.choice(clip.V, 48, replace=False))
    rx, ry = oracle.vertex_gradient(clip.x[idx], clip.y[idx], clip.s[idx], clip.T, K, G.astype(np.complex128))
    ex, ey = rel(gx[idx], rx), rel(gy[idx], ry)
    assert ex < 1e-5 and ey < 1e-5, (ex, ey)


def grad_mode(fc, clip, K, G, mode):
    fc.set_hybrid(mode)   # the adjoint sizes its workspace inside the call
    try:
        return gpu_grad(fc, clip, K, G, "split_f16")
    finally:
        fc.set_hybrid(1)


@pytest.mark.parametrize("K", [1, 7, 64, 129, 200])
def test_grouped_adjoint_random_cotangent(fc, K):
    """Corners grouped by b (y for gx, x for gy): the MMA's M dimension runs over
    the T + 1 values of b and the epilogue over each value's corners.  Forced on
    a small clip: against the oracle and against the per-corner contraction."""
    clip = make_clip(512, 30, 900 + K, smin=6, smax=40)
    rng = np.random.default_rng(100 + K)
    W = 2 * K + 1
    G = rng.standard_normal((W, W)) + 1j * rng.standard_normal((W, W))
    gx, gy = grad_mode(fc, clip, K, G, 2)
    gx0, gy0 = grad_mode(fc, clip, K, G, 0)
    rx, ry = oracle.vertex_gradient(clip.x, clip.y, clip.s, clip.T, K, G)
    assert rel(gx, rx) < TOL and rel(gy, ry) < TOL, (rel(gx, rx), rel(gy, ry))
    assert rel(gx, gx0) < 2e-6 and rel(gy, gy0) < 2e-6, (rel(gx, gx0), rel(gy, gy0))


def test_grouped_adjoint_tiny_period(fc):
    """T = 4 (five values of b, a one-level sincos table) and T = 16, forced grouped."""
    from synth import clip_from_rings, rect_ring
    for T, rings in ((4, [rect_ring(1, 1, 2, 3)]), (16, [rect_ring(1, 2, 5, 9), rect_ring(9, 0, 16, 4)])):
        clip = clip_from_rings(T, rings)
        K = 20
        rng = np.random.default_rng(T)
        W = 2 * K + 1
        G = rng.standard_normal((W, W)) + 1j * rng.standard_normal((W, W))
        gx, gy = grad_mode(fc, clip, K, G, 2)
        rx, ry = oracle.vertex_gradient(clip.x, clip.y, clip.s, clip.T, K, G)
        assert rel(gx, rx) < TOL and rel(gy, ry) < TOL, (T, rel(gx, rx), rel(gy, ry))


def test_grouped_adjoint_large_groups(fc):
    """10000 rectangles 5 wide on y in [0, 50]: the y groups of 20000 corners
    exceed the epilogue's staging (4096 corners), so the CTA of b in [0, 128)
    takes them in pieces.  Sampled corners against the oracle."""
    from synth import clip_from_rings, rect_ring
    T, K = 65536, 128
    clip = clip_from_rings(T, [rect_ring(6 * i, 0, 6 * i + 5, 50) for i in range(10000)])
    rng = np.random.default_rng(9)
    W = 2 * K + 1
    G = rng.standard_normal((W, W)) + 1j * rng.standard_normal((W, W))
    gx, gy = grad_mode(fc, clip, K, G, 1)   # automatic
    gx2, gy2 = grad_mode(fc, clip, K, G, 2)
    idx = np.sort(rng.choice(clip.V, 48, replace=False))
    rx, ry = oracle.vertex_gradient(clip.x[idx], clip.y[idx], clip.s[idx], T, K, G)
    for a, b in ((gx2[idx], rx), (gy2[idx], ry), (gx[idx], rx), (gy[idx], ry)):
        assert rel(a, b) < TOL, rel(a, b)


def test_grouped_adjoint_launches(fc):
    """Grouped tensor-core form: prep, coefficients, pack, count, scan, scatter,
    contraction, finalize; per corner: prep, coefficients, pack, contraction,
    finalize.  Workload 4 takes the pruned-FFT form automatically (measured
    0.044 ms against 0.075 for either tensor-core form): prep, count, scan,
    scatter, tables (with the transposed cotangent), FFTs, dots."""
    clip, K = config_clip(4)
    x, y, s = dev(clip.x), dev(clip.y), dev(clip.s)
    dF = torch.zeros((2 * K + 1, 2 * K + 1), dtype=torch.complex64, device="cuda")
    n0 = fc.launch_count()
    fc.adjoint(x, y, s, clip.T, K, dF, prec="split_f16")
    assert fc.launch_count() - n0 == 7
    try:
        for mode, n in ((0, 5), (2, 8)):
            fc.set_hybrid(mode)
            n0 = fc.launch_count()
            fc.adjoint(x, y, s, clip.T, K, dF, prec="split_f16")
            assert fc.launch_count() - n0 == n, mode
    finally:
        fc.set_hybrid(1)
