"""Continuous Haar transform on the GPU (through the C ABI) against the PCHT
oracle: every coefficient is an integer times a power of two, so the bar is
bit-exact equality."""
import numpy as np
import pytest
import torch

from oracle import haar
import oracle
from synth import config_clip, make_clip, clip_from_rings, rect_ring

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    from paper_1010_5562_gb300 import build as B
    B.build()
    from paper_1010_5562_gb300 import fcfs
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return fcfs


def to_dev(clip):
    return (torch.from_numpy(clip.x).cuda(), torch.from_numpy(clip.y).cuda(),
            torch.from_numpy(clip.s).cuda())


def gpu_haar(fc, clip, J):
    x, y, s = to_dev(clip)
    ws = fc.alloc_workspace(fc.haar_workspace_size(clip.V, clip.T, J), x.device)
    out = torch.full((1 << J, 1 << J), float("nan"), dtype=torch.float64, device="cuda")
    W = fc.haar(x, y, s, clip.T, J, out=out, workspace=ws)
    torch.cuda.synchronize()
    assert fc.get_status(ws) == "FCFS_OK"
    return W


CASES = [
    # (T, polygons, seed, smin, smax, J): tile passes for 2^J = 16 .. 4096
    (16, 4, 61, 1, 3, 4),         # one 16 x 16 tile
    (64, 12, 62, 3, 14, 6),       # one pass of 32 x 32 tiles, then a 2 x 2 grid
    (256, 40, 63, 4, 30, 8),      # 8 x 8 tiles, then one
    (1024, 300, 64, 6, 40, 10),   # 32 x 32 tiles
    (2048, 500, 65, 8, 60, 11),   # 64 x 64 tiles, then 2 x 2, then one
    (256, 40, 63, 4, 30, 3),      # coarse: cells 32 x 32, corners inside cells
    (4096, 600, 66, 8, 100, 7),   # coarse: cells of side 32
    (65536, 300, 67, 20, 2000, 9),  # cells of side 128 on the largest period
]


@pytest.mark.parametrize("case", CASES, ids=[f"T{c[0]}_J{c[5]}" for c in CASES])
def test_haar_bit_exact(fc, case):
    T, n, seed, smin, smax, J = case
    clip = make_clip(T, n, seed, smin=smin, smax=smax)
    W = gpu_haar(fc, clip, J).cpu().numpy()
    ref = haar.pcht(clip.x, clip.y, clip.poly_offsets, T, J)
    assert np.array_equal(W, ref), float(np.max(np.abs(W - ref)))


def test_haar_every_level_of_a_tiny_tile(fc):
    clip = make_clip(16, 4, 61, smin=1, smax=3)
    for J in range(5):
        W = gpu_haar(fc, clip, J).cpu().numpy()
        assert np.array_equal(W, haar.pcht(clip.x, clip.y, clip.poly_offsets, 16, J)), J


def test_haar_wide_cells(fc):
    """Cells wider than 1024 (Z and the tile pyramid in 64-bit integers) and the
    boundary w = 1024 (the widest cells on the 32-bit path)."""
    clip = make_clip(8192, 200, 68, smin=20, smax=400)
    for J in range(5):   # w = 8192 .. 512
        W = gpu_haar(fc, clip, J).cpu().numpy()
        assert np.array_equal(W, haar.pcht(clip.x, clip.y, clip.poly_offsets, 8192, J)), J
    clip = make_clip(65536, 300, 67, smin=20, smax=2000)
    for J in (0, 1, 5, 6):   # w = 65536 (splat weights up to 2^32), 32768, 2048, 1024
        W = gpu_haar(fc, clip, J).cpu().numpy()
        assert np.array_equal(W, haar.pcht(clip.x, clip.y, clip.poly_offsets, 65536, J)), J


def test_haar_workload2_clip(fc):
    """The T = 4096 bench clip (2000 polygons) at full depth J = 12: 16.8M
    coefficients, bit-exact; Parseval gives the area."""
    clip, _ = config_clip(2)
    W = gpu_haar(fc, clip, 12).cpu().numpy()
    ref = haar.pcht(clip.x, clip.y, clip.poly_offsets, clip.T, 12)
    assert np.array_equal(W, ref)
    A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    assert abs(float(np.sum(W * W)) - A) / A < 1e-12


def test_haar_border_and_empty(fc):
    T = 64
    c = clip_from_rings(T, [rect_ring(59, 0, 64, 64), rect_ring(3, 50, 20, 64)])
    for J in (6, 3):
        W = gpu_haar(fc, c, J).cpu().numpy()
        assert np.array_equal(W, haar.pcht(c.x, c.y, c.poly_offsets, T, J))
    x = torch.zeros(0, dtype=torch.int32, device="cuda")
    s = torch.zeros(0, dtype=torch.int8, device="cuda")
    W = fc.haar(x, x, s, 256, 8)
    torch.cuda.synchronize()
    assert torch.all(W == 0)


def test_haar_dense_band(fc):
    """A band of 32 cell rows holding more splats than the banded kernel stages
    in shared memory (8192 corners in the first 32 x 256 cells): its chunks are
    splatted straight from the corners; the other bands are staged."""
    rings = [rect_ring(2 * i, 2 * j, 2 * i + 1, 2 * j + 1) for i in range(16) for j in range(128)]
    rings += [rect_ring(100, 40, 900, 1700), rect_ring(1500, 3, 2047, 2048)]
    c = clip_from_rings(2048, rings)
    W = gpu_haar(fc, c, 11).cpu().numpy()
    assert np.array_equal(W, haar.pcht(c.x, c.y, c.poly_offsets, 2048, 11))


@pytest.mark.parametrize("J,scale", [(13, 8), (14, 4)])
def test_haar_banded_chunks_parseval(fc, J, scale):
    """Grids of 2^13 and 2^14 cells a side on T = 65536 (several 256-column
    chunks per CTA, row carries across them): with every coordinate a multiple
    of the cell side each cell is wholly inside or outside, the level-J
    projection is the image, and Parseval gives the area over all 2^2J
    coefficients; W[0][0] = area / T."""
    import dataclasses
    base = make_clip(65536 // scale, 30000, 70 + J, smin=2, smax=60)
    clip = dataclasses.replace(base, T=65536, x=base.x * scale, y=base.y * scale)
    A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    W = gpu_haar(fc, clip, J)
    assert abs(float(torch.sum(W * W)) - A) / A < 1e-12
    assert float(W[0, 0]) == A / 65536


def test_haar_deterministic_and_launches(fc):
    clip = make_clip(1024, 300, 64, smin=6, smax=40)
    x, y, s = to_dev(clip)
    ws = fc.alloc_workspace(fc.haar_workspace_size(clip.V, clip.T, 10), x.device)
    n0 = fc.launch_count()
    W1 = fc.haar(x, y, s, clip.T, 10, workspace=ws).clone()
    assert fc.launch_count() - n0 == 7   # grouping by x (3), band sums, band scan, bands, 32 x 32 grid
    W2 = fc.haar(x, y, s, clip.T, 10, workspace=ws)
    torch.cuda.synchronize()
    assert torch.equal(W1, W2)


def test_haar_largest_grid_sampled(fc):
    """T = 65536, ~0.95M corners, J = 14 (2^28 coefficients; the launch
    configuration of the large Haar workload): sampled coefficients of every
    level against Alg. 1 evaluated over all horizontal edges of the clip."""
    clip, _ = config_clip(5)
    T, J = clip.T, 14
    W = gpu_haar(fc, clip, J)
    xs, x1s, ys = [], [], []
    for m in range(clip.n_polys):
        a, b = int(clip.poly_offsets[m]), int(clip.poly_offsets[m + 1])
        e0, e1, ey = haar.horizontal_edges(clip.x[a:b], clip.y[a:b])
        xs.append(e0), x1s.append(e1), ys.append(ey)
    edges = (np.concatenate(xs), np.concatenate(x1s), np.concatenate(ys))
    rng = np.random.default_rng(9)
    picks = [(0, 0)]
    for j in (0, 1, 5, 9, 12, 13):
        for _ in range(3):
            kx, ky = (int(v) for v in rng.integers(0, 1 << j, 2))
            band = int(rng.integers(0, 3))
            P = 1 << j
            picks.append(((P + kx, ky), (kx, P + ky), (P + kx, P + ky))[band])
    # a dense neighbourhood at the finest level, where most coefficients are nonzero near edges
    picks += [((1 << 13) + 5000 + i, 7000) for i in range(4)]
    idx = torch.tensor([a * (1 << J) + b for a, b in picks], device="cuda")
    got = W.reshape(-1)[idx].cpu().numpy()
    for (a, b), g in zip(picks, got):
        if a == 0 and b == 0:
            ref = haar.intersection_area(edges, 0, T, 0, T) / T
        else:
            j = max(int(np.log2(a)) if a else 0, int(np.log2(b)) if b else 0)
            P, side = 1 << j, T >> (j + 1)
            kx, ky = (a - P if a >= P else a), (b - P if b >= P else b)
            A = [[haar.intersection_area(edges, (2 * kx + n) * side, (2 * kx + n + 1) * side,
                                         (2 * ky + m) * side, (2 * ky + m + 1) * side) for m in (0, 1)] for n in (0, 1)]
            sx = 1 if a >= P else 0
            sy = 1 if b >= P else 0
            num = sum(A[n][m] * (-1 if (sx and n) else 1) * (-1 if (sy and m) else 1) for n in (0, 1) for m in (0, 1))
            ref = num * 2.0 ** (j - 16)
        assert g == ref, ((a, b), g, ref)
