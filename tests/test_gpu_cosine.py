"""Continuous cosine series on the GPU (through the C ABI) against the FP64 oracle.

C(k, l) = integral of the clip image times cos(pi k x / T) cos(pi l y / T),
0 <= k, l <= K.  Error measure and bounds as for the Fourier block:
max |C_gpu - C_oracle| / area <= 1e-6 (plain FP32) or 1e-5 (split FP16); the
area and C(0,0) = float32(area) exact.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import config_clip, make_clip, clip_from_rings, rect_ring

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-6, "split_f16": 1e-5}
PRECS = ["fp32", "split_f16"]


@pytest.fixture(scope="module")
def fc():
    from paper_1010_5562_gb300 import build as B
    B.build()
    from paper_1010_5562_gb300 import fcfs
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    fcfs.set_splits(0)
    return fcfs


def to_dev(clip):
    return (torch.from_numpy(clip.x).cuda(), torch.from_numpy(clip.y).cuda(),
            torch.from_numpy(clip.s).cuda())


def gpu_cos(fc, clip, K, prec, splits=0):
    x, y, s = to_dev(clip)
    fc.set_splits(splits)
    try:
        ws = fc.alloc_workspace(fc.cosine_workspace_size(clip.V, clip.T, K, prec), x.device)
        out = torch.full((K + 1, K + 1), float("nan"), dtype=torch.float32, device="cuda")
        C, a = fc.cosine(x, y, s, clip.T, K, prec=prec, out=out, workspace=ws)
        torch.cuda.synchronize()
        assert fc.get_status(ws) == "FCFS_OK"
    finally:
        fc.set_splits(0)
    return C.cpu().numpy().astype(np.float64), int(a.item())


def check(fc, clip, K, prec):
    Cg, area = gpu_cos(fc, clip, K, prec)
    A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    assert area == A
    assert np.all(np.isfinite(Cg)), "block not fully written"
    assert Cg[0, 0] == np.float32(A)
    Co = oracle.cosine_block(clip.x, clip.y, clip.s, clip.T, K)
    err = np.max(np.abs(Cg - Co)) / max(A, 1)
    assert err <= TOL[prec], (prec, err)
    return err


CASES = [
    # (T, polygons, seed, smin, smax, K)
    (256, 40, 41, 4, 30, 128),        # K = 128: half a pair tile
    (1024, 300, 42, 6, 40, 200),      # ragged tiles
    (2048, 500, 43, 8, 60, 129),      # odd K: odd row stride of the partials
    (4096, 600, 44, 8, 100, 256),     # one full pair tile; full-period table (2T = 8192)
    (8192, 800, 45, 20, 200, 300),    # quarter-wave tables (2T = 16384), two tile rows
    (32768, 400, 46, 20, 2000, 64),   # largest period (2T = 65536)
    (16, 4, 47, 1, 3, 40),            # tiny period, K > T
    (64, 10, 48, 2, 10, 1),           # K = 1
]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", CASES, ids=[f"T{c[0]}_K{c[5]}" for c in CASES])
def test_cosine_matches_oracle(fc, case, prec):
    T, n, seed, smin, smax, K = case
    check(fc, make_clip(T, n, seed, smin=smin, smax=smax), K, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_cosine_workload2_clip(fc, prec):
    """The T = 4096 clip of the bench workload (V = 12576), K = 256."""
    clip, K = config_clip(2)
    check(fc, clip, K, prec)


@pytest.mark.parametrize("splits", [1, 3, 8])
def test_cosine_split_counts(fc, splits):
    clip = make_clip(1024, 300, 42, smin=6, smax=40)
    K = 200
    Cg, A = gpu_cos(fc, clip, K, "split_f16", splits=splits)
    Co = oracle.cosine_block(clip.x, clip.y, clip.s, clip.T, K)
    assert np.max(np.abs(Cg - Co)) / A <= TOL["split_f16"]


def test_cosine_against_fourier_block(fc):
    """cos a cos b = (cos(a + b) + cos(a - b)) / 2: the cosine block equals
    Re(F_2T(k, l) + F_2T(k, -l)) / 2 of the GPU Fourier block at period 2T
    (two different contractions: sine rows only vs. cos/sin row pairs)."""
    clip, K = config_clip(2)
    Cg, A = gpu_cos(fc, clip, K, "split_f16")
    x, y, s = to_dev(clip)
    F, a2 = fc.forward(x, y, s, 2 * clip.T, K, prec="split_f16")
    F = F.cpu().numpy().astype(np.complex128)
    ref = 0.5 * np.real(F[K:, K:] + F[K:, K::-1])
    assert int(a2.item()) == A
    assert np.max(np.abs(Cg - ref)) / A <= 2e-5


def test_cosine_deterministic(fc):
    clip, K = config_clip(2)
    C1, _ = gpu_cos(fc, clip, K, "split_f16")
    C2, _ = gpu_cos(fc, clip, K, "split_f16")
    assert np.array_equal(C1, C2)


def test_cosine_axis_lines_exact_sums(fc):
    """Row 0 and column 0 come from exact integer sums: far inside the bound."""
    clip = make_clip(2048, 500, 43, smin=8, smax=60)
    K = 129
    Co = oracle.cosine_block(clip.x, clip.y, clip.s, clip.T, K)
    for prec in PRECS:
        Cg, A = gpu_cos(fc, clip, K, prec)
        e = max(np.max(np.abs(Cg[0, :] - Co[0, :])), np.max(np.abs(Cg[:, 0] - Co[:, 0]))) / A
        assert e <= 1e-7, (prec, e)


@pytest.mark.parametrize("prec", PRECS)
def test_cosine_empty_and_single_rectangle(fc, prec):
    T, K = 512, 100
    x = torch.zeros(0, dtype=torch.int32, device="cuda")
    s = torch.zeros(0, dtype=torch.int8, device="cuda")
    C, a = fc.cosine(x, x, s, T, K, prec=prec)
    torch.cuda.synchronize()
    assert int(a.item()) == 0 and torch.all(C == 0)
    # the whole square: orthogonality leaves T^2 at (0, 0) only
    sq = clip_from_rings(T, [rect_ring(0, 0, T, T)])
    Cg, A = gpu_cos(fc, sq, K, prec)
    assert A == T * T and Cg[0, 0] == T * T
    Cg[0, 0] = 0.0
    assert np.max(np.abs(Cg)) / A <= TOL[prec]


def test_cosine_launches(fc):
    """prep, contraction, axis DFT, reduction."""
    clip, K = config_clip(2)
    x, y, s = to_dev(clip)
    for prec in PRECS:
        ws = fc.alloc_workspace(fc.cosine_workspace_size(clip.V, clip.T, K, prec), x.device)
        n0 = fc.launch_count()
        fc.cosine(x, y, s, clip.T, K, prec=prec, workspace=ws)
        assert fc.launch_count() - n0 == 4


def test_cosine_workspace_too_small(fc):
    clip, K = config_clip(2)
    x, y, s = to_dev(clip)
    need = fc.cosine_workspace_size(clip.V, clip.T, K, "split_f16")
    ws = fc.alloc_workspace(need - 256, x.device)
    with pytest.raises(fc.FCFSError):
        fc.cosine(x, y, s, clip.T, K, prec="split_f16", workspace=ws)


def test_cosine_largest_period_sampled(fc):
    """T = 32768 (sines of period 65536), ~126k corners, K = 1024, in the launch
    configuration of a large call: sampled entries against the oracle, which
    evaluates them one by one, including the axis lines and the +-K edges."""
    clip = make_clip(32768, 20000, 31, smin=20, smax=1500)
    K = 1024
    Cg, A = gpu_cos(fc, clip, K, "split_f16")
    assert A == oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    assert np.all(np.isfinite(Cg))
    rng = np.random.default_rng(5)
    pick = np.unique(np.concatenate([[0, 1, 2, K - 1, K], rng.integers(0, K + 1, 27)]))
    Co = oracle.cosine_entries(clip.x, clip.y, clip.s, clip.T, pick, pick)
    err = np.max(np.abs(Cg[np.ix_(pick, pick)] - Co)) / A
    assert err <= TOL["split_f16"], err
