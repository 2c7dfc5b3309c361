"""The forward entry point for callers that cannot allocate device memory.

fcfs_forward_noalloc runs the same transform as fcfs_forward but takes no
workspace: its scratch is a fixed array inside the library.  It is meant for
code that cannot call cudaMalloc where it needs the transform (a plugin whose
host framework owns all device memory, a real-time loop that must not stall
on an allocation).  Its blocks are checked against the FP64 oracle, two calls
in a row (the second reuses what the first left in the array), including
clips whose automatic split count does not fit the array and runs shrunk.
This file is collected last and also runs alone.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import config_clip

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-6, "split_f16": 1e-5}
PREC = {"fp32": 0, "split_f16": 1}


@pytest.fixture(scope="module")
def lib():
    from paper_1010_5562_gb300 import build as B
    B.build()
    from paper_1010_5562_gb300 import _lib
    assert torch.cuda.is_available()
    return _lib.load()


def _noalloc(lib, x, y, s, T, K, prec):
    W = 2 * K + 1
    F = torch.full((W, W), float("nan"), dtype=torch.complex64, device="cuda")
    area = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    code = lib.fcfs_forward_noalloc(x.data_ptr(), y.data_ptr(), s.data_ptr(), x.numel(), T, K, PREC[prec], 0,
                                    F.data_ptr(), area.data_ptr(), stream)
    assert code == 0, code
    assert lib.fcfs_noalloc_status(stream) == 0
    return F.cpu().numpy().astype(np.complex128), int(area.item())


@pytest.mark.parametrize("prec", ["fp32", "split_f16"])
@pytest.mark.parametrize("cfg", [1, 2])
def test_noalloc_matches_oracle_twice(lib, prec, cfg):
    clip, K = config_clip(cfg)
    x, y, s = (torch.from_numpy(a).cuda() for a in (clip.x, clip.y, clip.s))
    Fo = oracle.block(clip.x, clip.y, clip.s, clip.T, K)
    A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    for _ in range(2):   # the second call reuses the array the first one left behind
        F, area = _noalloc(lib, x, y, s, clip.T, K, prec)
        assert area == A
        assert np.all(np.isfinite(F))
        assert np.max(np.abs(F - Fo)) / A <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "split_f16"])
def test_noalloc_shrinks_the_split_count(lib, prec):
    """64 forced vertex splits of the T = 4096, K = 256 clip need 64 MiB of
    partial planes: the call runs with as many splits as the array holds."""
    clip, K = config_clip(2)
    x, y, s = (torch.from_numpy(a).cuda() for a in (clip.x, clip.y, clip.s))
    Fo = oracle.block(clip.x, clip.y, clip.s, clip.T, K)
    A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    lib.fcfs_debug_set_splits(64)
    try:
        for _ in range(2):
            F, area = _noalloc(lib, x, y, s, clip.T, K, prec)
            assert area == A
            assert np.max(np.abs(F - Fo)) / A <= TOL[prec]
    finally:
        lib.fcfs_debug_set_splits(0)


def test_noalloc_large_block_one_split(lib):
    """K = 1024 on the T = 4096 clip: 16 MiB per split, so only one split fits
    beside the tables; sampled rows against the oracle, then a smaller K again
    (the array's tables and tag from the K = 1024 call are reused)."""
    clip, _ = config_clip(2)
    K = 1024
    x, y, s = (torch.from_numpy(a).cuda() for a in (clip.x, clip.y, clip.s))
    A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    rows = np.array([-K, -K + 1, -517, -64, -1, 0, 1, 2, 255, 700, K - 1, K])
    Fo = oracle.block_entries(clip.x, clip.y, clip.s, clip.T, rows, oracle.freqs(K))
    for _ in range(2):
        F, area = _noalloc(lib, x, y, s, clip.T, K, "split_f16")
        assert area == A
        assert np.all(np.isfinite(F))
        assert np.max(np.abs(F[rows + K, :] - Fo)) / A <= TOL["split_f16"]
    Ks = 64
    F, area = _noalloc(lib, x, y, s, clip.T, Ks, "fp32")
    Fo = oracle.block(clip.x, clip.y, clip.s, clip.T, Ks)
    assert area == A and np.max(np.abs(F - Fo)) / A <= TOL["fp32"]


def test_noalloc_rejects_what_does_not_fit(lib):
    clip, _ = config_clip(1)
    x, y, s = (torch.from_numpy(a).cuda() for a in (clip.x, clip.y, clip.s))
    F = torch.empty((1, 2), dtype=torch.complex64, device="cuda")
    area = torch.zeros(1, dtype=torch.int64, device="cuda")
    code = lib.fcfs_forward_noalloc(x.data_ptr(), y.data_ptr(), s.data_ptr(), x.numel(), 256, 4096, 1, 0,
                                    F.data_ptr(), area.data_ptr(), None)
    assert code == 6     # FCFS_EUNSUPPORTED: even one vertex split exceeds the array
    code = lib.fcfs_forward_noalloc(x.data_ptr(), y.data_ptr(), s.data_ptr(), x.numel(), 256, 8, 1, 1,
                                    F.data_ptr(), area.data_ptr(), None)
    assert code == 1     # FCFS_EINVAL: no flags on this entry point
